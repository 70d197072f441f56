"""ctypes binding of libsmcchees (include/smc.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; device
arrays are passed as raw pointers (``tensor.data_ptr()``), streams as the raw
``cudaStream_t`` value.  Loading fails loudly when the library has not been
built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SMC_OK, SMC_E_INVAL, SMC_E_NOMEM, SMC_E_CUDA, SMC_E_DEGENERATE, SMC_E_TIMEOUT, SMC_E_STATE = \
    0, -1, -2, -3, -4, -5, -6
GAUSS_DENSE, LOGISTIC, HIER_NORMAL, BANANA, LINEAR_GAUSS = 0, 1, 2, 3, 4
PREC_FP32, PREC_BF16X3, PREC_BF16, PREC_BF16X2, PREC_BF16C = 0, 1, 2, 3, 4
# trajectory-length jitter schemes (Sec. 3.2.1), smc_config.jitter
(JITTER_NONE, JITTER_HALTON1, JITTER_UNIFORM, JITTER_HALTON_ND, JITTER_HALTON_ND_INV, JITTER_PRIMES,
 JITTER_PRIMES_INV, JITTER_GOLDEN, JITTER_EQUIDISTANT, JITTER_EQUIDISTANT_OFFSET, JITTER_SOBOL1,
 JITTER_HALTON1_ITER) = range(12)
(BUF_THETA, BUF_GRAD, BUF_LOGPI, BUF_LOGW, BUF_W, BUF_ANCESTORS, BUF_STEPS, BUF_P_FINAL,
 BUF_DH, BUF_ALPHA, BUF_THETA_PREV, BUF_RUNSTATE, BUF_Z0, BUF_Z1, BUF_ORDER) = range(15)

_DP = C.POINTER(C.c_double)


class SmcModel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("dim", C.c_int64), ("n_obs", C.c_int64),
                ("X", _DP), ("y", _DP), ("mu", _DP), ("prec", _DP), ("group_mean", _DP),
                ("group_n", _DP), ("group_ss", _DP), ("c", C.c_double), ("hyper", C.c_double * 4)]


class SmcConfig(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_iters", C.c_int64), ("n_warmup", C.c_int64),
                ("step_size", C.c_double), ("traj_len0", C.c_double), ("max_steps", C.c_int32),
                ("jitter", C.c_int32), ("ess_frac", C.c_double), ("seed", C.c_uint64),
                ("accept_reject", C.c_int32), ("adapt", C.c_int32), ("adam_lr", C.c_double),
                ("adam_b1", C.c_double), ("adam_b2", C.c_double), ("adam_eps", C.c_double),
                ("init_scale", C.c_double), ("precision", C.c_int32), ("pad", C.c_int32),
                ("step_adapt_rate", C.c_double), ("step_adapt_target", C.c_double),
                ("resample_scheme", C.c_int32), ("mcmc", C.c_int32),
                ("init_mean", _DP), ("init_chol", _DP)]


class SmcFlowConfig(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("layers", C.c_int32), ("train_every", C.c_int32),
                ("epochs", C.c_int32), ("lr", C.c_double), ("min_ess_frac", C.c_double),
                ("precision", C.c_int32), ("train_precision", C.c_int32)]


class SmcStats(C.Structure):
    _fields_ = [("ess", C.c_double), ("ess_pre", C.c_double), ("log_z_inc", C.c_double),
                ("mean_alpha", C.c_double), ("traj_len", C.c_double), ("grad_evals", C.c_int64),
                ("steps_min", C.c_int32), ("steps_max", C.c_int32), ("resampled", C.c_int32),
                ("pad", C.c_int32)]


class SmcSummary(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("grad_evals", C.c_int64), ("ess_sum", C.c_double),
                ("ess_sum_post_warmup", C.c_double), ("log_z", C.c_double), ("resamples", C.c_int64)]


EXPORTS = {
    # name: (restype, argtypes)
    "smc_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(SmcConfig), C.POINTER(SmcModel), C.c_void_p]),
    "smc_init_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.POINTER(SmcConfig),
                                 C.POINTER(SmcModel), C.c_void_p]),
    "smc_step": (C.c_int, [C.c_void_p, C.POINTER(SmcStats)]),
    "smc_run": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(SmcStats)]),
    "smc_log_evidence": (C.c_int, [C.c_void_p, _DP]),
    "smc_get_particles": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "smc_moments": (C.c_int, [C.c_void_p, _DP, _DP]),
    "smc_get_buffer": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32]),
    "smc_get_layout": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "smc_last_error": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64]),
    "smc_reset": (C.c_int, [C.c_void_p, C.c_uint64]),
    "smc_get_summary": (C.c_int, [C.c_void_p, C.POINTER(SmcSummary)]),
    "smc_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "smc_get_plan": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _DP]),
    "smc_set_plan": (C.c_int, [C.c_void_p, C.c_int32]),
    "smc_get_profile": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
    "smc_destroy": (None, [C.c_void_p]),
    "smc_model_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(SmcModel), C.c_void_p]),
    "smc_model_destroy": (None, [C.c_void_p]),
    "smc_k_philox": (C.c_int, [C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "smc_k_normals": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, C.c_void_p,
                                C.c_int64, C.c_void_p]),
    "smc_k_steps": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_int32,
                              C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_k_jitter": (C.c_int, [C.c_int32, C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                               C.c_void_p]),
    "smc_k_target": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                               C.c_int32, C.c_void_p]),
    "smc_k_leapfrog": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_double, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]),
    "smc_k_normalise": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "smc_k_resample_scratch_bytes": (C.c_int64, [C.c_int64]),
    "smc_k_lookback_wait_check": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_k_resample": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "smc_k_resample_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p]),
    "smc_flow_num_params": (C.c_int64, [C.c_int64, C.c_int32, C.c_int32]),
    "smc_flow_enable": (C.c_int, [C.c_void_p, C.POINTER(SmcFlowConfig), _DP]),
    "smc_flow_get_params": (C.c_int, [C.c_void_p, _DP, C.c_int64]),
    "smc_k_flow_leapfrog": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int64, C.c_int64,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "smc_k_flow_loss_grad": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p]),
}
NOALLOC_MAX_N = 4194304     # SMC_NOALLOC_MAX_N in include/smc.h

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libsmcchees.so (building it first if allowed); raises if absent."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libsmcchees.so not built ({path}); run paper_2504_02627_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str = "", handle=None):
    if status != SMC_OK:
        msg = ""
        if handle:
            buf = C.create_string_buffer(512)
            lib().smc_last_error(handle, buf, 512)
            msg = buf.value.decode(errors="replace")
        raise RuntimeError(f"{what} failed with status {status}: {msg}")


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


class ModelData:
    """Owns the host arrays behind an ``smc_model`` struct."""

    def __init__(self, kind, dim, n_obs=0, X=None, y=None, mu=None, prec=None, group_mean=None,
                 group_n=None, group_ss=None, c=0.0, hyper=()):
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        self.arrays = [f(X), f(y), f(mu), f(prec), f(group_mean), f(group_n), f(group_ss)]
        h = list(hyper) + [0.0] * (4 - len(hyper))
        self.struct = SmcModel(int(kind), 0, int(dim), int(n_obs), *[_dp(a) for a in self.arrays],
                               float(c), (C.c_double * 4)(*h))

    @staticmethod
    def from_workload(w: dict) -> "ModelData":
        k = w["kind"]
        if k == "gauss_dense":
            return ModelData(GAUSS_DENSE, w["D"], mu=w["mu"], prec=w["P"], c=w.get("c", 0.0))
        if k == "logistic":
            return ModelData(LOGISTIC, w["D"], w["n"], X=w["X"], y=w["y"], hyper=(w.get("tau", 1.0),))
        if k == "linear_gauss":
            return ModelData(LINEAR_GAUSS, w["D"], w["n"], X=w["X"], y=w["y"],
                             hyper=(w["sigma"], w["tau"]))
        if k == "hier_normal":
            return ModelData(HIER_NORMAL, w["D"], w["n"], group_mean=w["ybar"], group_n=w["n_g"],
                             group_ss=w["ss"], hyper=(w["sigma"],))
        if k == "banana":
            return ModelData(BANANA, w["D"], hyper=(w["a"], w["b"]))
        raise ValueError(k)


def make_config(n_particles, n_iters, n_warmup, step_size, traj_len0=5.0, max_steps=500, jitter=1,
                ess_frac=0.5, seed=1000, adapt=1, adam_lr=0.025, adam_b1=0.9, adam_b2=0.999,
                adam_eps=1e-8, init_scale=1.0, precision=PREC_FP32, accept_reject=0,
                step_adapt_rate=0.0, step_adapt_target=0.651, resample_scheme=0, mcmc=0,
                init_mean=None, init_chol=None) -> SmcConfig:
    """An smc_config.  init_mean [D] / init_chol [D, D] (lower-triangular)
    give q_init = N(init_mean, init_chol init_chol^T); the arrays are kept
    alive with the struct and copied by smc_init."""
    c = SmcConfig(int(n_particles), int(n_iters), int(n_warmup), float(step_size), float(traj_len0),
                  int(max_steps), int(jitter), float(ess_frac), int(seed) & (2**64 - 1), int(accept_reject),
                  int(adapt),
                  float(adam_lr), float(adam_b1), float(adam_b2), float(adam_eps), float(init_scale),
                  int(precision), 0, float(step_adapt_rate), float(step_adapt_target),
                  int(resample_scheme), int(mcmc))
    keep = []
    for name, a in (("init_mean", init_mean), ("init_chol", init_chol)):
        if a is not None:
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            setattr(c, name, a.ctypes.data_as(_DP))
    c._keep = keep
    return c


def stats_dicts(arr):
    return [{f: getattr(s, f) for f, _ in SmcStats._fields_ if f != "pad"} for s in arr]


class Sampler:
    """One handle (``smc_init`` or ``smc_init_batch``) on a CUDA stream."""

    def __init__(self, model: ModelData, configs, stream: int = 0):
        self.model = model
        cfgs = configs if isinstance(configs, (list, tuple)) else [configs]
        self.n_runs = len(cfgs)
        self._cfg = (SmcConfig * self.n_runs)(*cfgs)
        self._cfg_keep = [getattr(c, "_keep", None) for c in cfgs]   # initial-distribution arrays
        h = C.c_void_p()
        if self.n_runs == 1:
            st = lib().smc_init(C.byref(h), self._cfg, C.byref(model.struct), C.c_void_p(stream))
        else:
            st = lib().smc_init_batch(C.byref(h), self.n_runs, self._cfg, C.byref(model.struct),
                                      C.c_void_p(stream))
        check(st, "smc_init")
        self.h = h
        ld, n, r = C.c_int64(), C.c_int64(), C.c_int64()
        lib().smc_get_layout(h, C.byref(ld), C.byref(n), C.byref(r))
        self.ld, self.n_total = ld.value, n.value
        self.dim = model.struct.dim

    def step(self, with_stats: bool = True):
        if with_stats:
            st = (SmcStats * self.n_runs)()
            check(lib().smc_step(self.h, st), "smc_step", self.h)
            return stats_dicts(st)
        check(lib().smc_step(self.h, None), "smc_step", self.h)
        return None

    def run(self, n_iters: int, with_stats: bool = False):
        if with_stats:
            st = (SmcStats * (n_iters * self.n_runs))()
            check(lib().smc_run(self.h, n_iters, st), "smc_run", self.h)
            return stats_dicts(st)
        check(lib().smc_run(self.h, n_iters, None), "smc_run", self.h)
        return None

    def reset(self, seed: int):
        check(lib().smc_reset(self.h, int(seed) & (2**64 - 1)), "smc_reset", self.h)

    def summary(self):
        out = (SmcSummary * self.n_runs)()
        check(lib().smc_get_summary(self.h, out), "smc_get_summary", self.h)
        return [{f: getattr(s, f) for f, _ in SmcSummary._fields_} for s in out]

    def profile(self, enable: bool):
        check(lib().smc_profile(self.h, int(enable)), "smc_profile", self.h)

    def get_profile(self):
        ms, n, k = C.c_double(), C.c_int64(), C.c_int64()
        check(lib().smc_get_profile(self.h, C.byref(ms), C.byref(n), C.byref(k)), "smc_get_profile",
              self.h)
        return {"traj_ms": ms.value, "traj_launches": n.value, "kernel_launches": k.value}

    def plan(self):
        """smc_get_plan: the trajectory-kernel variant the autotuner chose."""
        tile, n = C.c_int32(), C.c_int32()
        check(lib().smc_get_plan(self.h, C.byref(tile), C.byref(n), None), "smc_get_plan", self.h)
        ms = np.zeros(n.value)
        check(lib().smc_get_plan(self.h, None, None, _dp(ms)), "smc_get_plan", self.h)
        return {"traj_tile": tile.value, "n_tiles": n.value, "tile_ms": ms.tolist()}

    def set_plan(self, traj_tile: int):
        """smc_set_plan: force a trajectory-kernel variant."""
        check(lib().smc_set_plan(self.h, int(traj_tile)), "smc_set_plan", self.h)

    def log_evidence(self):
        out = np.empty(self.n_runs)
        check(lib().smc_log_evidence(self.h, _dp(out)), "smc_log_evidence", self.h)
        return out

    def particles(self):
        th = np.empty((self.dim, self.n_total), dtype=np.float32)
        lw = np.empty(self.n_total)
        check(lib().smc_get_particles(self.h, th.ctypes.data, lw.ctypes.data, 0), "smc_get_particles",
              self.h)
        return th, lw

    def moments(self):
        m, v = np.empty(self.dim), np.empty(self.dim)
        check(lib().smc_moments(self.h, _dp(m), _dp(v)), "smc_moments", self.h)
        return m, v

    def buffer(self, which: int):
        """Host copy of an internal buffer (see smc_buffer in smc.h)."""
        D, ld, N = self.dim, self.ld, self.n_total
        shapes = {BUF_THETA: ((D, ld), np.float32), BUF_GRAD: ((D, ld), np.float32),
                  BUF_P_FINAL: ((D, ld), np.float32), BUF_THETA_PREV: ((D, ld), np.float32),
                  BUF_LOGPI: ((N,), np.float64), BUF_LOGW: ((N,), np.float64),
                  BUF_W: ((N,), np.float64), BUF_DH: ((N,), np.float64),
                  BUF_ALPHA: ((N,), np.float64), BUF_ANCESTORS: ((N,), np.int32),
                  BUF_STEPS: ((N,), np.int32), BUF_RUNSTATE: ((self.n_runs, 9), np.float64),
                  BUF_Z0: ((D, ld), np.float32), BUF_Z1: ((D, ld), np.float32), BUF_ORDER: ((N,), np.int32)}
        shape, dt = shapes[which]
        out = np.empty(shape, dtype=dt)
        check(lib().smc_get_buffer(self.h, which, out.ctypes.data, out.nbytes, 0), "smc_get_buffer",
              self.h)
        if len(shape) == 2 and which != BUF_RUNSTATE:
            out = out[:, :N]
        return out

    def enable_flow(self, params, hidden: int, layers: int, train_every: int = 2, epochs: int = 10,
                    lr: float = 1e-3, min_ess_frac: float = 0.25, precision: int = 0, train_precision: int = 0):
        """smc_flow_enable: the affine-coupling transport map (FP64 host params);
        precision PREC_FP32 or PREC_BF16 (conditioner products of the
        trajectories on BF16 warp MMAs), train_precision the same for the
        training gradient's products."""
        p = np.ascontiguousarray(params, dtype=np.float64)
        n = lib().smc_flow_num_params(self.dim, hidden, layers)
        if p.size != n:
            raise ValueError(f"flow needs {n} parameters, got {p.size}")
        fc = SmcFlowConfig(hidden, layers, train_every, epochs, lr, min_ess_frac, precision, train_precision)
        check(lib().smc_flow_enable(self.h, C.byref(fc), _dp(p)), "smc_flow_enable", self.h)
        self.flow_shape = (hidden, layers)

    def flow_params(self):
        hidden, layers = self.flow_shape
        out = np.empty(lib().smc_flow_num_params(self.dim, hidden, layers))
        check(lib().smc_flow_get_params(self.h, _dp(out), out.size), "smc_flow_get_params", self.h)
        return out

    def runstate(self):
        rs = self.buffer(BUF_RUNSTATE)
        keys = ["log_z", "log_L", "adam_m", "adam_v", "Lbar", "adam_t", "L_last", "ess", "eps"]
        return [dict(zip(keys, row)) for row in rs]

    def close(self):
        if getattr(self, "h", None):
            lib().smc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DevModel:
    """Device-resident target for the kernel-level entry points."""

    def __init__(self, model: ModelData, stream: int = 0):
        self.model = model
        h = C.c_void_p()
        check(lib().smc_model_create(C.byref(h), C.byref(model.struct), C.c_void_p(stream)),
              "smc_model_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().smc_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
