"""FP64 CPU oracle for SMC with a ChEES-HMC proposal (arXiv 2504.02627).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The oracle is plain C
(``oracle/*.c``) compiled to ``liboracle.so`` and wrapped here with ctypes; it
shares no code with the CUDA library.  Arrays are numpy, particle-major
``[N, D]`` (particle j's coordinates contiguous).

Each wrapper names the passage of the paper it follows; the pins that fix each
function independently live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["rng.c", "targets.c", "hmc.c", "weights.c", "chees.c", "smc.c", "flow.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

GAUSS_DENSE, LOGISTIC, HIER_NORMAL, BANANA, LINEAR_GAUSS = 0, 1, 2, 3, 4
TAG_INIT, TAG_MOM, TAG_RESAMPLE, TAG_MH = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP contraction off: identical bits on
    x86-64 and aarch64).  OpenMP is used when the compiler has it."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
    cs = [os.path.join(_HERE, s) for s in _SOURCES]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp"] + cs + ["-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + cs + ["-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Target(C.Structure):
    _fields_ = [("kind", C.c_int32), ("D", C.c_int64), ("n", C.c_int64),
                ("X", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("P", C.POINTER(C.c_double)),
                ("c", C.c_double), ("hyper", C.c_double * 4)]


class Config(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_iters", C.c_int64), ("n_warmup", C.c_int64),
                ("step_size", C.c_double), ("traj_len0", C.c_double),
                ("max_steps", C.c_int32), ("ess_frac", C.c_double), ("seed", C.c_uint64),
                ("jitter", C.c_int32), ("accept_reject", C.c_int32), ("adapt", C.c_int32),
                ("chees_initial_p", C.c_int32), ("adam_lr", C.c_double),
                ("adam_b1", C.c_double), ("adam_b2", C.c_double), ("adam_eps", C.c_double),
                ("init_scale", C.c_double), ("flow_train_every", C.c_int32), ("flow_epochs", C.c_int32),
                ("flow_lr", C.c_double), ("flow_min_ess", C.c_double),
                ("step_adapt_rate", C.c_double), ("step_adapt_target", C.c_double),
                ("resample_scheme", C.c_int32), ("mcmc", C.c_int32),
                ("init_mean", C.POINTER(C.c_double)), ("init_chol", C.POINTER(C.c_double))]


class Stats(C.Structure):
    _fields_ = [("ess", C.c_double), ("ess_pre", C.c_double), ("log_z_inc", C.c_double),
                ("mean_alpha", C.c_double), ("traj_len", C.c_double),
                ("grad_evals", C.c_int64), ("steps_min", C.c_int32),
                ("steps_max", C.c_int32), ("resampled", C.c_int32), ("pad", C.c_int32)]


class CheesState(C.Structure):
    _fields_ = [("log_L", C.c_double), ("m", C.c_double), ("v", C.c_double),
                ("t", C.c_int32), ("Lbar", C.c_double)]


_DP = C.POINTER(C.c_double)
_I32P = C.POINTER(C.c_int32)
_U64P = C.POINTER(C.c_uint64)


class IterIO(C.Structure):
    _fields_ = [("theta", _DP), ("grad", _DP), ("logpi", _DP), ("logw", _DP),
                ("chees", C.POINTER(CheesState)), ("log_z", _DP),
                ("ancestors", _I32P), ("steps", _I32P), ("p0", _DP), ("p1", _DP),
                ("dH", _DP), ("alpha", _DP), ("flow_params", _DP), ("flow_m", _DP), ("flow_v", _DP),
                ("flow_t", C.POINTER(C.c_int32)), ("flow_H", C.c_int64), ("flow_L", C.c_int64),
                ("eps", _DP)]


class Flow(C.Structure):
    _fields_ = [("D", C.c_int64), ("H", C.c_int64), ("L", C.c_int64), ("params", _DP)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.oracle_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.c_uint64, C.POINTER(C.c_uint32)]
        L.oracle_u01.argtypes = [C.c_uint32, C.c_uint32]
        L.oracle_u01.restype = C.c_double
        L.oracle_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, _DP]
        L.oracle_resample_r64.argtypes = [C.c_uint64, C.c_uint32]
        L.oracle_resample_r64.restype = C.c_uint64
        L.oracle_multinomial_u64.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        L.oracle_multinomial_u64.restype = C.c_uint64
        L.oracle_jitter.argtypes = [C.c_int32, C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_int64]
        L.oracle_jitter.restype = C.c_double
        L.oracle_nth_prime.argtypes = [C.c_int64]
        L.oracle_nth_prime.restype = C.c_int64
        L.oracle_radical_inverse.argtypes = [C.c_uint64, C.c_uint64]
        L.oracle_radical_inverse.restype = C.c_double
        L.oracle_shuffle_index.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.oracle_shuffle_index.restype = C.c_uint32
        L.oracle_halton2.argtypes = [C.c_uint32]
        L.oracle_halton2.restype = C.c_double
        L.oracle_step_count.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32]
        L.oracle_step_count.restype = C.c_int32
        L.oracle_logpi.argtypes = [C.POINTER(Target), _DP, _DP]
        L.oracle_logpi.restype = C.c_double
        L.oracle_hamiltonian.argtypes = [_DP, C.c_int64, C.c_double]
        L.oracle_hamiltonian.restype = C.c_double
        L.oracle_leapfrog.argtypes = [C.POINTER(Target), _DP, _DP, _DP, _DP, C.c_double, C.c_int32]
        L.oracle_normalise.argtypes = [_DP, C.c_int64, _DP, _DP, _DP]
        L.oracle_quantise.argtypes = [_DP, C.c_int64, _U64P]
        L.oracle_quantise.restype = C.c_int32
        L.oracle_systematic.argtypes = [_U64P, C.c_int64, C.c_uint64, _I32P]
        L.oracle_systematic.restype = C.c_uint64
        L.oracle_multinomial.argtypes = [_U64P, C.c_int64, _U64P, _I32P]
        L.oracle_chees_gradient.argtypes = [_DP, _DP, _DP, _DP, _DP, C.c_int64, C.c_int64, _DP, _DP]
        L.oracle_chees_gradient.restype = C.c_int
        L.oracle_harmonic_mean_alpha.argtypes = [_DP, C.c_int64]
        L.oracle_harmonic_mean_alpha.restype = C.c_double
        L.oracle_step_size_update.argtypes = [C.c_double, _DP, C.c_int64, C.c_double, C.c_double]
        L.oracle_step_size_update.restype = C.c_double
        L.oracle_chees_adam.argtypes = [C.POINTER(CheesState), C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_int32]
        L.oracle_smc_init.argtypes = [C.POINTER(Target), C.POINTER(Config), _DP, _DP, _DP, _DP, C.c_int32]
        L.oracle_smc_init.restype = C.c_double
        L.oracle_smc_iteration.argtypes = [C.POINTER(Target), C.POINTER(Config), C.c_int64,
                                           C.POINTER(IterIO), C.POINTER(Stats), C.c_int32]
        L.oracle_smc_iteration.restype = C.c_int
        L.oracle_smc_run.argtypes = [C.POINTER(Target), C.POINTER(Config), _DP, _DP, _DP,
                                     C.POINTER(Stats), C.c_int32]
        L.oracle_smc_run.restype = C.c_int
        L.oracle_moments.argtypes = [_DP, _DP, C.c_int64, C.c_int64, _DP, _DP]
        L.oracle_flow_num_params.argtypes = [C.c_int64, C.c_int64, C.c_int64]
        L.oracle_flow_num_params.restype = C.c_int64
        L.oracle_flow_forward.argtypes = [C.POINTER(Flow), _DP, _DP, _DP]
        L.oracle_flow_inverse.argtypes = [C.POINTER(Flow), _DP, _DP, _DP]
        L.oracle_flow_logpi_z.argtypes = [C.POINTER(Flow), C.POINTER(Target), _DP, _DP, _DP, _DP, _DP]
        L.oracle_flow_logpi_z.restype = C.c_double
        L.oracle_flow_loss_grad.argtypes = [C.POINTER(Flow), _DP, _DP, C.c_int64, _DP]
        L.oracle_flow_loss_grad.restype = C.c_double
        L.oracle_flow_adam.argtypes = [_DP, _DP, _DP, _DP, C.c_int64, C.c_int32, C.c_double, C.c_double,
                                       C.c_double, C.c_double]
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- targets
class TargetSpec:
    """Owns the numpy arrays behind an ``oracle_target`` struct (Sec. 2)."""

    def __init__(self, kind, D, n=0, X=None, y=None, mu=None, P=None, c=0.0, hyper=()):
        self.kind, self.D, self.n = int(kind), int(D), int(n)
        self.X = None if X is None else _f64(X)
        self.y = None if y is None else _f64(y)
        self.mu = None if mu is None else _f64(mu)
        self.P = None if P is None else _f64(P)
        h = list(hyper) + [0.0] * (4 - len(hyper))
        self.struct = Target(self.kind, self.D, self.n, _dp(self.X), _dp(self.y), _dp(self.mu),
                             _dp(self.P), float(c), (C.c_double * 4)(*h))

    @staticmethod
    def gauss_dense(mu, P, c=0.0):
        mu = _f64(mu)
        return TargetSpec(GAUSS_DENSE, mu.size, mu=mu, P=P, c=c)

    @staticmethod
    def logistic(X, y, tau=1.0):
        X = _f64(X)
        return TargetSpec(LOGISTIC, X.shape[1], X.shape[0], X=X, y=y, hyper=(tau,))

    @staticmethod
    def linear_gauss(X, y, sigma=1.0, tau=1.0):
        X = _f64(X)
        return TargetSpec(LINEAR_GAUSS, X.shape[1], X.shape[0], X=X, y=y, hyper=(sigma, tau))

    @staticmethod
    def hier_normal(ybar, n_g, ss, sigma=1.0):
        ybar = _f64(ybar)
        return TargetSpec(HIER_NORMAL, 2 + ybar.size, ybar.size, y=ybar, mu=n_g, P=ss,
                          hyper=(sigma,))

    @staticmethod
    def banana(D, a, b):
        return TargetSpec(BANANA, D, hyper=(a, b))


def logpi(t: TargetSpec, theta):
    """log pi and its gradient for each row of ``theta`` ([N, D] or [D])."""
    th = _f64(np.atleast_2d(theta))
    g = np.empty_like(th)
    lp = np.empty(th.shape[0])
    for j in range(th.shape[0]):
        row = th[j]
        gr = g[j]
        lp[j] = lib().oracle_logpi(C.byref(t.struct), _dp(row), _dp(gr))
    return lp, g


def leapfrog(t: TargetSpec, theta, p, eps, steps):
    """``steps`` leapfrog steps (Algorithm 1) for every row; returns
    (theta, p, grad, logpi) after the trajectory."""
    th = _f64(np.atleast_2d(theta)).copy()
    pp = _f64(np.atleast_2d(p)).copy()
    lp, g = logpi(t, th)
    steps = np.broadcast_to(np.asarray(steps, dtype=np.int64), (th.shape[0],))
    for j in range(th.shape[0]):
        lpj = C.c_double(lp[j])
        r_th, r_p, r_g = th[j], pp[j], g[j]
        lib().oracle_leapfrog(C.byref(t.struct), _dp(r_th), _dp(r_p), _dp(r_g), C.byref(lpj),
                              float(eps), int(steps[j]))
        lp[j] = lpj.value
    return th, pp, g, lp


def hamiltonian(p, logpi_value):
    p = _f64(p)
    return lib().oracle_hamiltonian(_dp(p), p.size, float(logpi_value))


# ---------------------------------------------------------------- rng
def philox(ctr, seed):
    """Philox4x32-10 block for a counter (4 x uint32) and 64-bit seed."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    out = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, C.c_uint64(int(seed)), out)
    return np.array(list(out), dtype=np.uint32)


def u01(w0, w1):
    return lib().oracle_u01(int(w0), int(w1))


def normals(seed, tag, k, j, D):
    out = np.empty(D)
    lib().oracle_normals(C.c_uint64(int(seed)), tag, k, j, D, _dp(out))
    return out


def resample_r64(seed, k):
    return int(lib().oracle_resample_r64(C.c_uint64(int(seed)), int(k)))


def multinomial_u64(seed, k, i):
    return int(lib().oracle_multinomial_u64(C.c_uint64(int(seed)), int(k), int(i)))


# jitter schemes (Sec. 3.2.1): names of the `jitter` values
JITTER = {"none": 0, "halton1": 1, "uniform": 2, "halton_nd": 3, "halton_nd_inv": 4, "primes": 5,
          "primes_inv": 6, "golden": 7, "equidistant": 8, "equidistant_offset": 9, "sobol1": 10,
          "halton1_iter": 11}


def jitter(scheme, seed, j, k, J, K):
    return lib().oracle_jitter(int(scheme), C.c_uint64(int(seed)), int(j), int(k), int(J), int(K))


def jitter_matrix(scheme, seed, J, K):
    """h [J, K] (particle j, iteration k = 1..K)."""
    return np.array([[jitter(scheme, seed, j, k, J, K) for k in range(1, K + 1)] for j in range(J)])


def nth_prime(m):
    return int(lib().oracle_nth_prime(int(m)))


def radical_inverse(n, b):
    return lib().oracle_radical_inverse(C.c_uint64(int(n)), C.c_uint64(int(b)))


def shuffle_index(seed, k, j, J):
    return int(lib().oracle_shuffle_index(C.c_uint64(int(seed)), int(k), int(j), int(J)))


def halton2(n):
    return lib().oracle_halton2(int(n))


def step_count(h, L, eps, max_steps):
    return int(lib().oracle_step_count(float(h), float(L), float(eps), int(max_steps)))


# ---------------------------------------------------------------- weights
def normalise(logw):
    lw = _f64(logw)
    lse, ess = C.c_double(), C.c_double()
    W = np.empty_like(lw)
    lib().oracle_normalise(_dp(lw), lw.size, C.byref(lse), C.byref(ess), _dp(W))
    return lse.value, ess.value, W


def quantise(W):
    W = _f64(W)
    q = np.empty(W.size, dtype=np.uint64)
    S = lib().oracle_quantise(_dp(W), W.size, q.ctypes.data_as(_U64P))
    return S, q


def systematic(q, r64):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    anc = np.empty(q.size, dtype=np.int32)
    T = lib().oracle_systematic(q.ctypes.data_as(_U64P), q.size, C.c_uint64(int(r64)),
                                anc.ctypes.data_as(_I32P))
    return int(T), anc


def multinomial(q, u64):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    u = np.ascontiguousarray(u64, dtype=np.uint64)
    anc = np.empty(q.size, dtype=np.int32)
    lib().oracle_multinomial(q.ctypes.data_as(_U64P), q.size, u.ctypes.data_as(_U64P),
                             anc.ctypes.data_as(_I32P))
    return anc


def moments(theta, logw):
    th = _f64(theta)
    lw = _f64(logw)
    N, D = th.shape
    mean, var = np.empty(D), np.empty(D)
    lib().oracle_moments(_dp(th), _dp(lw), N, D, _dp(mean), _dp(var))
    return mean, var


# ---------------------------------------------------------------- ChEES
def chees_gradient(theta0, theta1, p, l, alpha):
    t0, t1, pp = _f64(theta0), _f64(theta1), _f64(p)
    N, D = t0.shape
    l, a = _f64(l), _f64(alpha)
    g = C.c_double()
    per = np.empty(N)
    ok = lib().oracle_chees_gradient(_dp(t0), _dp(t1), _dp(pp), _dp(l), _dp(a), N, D,
                                     C.byref(g), _dp(per))
    return (g.value if ok else None), per


def harmonic_mean_alpha(alpha):
    a = _f64(alpha)
    return lib().oracle_harmonic_mean_alpha(_dp(a), a.size)


def step_size_update(eps, alpha, rate, target=0.651):
    """Optional warm-up step-size rule: log eps += rate (a_h - target)."""
    a = _f64(alpha)
    return lib().oracle_step_size_update(float(eps), _dp(a), a.size, float(rate), float(target))


def chees_adam(state: CheesState, ghat, lr, b1, b2, adam_eps, eps, max_steps):
    lib().oracle_chees_adam(C.byref(state), float(ghat), lr, b1, b2, adam_eps, eps, max_steps)
    return state


# ---------------------------------------------------------------- sampler
@dataclass
class SMCConfig:
    """Sampler settings (Algorithm 3 + Algorithm 2).  Defaults follow the
    paper where it speaks (ESS threshold J/2, 1-d Halton jitter, no
    accept-reject); the Adam constants are this project's choice."""
    n_particles: int = 256
    n_iters: int = 20
    n_warmup: int = 10
    step_size: float = 0.1
    traj_len0: float = 5.0
    max_steps: int = 500
    ess_frac: float = 0.5
    seed: int = 1000
    jitter: int = 1
    accept_reject: int = 0
    adapt: int = 1
    chees_initial_p: int = 0
    adam_lr: float = 0.025
    adam_b1: float = 0.9
    adam_b2: float = 0.999
    adam_eps: float = 1e-8
    init_scale: float = 1.0
    flow_train_every: int = 2
    flow_epochs: int = 10
    flow_lr: float = 1e-3
    flow_min_ess: float = 0.25
    step_adapt_rate: float = 0.0      # 0: fixed epsilon, as in the paper
    step_adapt_target: float = 0.651
    resample_scheme: int = 0          # 0 systematic, 1 multinomial (the paper's choice)
    mcmc: int = 0                     # 1: Algorithm 2 as independent chains (no weights)
    init_mean: Optional[np.ndarray] = None   # q_init = N(init_mean, init_chol init_chol^T)
    init_chol: Optional[np.ndarray] = None   # lower-triangular [D, D]; None: init_scale * I

    def struct(self):
        cs = Config(self.n_particles, self.n_iters, self.n_warmup, self.step_size,
                    self.traj_len0, self.max_steps, self.ess_frac, self.seed & (2**64 - 1),
                    self.jitter, self.accept_reject, self.adapt, self.chees_initial_p,
                    self.adam_lr, self.adam_b1, self.adam_b2, self.adam_eps, self.init_scale,
                    self.flow_train_every, self.flow_epochs, self.flow_lr, self.flow_min_ess,
                    self.step_adapt_rate, self.step_adapt_target, self.resample_scheme, self.mcmc)
        keep = []
        for name in ("init_mean", "init_chol"):
            a = getattr(self, name)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                setattr(cs, name, a.ctypes.data_as(C.POINTER(C.c_double)))
        cs._keep = keep          # the arrays live as long as the struct
        return cs


def stats_to_dicts(arr):
    return [{f: getattr(s, f) for f, _ in Stats._fields_ if f != "pad"} for s in arr]


def smc_run(t: TargetSpec, cfg: SMCConfig, nthreads: int = 0):
    """Whole sampler (Algorithm 3).  Returns dict with theta [N, D], logw,
    log_z, stats (list of per-iteration dicts) and status."""
    N, D, K = cfg.n_particles, t.D, cfg.n_iters
    theta = np.empty((N, D))
    logw = np.empty(N)
    lz = C.c_double()
    st = (Stats * K)()
    c = cfg.struct()
    status = lib().oracle_smc_run(C.byref(t.struct), C.byref(c), _dp(theta), _dp(logw),
                                  C.byref(lz), st, int(nthreads))
    return {"theta": theta, "logw": logw, "log_z": lz.value, "stats": stats_to_dicts(st),
            "status": status}


def smc_init(t: TargetSpec, cfg: SMCConfig, nthreads: int = 0):
    N, D = cfg.n_particles, t.D
    theta, grad = np.empty((N, D)), np.empty((N, D))
    lp, lw = np.empty(N), np.empty(N)
    c = cfg.struct()
    lz = lib().oracle_smc_init(C.byref(t.struct), C.byref(c), _dp(theta), _dp(grad), _dp(lp),
                               _dp(lw), int(nthreads))
    return {"theta": theta, "grad": grad, "logpi": lp, "logw": lw, "log_z": lz}


class FlowSpec:
    """Affine-coupling flow parameters (FP64 array, layout of oracle/flow.c)."""

    def __init__(self, D, H, L, params):
        self.D, self.H, self.L = int(D), int(H), int(L)
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        assert self.params.size == num_flow_params(D, H, L)
        self.struct = Flow(self.D, self.H, self.L, _dp(self.params))


def num_flow_params(D, H, L):
    return int(lib().oracle_flow_num_params(D, H, L))


def flow_forward(f: FlowSpec, z):
    z = _f64(np.atleast_2d(z))
    x = np.empty_like(z)
    ld = np.empty(z.shape[0])
    for j in range(z.shape[0]):
        v = C.c_double()
        lib().oracle_flow_forward(C.byref(f.struct), _dp(z[j]), _dp(x[j]), C.byref(v))
        ld[j] = v.value
    return x, ld


def flow_inverse(f: FlowSpec, x):
    x = _f64(np.atleast_2d(x))
    z = np.empty_like(x)
    ld = np.empty(x.shape[0])
    for j in range(x.shape[0]):
        v = C.c_double()
        lib().oracle_flow_inverse(C.byref(f.struct), _dp(x[j]), _dp(z[j]), C.byref(v))
        ld[j] = v.value
    return z, ld


def flow_logpi_z(f: FlowSpec, t: TargetSpec, z):
    """log pi_z(z) = log pi(T(z)) + log|det dT/dz|, its z-gradient, and x = T(z)."""
    z = _f64(np.atleast_2d(z))
    N, D = z.shape
    lpz, gz, x, gx, lpx = np.empty(N), np.empty((N, D)), np.empty((N, D)), np.empty((N, D)), np.empty(N)
    for j in range(N):
        v = C.c_double()
        lpz[j] = lib().oracle_flow_logpi_z(C.byref(f.struct), C.byref(t.struct), _dp(z[j]), _dp(gz[j]),
                                           _dp(x[j]), _dp(gx[j]), C.byref(v))
        lpx[j] = v.value
    return lpz, gz, x, gx, lpx


def flow_loss_grad(f: FlowSpec, theta, W):
    th = _f64(theta)
    W = _f64(W)
    grad = np.empty(f.params.size)
    loss = lib().oracle_flow_loss_grad(C.byref(f.struct), _dp(th), _dp(W), th.shape[0], _dp(grad))
    return loss, grad


def flow_adam(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    lib().oracle_flow_adam(_dp(params), _dp(_f64(grad)), _dp(m), _dp(v), params.size, int(t), lr, b1, b2, eps)


def smc_iteration(t: TargetSpec, cfg: SMCConfig, k: int, state: dict, nthreads: int = 0):
    """One iteration (Algorithm 3 body) on a state dict as returned by
    ``smc_init`` plus ``chees`` (CheesState), optionally ``flow`` (dict
    with params, m, v, t (c_int32), H, L) for the learned preconditioner, and
    optionally ``eps`` (c_double, the current step size; absent: the fixed
    ``cfg.step_size``).  Mutates theta/grad/logpi/logw/log_z/chees/flow/eps in
    place and returns the per-iteration intermediates."""
    N, D = cfg.n_particles, t.D
    for key in ("theta", "grad", "logpi", "logw"):
        state[key] = _f64(state[key])
    out = {"ancestors": np.empty(N, np.int32), "steps": np.empty(N, np.int32),
           "p0": np.empty((N, D)), "p1": np.empty((N, D)), "dH": np.empty(N),
           "alpha": np.empty(N)}
    lz = C.c_double(state["log_z"])
    fl = state.get("flow")
    io = IterIO(_dp(state["theta"]), _dp(state["grad"]), _dp(state["logpi"]),
                _dp(state["logw"]), C.pointer(state["chees"]), C.pointer(lz),
                out["ancestors"].ctypes.data_as(_I32P), out["steps"].ctypes.data_as(_I32P),
                _dp(out["p0"]), _dp(out["p1"]), _dp(out["dH"]), _dp(out["alpha"]),
                _dp(fl["params"]) if fl else None, _dp(fl["m"]) if fl else None,
                _dp(fl["v"]) if fl else None, C.pointer(fl["t"]) if fl else None,
                int(fl["H"]) if fl else 0, int(fl["L"]) if fl else 0,
                C.pointer(state["eps"]) if "eps" in state else None)
    st = Stats()
    c = cfg.struct()
    out["status"] = lib().oracle_smc_iteration(C.byref(t.struct), C.byref(c), int(k),
                                               C.byref(io), C.byref(st), int(nthreads))
    state["log_z"] = lz.value
    out["stats"] = stats_to_dicts([st])[0]
    return out


def new_flow_state(params, H, L):
    p = np.array(params, dtype=np.float64, copy=True)
    return {"params": p, "m": np.zeros_like(p), "v": np.zeros_like(p), "t": C.c_int32(0),
            "H": int(H), "L": int(L)}


def smc_run_flow(t: TargetSpec, cfg: SMCConfig, flow_params, H, L, nthreads: int = 0):
    """The sampler with the learned preconditioner (iteration by iteration)."""
    st = smc_init(t, cfg, nthreads)
    st["chees"] = initial_chees_state(cfg)
    st["flow"] = new_flow_state(flow_params, H, L)
    st["eps"] = C.c_double(cfg.step_size)
    stats, status = [], 0
    for k in range(1, cfg.n_iters + 1):
        out = smc_iteration(t, cfg, k, st, nthreads)
        stats.append(out["stats"])
        status = out["status"]
        if status != 0:
            break
    return {"theta": st["theta"], "logw": st["logw"], "log_z": st["log_z"], "stats": stats,
            "status": status, "flow": st["flow"]}


def initial_chees_state(cfg: SMCConfig) -> CheesState:
    lo, hi = np.log(cfg.step_size), np.log(cfg.max_steps * cfg.step_size)
    return CheesState(float(np.clip(np.log(cfg.traj_len0), lo, hi)), 0.0, 0.0, 0, 0.0)
