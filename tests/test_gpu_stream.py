"""GPU parity of the streamed tensor-core trajectory kernel (data that do not
fit on chip: X streamed chunk by chunk through shared memory) against the
FP64 oracle, through the C-ABI.

The kernel rounds X once to BF16 -- a fixed perturbation of the data the
integrator sees -- so its gradients and trajectories are compared with the
oracle run on the same BF16-rounded data; what is left is the hi + lo split
of theta and of the residuals (a few 2^-16 of the summand scale) and FP32
accumulation.  The end-point log pi, which enters the importance weight, is
compared with the oracle on the FP32 data themselves.  Shapes cover ragged
observation chunks, ragged particle tiles, D = 7 .. 128 and the full
1e5-observation, 100-dimensional, 16384-particle launch.

The plain FP32 streamed kernel (precision 0 when X does not fit in shared
memory) is compared with the oracle on the FP32 data, at the same shapes.
"""
import numpy as np
import pytest

from gpu_util import dev, f32r, need_gpu, oracle_target, ptr, rounded_workload, stream, torch  # noqa: F401
import oracle
import paper_2504_02627_gb300 as g
import workloads
from paper_2504_02627_gb300 import _binding as B

pytestmark = pytest.mark.gpu

PREC = B.PREC_BF16X2
GRAD_TOL = 6e-5          # x (2^-16 .. 2^-15) of the summand scale, as for the three-term split


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def bf16_round(x):
    """Round-to-nearest-even to BF16 of the FP32 value, as FP64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _cases():
    return {
        "logistic": workloads.logistic(),                                     # n=1000, D=25
        "logistic_mid": workloads.logistic_large(n=3000, D=100),              # 46 chunks + 56 rows, dk 112
        "logistic_d128": workloads.logistic_large(n=500, D=128),              # dk 128, two stages
        "linear": workloads.linear_gauss(n=200, D=6),
        "logistic_d7": workloads.logistic(n=300, d_features=6),
    }


def _bf16_workload(w):
    v = dict(w)
    v["X"] = bf16_round(w["X"])
    return v


def _summand_scale(w, th):
    """Sum of absolute summands of each gradient component and of log pi."""
    eta = th @ w["X"].T
    eta_abs = np.abs(th) @ np.abs(w["X"]).T
    if w["kind"] == "logistic":
        r = np.abs(w["y"][None, :] - 1.0 / (1.0 + np.exp(-eta))) + 0.25 * eta_abs
        terms = np.abs(w["y"][None, :] * eta) + np.logaddexp(0, eta) + eta_abs
        tau2 = w.get("tau", 1.0) ** 2
    else:
        r = (np.abs(w["y"][None, :]) + eta_abs) / w["sigma"] ** 2
        terms = 0.5 * ((np.abs(w["y"][None, :]) + eta_abs) / w["sigma"]) ** 2
        tau2 = w["tau"] ** 2
    gs = r @ np.abs(w["X"]) + np.abs(th) / tau2
    return gs, terms.sum(axis=1) + 0.5 * (th**2).sum(axis=1) / tau2 + 1.0


def _theta(w, N, seed=3):
    """Particles around the data-generating coefficients (where a sampler
    spends its time), spread well beyond the posterior width."""
    rng = np.random.default_rng(seed)
    centre = w.get("beta_true", np.zeros(w["D"]))
    return f32r(centre[None, :] + 0.05 * rng.standard_normal((N, w["D"])))


def _dev_state(th, ld):
    N, D = th.shape
    t = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    t[:, :N] = torch.as_tensor(th.T.astype(np.float32)).cuda()
    return t


@pytest.mark.parametrize("name", ["logistic", "logistic_mid", "logistic_d128", "linear", "logistic_d7"])
@pytest.mark.parametrize("N", [1, 45, 300])
def test_streamed_target_value_and_gradient(name, N):
    w = rounded_workload(_cases()[name])
    wb = _bf16_workload(w)
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    th = _theta(w, N)
    ld = ((N + 31) // 32) * 32
    t_d = _dev_state(th, ld)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), PREC, stream()), "target")
    lp_g, gr_g = lp_d.cpu().numpy()[:N], g_d.cpu().numpy()[:, :N].T
    _, gr_o = oracle.logpi(oracle_target(wb), th)          # the data the integrator sees
    lp_o, _ = oracle.logpi(oracle_target(w), th)           # the data of the target
    gs, ls = _summand_scale(wb, th)
    err = np.abs(gr_g - gr_o) / (GRAD_TOL * gs + 1e-6)
    assert err.max() <= 1.0, err.max()
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls), np.max(np.abs(lp_g - lp_o) / ls)
    dm.close()


@pytest.mark.parametrize("name,eps", [("logistic", 1e-3), ("logistic_mid", 2e-3), ("linear", 0.005),
                                      ("logistic_d128", 2e-3)])
def test_streamed_leapfrog_trajectories(name, eps):
    """Ragged step counts 1..6: positions and momenta against the oracle's
    leapfrog on the BF16-rounded data (a gradient error dg moves p by at most
    S eps dg and theta by S^2 eps^2 dg), and the end-point energy against the
    oracle on the FP32 data at the GPU's own end points."""
    w = rounded_workload(_cases()[name])
    wb = _bf16_workload(w)
    tb, t = oracle_target(wb), oracle_target(w)
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 173                                                  # one full tile and a ragged one
    th = _theta(w, N, seed=5)
    p = f32r(np.random.default_rng(9).standard_normal((N, w["D"])))
    S = np.random.default_rng(10).integers(1, 7, N).astype(np.int32)
    ld = 192
    t_d, p_d = _dev_state(th, ld), _dev_state(p, ld)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), PREC, stream()), "target")
    s_d = dev(S)
    g.check(g.lib().smc_k_leapfrog(dm.h, ptr(t_d), ptr(p_d), ptr(g_d), ptr(lp_d), ptr(s_d), eps, N, ld, PREC,
                                   stream()), "leapfrog")
    th_g = t_d.cpu().numpy()[:, :N].T.astype(np.float64)
    p_g = p_d.cpu().numpy()[:, :N].T.astype(np.float64)
    lp_g = lp_d.cpu().numpy()[:N]
    th_o, p_o, _, _ = oracle.leapfrog(tb, th, p, eps, S)
    gs0, _ = _summand_scale(wb, th)
    gs1, _ = _summand_scale(wb, th_o)
    dg = GRAD_TOL * np.maximum(gs0, gs1) + 1e-6
    Sc = S[:, None].astype(np.float64)
    rms = lambda a: np.sqrt(np.mean(a**2))
    tol_p = Sc * eps * dg + 1e-5 * Sc * (np.abs(p_o) + rms(p_o))
    tol_t = Sc**2 * eps**2 * dg + 1e-5 * Sc * (np.abs(th_o) + rms(th_o))
    assert np.all(np.abs(p_g - p_o) <= tol_p), np.max(np.abs(p_g - p_o) / tol_p)
    assert np.all(np.abs(th_g - th_o) <= tol_t), np.max(np.abs(th_g - th_o) / tol_t)
    lp_at_g, _ = oracle.logpi(t, th_g)
    _, ls = _summand_scale(w, th_g)
    assert np.all(np.abs(lp_g - lp_at_g) <= 1e-5 * ls)
    dm.close()


def test_streamed_full_size_launch_on_sampled_particles():
    """The launch the benchmark times: n = 1e5 observations, D = 100,
    16384 particles (128 tiles, 1563 chunks).  Gradients and log pi of 24
    sampled particles against the oracle."""
    w = rounded_workload(workloads.logistic_large())
    wb = _bf16_workload(w)
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 16384
    th = _theta(w, N, seed=7)
    t_d = _dev_state(th, N)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(N, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, N, ptr(lp_d), ptr(g_d), PREC, stream()), "target")
    idx = np.sort(np.random.default_rng(11).choice(N, 24, replace=False))
    idx[-1] = N - 1
    lp_g, gr_g = lp_d.cpu().numpy()[idx], g_d.cpu().numpy()[:, idx].T
    _, gr_o = oracle.logpi(oracle_target(wb), th[idx])
    lp_o, _ = oracle.logpi(oracle_target(w), th[idx])
    gs, ls = _summand_scale(wb, th[idx])
    err = np.abs(gr_g - gr_o) / (GRAD_TOL * gs + 1e-6)
    assert err.max() <= 1.0, err.max()
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls)
    dm.close()


def test_streamed_eval_is_deterministic_and_tile_independent():
    """Each particle's result depends on its own state only: the same
    particles in another order (another tile assignment) give identical bits."""
    w = rounded_workload(_cases()["logistic_mid"])
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 300
    th = _theta(w, N, seed=12)
    perm = np.random.default_rng(13).permutation(N)
    out = []
    for order in (np.arange(N), perm):
        t_d = _dev_state(th[order], 320)
        g_d = torch.zeros_like(t_d)
        lp_d = torch.zeros(320, dtype=torch.float64, device="cuda")
        g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, 320, ptr(lp_d), ptr(g_d), PREC, stream()), "target")
        gr = np.empty((N, w["D"]), np.float32)
        gr[order] = g_d.cpu().numpy()[:, :N].T
        lp = np.empty(N)
        lp[order] = lp_d.cpu().numpy()[:N]
        out.append((gr, lp))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    dm.close()


# ------------------------------------------------------------- FP32 streamed path
# The plain FP32 kernel for data that do not fit in shared memory streams the
# FP32 data themselves, so it is compared with the oracle on the same FP32
# data: FP32 accumulation error of a few 2^-20 of the summand scale.
FP32_GRAD_TOL = 2e-5


def _fp32_cases():
    return {
        "logistic_mid": workloads.logistic_large(n=3000, D=100),            # D=100: quarters of 28
        "logistic_d128": workloads.logistic_large(n=500, D=128),            # too wide for the resident kernel
        "logistic_n3000_d25": workloads.logistic(n=3000, d_features=24),    # X too large for shared memory
        "linear_n5000": workloads.linear_gauss(n=5000, D=6),
    }


@pytest.mark.parametrize("name", ["logistic_mid", "logistic_d128", "logistic_n3000_d25", "linear_n5000"])
@pytest.mark.parametrize("N", [1, 45, 300])
def test_fp32_streamed_target_value_and_gradient(name, N):
    w = rounded_workload(_fp32_cases()[name])
    t = oracle_target(w)
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    th = _theta(w, N)
    ld = ((N + 31) // 32) * 32
    t_d = _dev_state(th, ld)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), B.PREC_FP32, stream()), "target")
    lp_g, gr_g = lp_d.cpu().numpy()[:N], g_d.cpu().numpy()[:, :N].T
    lp_o, gr_o = oracle.logpi(t, th)
    gs, ls = _summand_scale(w, th)
    err = np.abs(gr_g - gr_o) / (FP32_GRAD_TOL * gs + 1e-6)
    assert err.max() <= 1.0, err.max()
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls), np.max(np.abs(lp_g - lp_o) / ls)
    dm.close()


@pytest.mark.parametrize("name,eps", [("logistic_mid", 2e-3), ("logistic_n3000_d25", 1e-3), ("linear_n5000", 2e-3)])
def test_fp32_streamed_leapfrog_trajectories(name, eps):
    """Ragged step counts 1..6 against the oracle's leapfrog on the same FP32
    data: per step 1e-5 relative, plus what the FP32 gradient error moves."""
    w = rounded_workload(_fp32_cases()[name])
    t = oracle_target(w)
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 173
    th = _theta(w, N, seed=5)
    p = f32r(np.random.default_rng(9).standard_normal((N, w["D"])))
    S = np.random.default_rng(10).integers(1, 7, N).astype(np.int32)
    ld = 192
    t_d, p_d = _dev_state(th, ld), _dev_state(p, ld)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), B.PREC_FP32, stream()), "target")
    s_d = dev(S)
    g.check(g.lib().smc_k_leapfrog(dm.h, ptr(t_d), ptr(p_d), ptr(g_d), ptr(lp_d), ptr(s_d), eps, N, ld,
                                   B.PREC_FP32, stream()), "leapfrog")
    th_g = t_d.cpu().numpy()[:, :N].T.astype(np.float64)
    p_g = p_d.cpu().numpy()[:, :N].T.astype(np.float64)
    lp_g = lp_d.cpu().numpy()[:N]
    th_o, p_o, _, _ = oracle.leapfrog(t, th, p, eps, S)
    gs0, _ = _summand_scale(w, th)
    gs1, _ = _summand_scale(w, th_o)
    dg = FP32_GRAD_TOL * np.maximum(gs0, gs1) + 1e-6
    Sc = S[:, None].astype(np.float64)
    rms = lambda a: np.sqrt(np.mean(a**2))
    tol_p = Sc * eps * dg + 1e-5 * Sc * (np.abs(p_o) + rms(p_o))
    tol_t = Sc**2 * eps**2 * dg + 1e-5 * Sc * (np.abs(th_o) + rms(th_o))
    assert np.all(np.abs(p_g - p_o) <= tol_p), np.max(np.abs(p_g - p_o) / tol_p)
    assert np.all(np.abs(th_g - th_o) <= tol_t), np.max(np.abs(th_g - th_o) / tol_t)
    lp_at_g, _ = oracle.logpi(t, th_g)
    _, ls = _summand_scale(w, th_g)
    assert np.all(np.abs(lp_g - lp_at_g) <= 1e-5 * ls)
    dm.close()


def test_fp32_streamed_full_size_launch_on_sampled_particles():
    """n = 1e5, D = 100, 16384 particles (256 CTAs of 64): gradients and
    log pi of 24 sampled particles against the oracle."""
    w = rounded_workload(workloads.logistic_large())
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 16384
    th = _theta(w, N, seed=7)
    t_d = _dev_state(th, N)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(N, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, N, ptr(lp_d), ptr(g_d), B.PREC_FP32, stream()), "target")
    idx = np.sort(np.random.default_rng(11).choice(N, 24, replace=False))
    idx[-1] = N - 1
    lp_g, gr_g = lp_d.cpu().numpy()[idx], g_d.cpu().numpy()[:, idx].T
    lp_o, gr_o = oracle.logpi(oracle_target(w), th[idx])
    gs, ls = _summand_scale(w, th[idx])
    err = np.abs(gr_g - gr_o) / (FP32_GRAD_TOL * gs + 1e-6)
    assert err.max() <= 1.0, err.max()
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls)
    dm.close()
