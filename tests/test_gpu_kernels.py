"""GPU parity of the single stages, through the C-ABI kernel-level entry
points, against the FP64 oracle on the same seeded inputs.

Bars: bit-exact for Philox words, Halton values, step counts, fixed-point
weights and resampling ancestors; FP64 normals within 1e-12; FP32 target
gradients within 1e-5 of the sum of absolute summands; one leapfrog step
within 1e-5 relative (spec tolerance), S steps within S * 1e-5.
"""
import numpy as np
import pytest

from gpu_util import dev, f32r, need_gpu, oracle_target, ptr, rounded_workload, stream, torch  # noqa: F401
import oracle
import paper_2504_02627_gb300 as g
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_philox_words_bit_exact():
    rng = np.random.default_rng(0)
    n = 5000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [2**32 - 1] * 4]
    seed = 0x0123456789ABCDEF
    c_d = dev(ctr.view(np.int32))
    o_d = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    g.check(g.lib().smc_k_philox(seed, ptr(c_d), ptr(o_d), n, stream()), "smc_k_philox")
    got = o_d.cpu().numpy().view(np.uint32)
    want = np.stack([oracle.philox(c, seed) for c in ctr])
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("D", [1, 10, 25])
def test_normals_match_oracle(D):
    N, ld, seed, k = 333, 352, 77, 5
    out = torch.zeros((D, ld), dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_normals(seed, oracle.TAG_MOM, k, N, D, ptr(out), ld, stream()), "normals")
    got = out.cpu().numpy()[:, :N].T
    want = np.stack([oracle.normals(seed, oracle.TAG_MOM, k, j, D) for j in range(N)])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", range(12))
@pytest.mark.parametrize("J,K", [(1000, 50), (37, 9)])
def test_jitter_schemes_bit_exact(scheme, J, K):
    """The jitter schemes of Sec. 3.2.1 (smc_k_jitter): every h bit-exact
    against the oracle (integer radical inverses, correctly rounded sqrt,
    products and frac, Philox uniforms, the Feistel shuffle with cycle
    walking at a non-power-of-4 J)."""
    seed = 0xC0FFEE
    out = torch.zeros(J, dtype=torch.float64, device="cuda")
    for k in sorted({1, 2, K // 2, K}):
        g.check(g.lib().smc_k_jitter(scheme, seed, J, K, k, ptr(out), stream()), "smc_k_jitter")
        got = out.cpu().numpy()
        want = np.array([oracle.jitter(scheme, seed, j, k, J, K) for j in range(J)])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("K,k,L,eps,jitter", [(50, 1, 0.5, 1e-3, 1), (50, 50, 0.123456, 1e-3, 1),
                                             (20, 7, 4.8, 0.1, 1), (20, 3, 0.75, 0.1, 0)])
def test_halton_and_step_counts_bit_exact(K, k, L, eps, jitter):
    N = 4100
    h_d = torch.empty(N, dtype=torch.float64, device="cuda")
    s_d = torch.empty(N, dtype=torch.int32, device="cuda")
    g.check(g.lib().smc_k_steps(N, K, k, L, eps, 500, jitter, ptr(h_d), ptr(s_d), stream()), "steps")
    h = h_d.cpu().numpy()
    S = s_d.cpu().numpy()
    want_h = np.array([oracle.halton2(j * K + k) if jitter else 1.0 for j in range(N)])
    np.testing.assert_array_equal(h, want_h)
    want_s = np.array([oracle.step_count(x, L, eps, 500) for x in want_h])
    np.testing.assert_array_equal(S, want_s)


# ------------------------------------------------------------- targets
def _workloads():
    return {
        "gauss10": workloads.gauss10(),
        "logistic": workloads.logistic(),                              # n=1000, D=25
        "logistic_small": workloads.logistic(n=37, d_features=4),
        "logistic_d4": workloads.logistic(n=123, d_features=3),        # Dp=4
        "logistic_d12": workloads.logistic(n=400, d_features=11),      # Dp=16
        "logistic_d28": workloads.logistic(n=500, d_features=27),      # Dp=28, no padding column
        "logistic_n1300": workloads.logistic(n=1300),
        "logistic_n1700": workloads.logistic(n=1700),                  # x3 operands too large for one CTA
        "linear_d25": workloads.linear_gauss(n=700, D=25),
        "linear": workloads.linear_gauss(n=200, D=6),
        "hier": workloads.hier(),                                      # 50 groups, D=52
        "banana50": workloads.banana50(),
        "banana2": workloads.paper_banana2(),
        "gauss100": workloads.gauss100_cond(),       # dense precision, D=100 (CTA kernel)
        "illcond100": workloads.paper_illcond100(),  # Sec. 4 ill-conditioned Gaussian
        # dense Gaussians for the warp-MMA kernel's shapes: one k-step (D = 1),
        # a ragged second k-step (D = 17), the eight-warp maximum (D = 128)
        "gauss_d1": workloads._gauss_from_spectrum(np.array([2.0]), 7),
        "gauss_d17": workloads._gauss_from_spectrum(np.geomspace(1.0, 100.0, 17), 7),
        "gauss_d128": workloads._gauss_from_spectrum(np.geomspace(1.0, 1000.0, 128), 7),
    }


def _model(w):
    return g.DevModel(g.ModelData.from_workload(w), stream())


def _theta(w, N, seed=3, scale=0.3):
    rng = np.random.default_rng(seed)
    th = rng.standard_normal((N, w["D"])) * scale
    if w["kind"] == "hier_normal":
        # near the posterior of the non-centred model, where trajectories are
        # stable: mu ~ mean of group means, tau ~ their spread
        mu, tau = w["ybar"].mean(), w["ybar"].std()
        th[:, 0] = mu + 0.1 * th[:, 0]
        th[:, 1] = np.log(tau) + 0.1 * th[:, 1]
        th[:, 2:] = (w["ybar"] - mu)[None, :] / tau + 0.1 * th[:, 2:]
    return f32r(th)


def _eval_gpu(dm, th, ld):
    N, D = th.shape
    t_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    t_d[:, :N] = torch.as_tensor(th.T.astype(np.float32)).cuda()
    g_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), 0, stream()), "target")
    return lp_d.cpu().numpy()[:N], g_d.cpu().numpy()[:, :N].T


def _summand_scale(w, th):
    """Sum of absolute summands of each gradient component (and of log pi),
    the scale against which FP32 accumulation error is bounded."""
    N, D = th.shape
    if w["kind"] in ("logistic", "linear_gauss"):
        eta = th @ w["X"].T
        eta_abs = np.abs(th) @ np.abs(w["X"]).T          # operands of the inner products
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
    if w["kind"] == "gauss_dense":
        gs = np.abs(th - w["mu"]) @ np.abs(w["P"]).T
        return gs, (np.abs(th - w["mu"]) * gs).sum(axis=1) + 1.0
    if w["kind"] == "hier_normal":
        mu, logtau, eta = th[:, :1], th[:, 1:2], th[:, 2:]
        tau = np.exp(logtau)
        # the residual ybar - (mu + tau eta) cancels near the posterior: bound
        # its FP32 error by the magnitudes of its operands, each counted once
        # per rounding it goes through -- ybar and mu enter the two sums once,
        # tau eta carries the error of expf (within 2 ulp in CUDA's
        # documentation) plus the rounding of the product: 3 units
        dev_ops = np.abs(w["ybar"][None, :]) + np.abs(mu) + 3.0 * np.abs(tau * eta)
        r = w["n_g"][None, :] * dev_ops / w["sigma"] ** 2
        gs = np.concatenate([r.sum(1, keepdims=True) + np.abs(mu),
                             (r * tau * np.abs(eta)).sum(1, keepdims=True) + np.abs(logtau),
                             r * tau + np.abs(eta)], axis=1)
        ls = ((w["ss"][None, :] + w["n_g"][None, :] * dev_ops**2) / (2 * w["sigma"] ** 2)).sum(1)
        return gs, ls + 0.5 * (th**2).sum(1) + 100.0
    # banana pairs
    a, b = w["a"], w["b"]
    xo, xe = th[:, 0::2], th[:, 1::2]
    u = np.abs(xe) + abs(b) * (xo**2 + a)
    gs = np.empty_like(th)
    gs[:, 0::2] = np.abs(xo) / a + 2 * abs(b) * u * np.abs(xo)
    gs[:, 1::2] = u
    return gs, (0.5 * xo**2 / a + 0.5 * u**2).sum(1) + 10.0


@pytest.mark.parametrize("name", ["gauss10", "logistic", "logistic_small", "logistic_d4", "logistic_d12",
                                  "logistic_d28", "logistic_n1300", "linear", "linear_d25", "hier", "banana50",
                                  "banana2", "gauss100", "illcond100"])
@pytest.mark.parametrize("N", [1, 45, 300])
def test_target_value_and_gradient(name, N):
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    th = _theta(w, N)
    lp_g, gr_g = _eval_gpu(dm, th, ((N + 31) // 32) * 32)
    lp_o, gr_o = oracle.logpi(t, th)
    gs, ls = _summand_scale(w, th)
    assert np.all(np.abs(gr_g - gr_o) <= 1e-5 * gs + 1e-6), np.max(np.abs(gr_g - gr_o) / (gs + 1e-30))
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls), np.max(np.abs(lp_g - lp_o) / ls)


# ------------------------------------------------------------- leapfrog
def _leapfrog_gpu(dm, th, p, steps, eps):
    N, D = th.shape
    ld = ((N + 31) // 32) * 32
    t_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    t_d[:, :N] = torch.as_tensor(th.T.astype(np.float32)).cuda()
    p_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    p_d[:, :N] = torch.as_tensor(p.T.astype(np.float32)).cuda()
    g_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), 0, stream()), "target")
    s_d = dev(np.asarray(steps, dtype=np.int32))
    g.check(g.lib().smc_k_leapfrog(dm.h, ptr(t_d), ptr(p_d), ptr(g_d), ptr(lp_d), ptr(s_d), eps, N, ld, 0,
                                   stream()), "leapfrog")
    return (t_d.cpu().numpy()[:, :N].T.astype(np.float64), p_d.cpu().numpy()[:, :N].T.astype(np.float64),
            lp_d.cpu().numpy()[:N])


def _rms(a):
    return np.sqrt(np.mean(np.square(a))) + 1e-30


@pytest.mark.parametrize("name,eps", [("gauss10", 0.1), ("logistic", 1e-3), ("logistic_small", 0.01),
                                      ("logistic_d4", 0.005), ("logistic_d12", 0.002), ("logistic_d28", 0.002),
                                      ("logistic_n1300", 1e-3), ("linear", 0.005), ("linear_d25", 1e-3),
                                      ("hier", 0.05), ("banana50", 0.01),
                                      ("banana2", 0.01), ("gauss100", 0.01), ("illcond100", 1e-3)])
def test_one_leapfrog_step_within_1e5(name, eps):
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    N = 257
    th = _theta(w, N)
    p = f32r(np.random.default_rng(9).standard_normal((N, w["D"])))
    th_g, p_g, _ = _leapfrog_gpu(dm, th, p, np.ones(N), eps)
    th_o, p_o, _, _ = oracle.leapfrog(t, th, p, eps, 1)
    np.testing.assert_allclose(th_g, th_o, rtol=1e-5, atol=1e-5 * _rms(th_o))
    np.testing.assert_allclose(p_g, p_o, rtol=1e-5, atol=1e-5 * _rms(p_o))


@pytest.mark.parametrize("name,eps", [("gauss10", 0.1), ("logistic", 1e-3), ("hier", 0.01),
                                      ("banana50", 0.01), ("gauss100", 0.005)])
def test_ragged_trajectories(name, eps):
    """Different step counts per particle (1..40), across several CTAs and a
    ragged tail; tolerance grows linearly with the step count."""
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    N = 83
    th = _theta(w, N)
    p = f32r(np.random.default_rng(10).standard_normal((N, w["D"])))
    steps = np.random.default_rng(11).integers(1, 41, N)
    steps[0] = 0
    th_g, p_g, lp_g = _leapfrog_gpu(dm, th, p, steps, eps)
    th_o, p_o, _, lp_o = oracle.leapfrog(t, th, p, eps, steps)
    for j in range(N):
        tol = 1e-5 * max(1, steps[j])
        np.testing.assert_allclose(th_g[j], th_o[j], rtol=tol, atol=tol * _rms(th_o[j]))
        np.testing.assert_allclose(p_g[j], p_o[j], rtol=tol, atol=tol * _rms(p_o[j]))
    _, ls = _summand_scale(w, th_o)
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * steps.clip(1) * ls)


@pytest.mark.parametrize("name", ["logistic", "linear_d25"])
@pytest.mark.parametrize("N", [4096, 20000])
def test_glm_trajectories_many_particles(name, N):
    """The regression kernels at the particle counts of the benchmark and
    above (several particle pairs per CTA, every CTA count regime): ragged
    step counts 0..8, a seeded sample of 150 particles against the oracle."""
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    rng = np.random.default_rng(N)
    th = _theta(w, N, seed=N + 1)
    p = f32r(rng.standard_normal((N, w["D"])))
    steps = rng.integers(0, 9, N)
    eps = 1e-3
    th_g, p_g, lp_g = _leapfrog_gpu(dm, th, p, steps, eps)
    idx = np.sort(rng.choice(N, 150, replace=False))
    idx[-1] = N - 1                                         # the ragged tail
    th_o, p_o, _, lp_o = oracle.leapfrog(t, th[idx], p[idx], eps, steps[idx])
    for a, j in enumerate(idx):
        tol = 1e-5 * max(1, steps[j])
        np.testing.assert_allclose(th_g[j], th_o[a], rtol=tol, atol=tol * _rms(th_o[a]))
        np.testing.assert_allclose(p_g[j], p_o[a], rtol=tol, atol=tol * _rms(p_o[a]))
    _, ls = _summand_scale(w, th_o)
    assert np.all(np.abs(lp_g[idx] - lp_o) <= 1e-5 * steps[idx].clip(1) * ls)


# ------------------------------------------------------------- weights
@pytest.mark.parametrize("N", [1, 5, 1000, 4096, 20000])
def test_normalise_matches_oracle(N):
    rng = np.random.default_rng(N)
    lw = rng.standard_normal(N) * 5 - 100
    if N > 3:
        lw[2] = -np.inf
    lw_d = dev(lw)
    W_d = torch.empty(N, dtype=torch.float64, device="cuda")
    sc = torch.empty(2, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_normalise(ptr(lw_d), N, ptr(W_d), ptr(sc), ptr(sc) + 8, stream()), "normalise")
    lse, ess, W = oracle.normalise(lw)
    s = sc.cpu().numpy()
    assert abs(s[0] - lse) <= 1e-12 * abs(lse) and abs(s[1] - ess) <= 1e-12 * ess
    np.testing.assert_allclose(W_d.cpu().numpy(), W, rtol=1e-13, atol=0)


def _resample_gpu(W, r64):
    N = W.size
    W_d = dev(W)
    q_d = torch.empty(N, dtype=torch.int64, device="cuda")
    a_d = torch.empty(N, dtype=torch.int32, device="cuda")
    st_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = g.lib().smc_k_resample_scratch_bytes(N)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g.check(g.lib().smc_k_resample(ptr(W_d), N, r64, ptr(q_d), ptr(a_d), ptr(st_d), ptr(scratch), stream()),
            "resample")
    return q_d.cpu().numpy().view(np.uint64), a_d.cpu().numpy(), int(st_d.cpu().numpy()[0])


@pytest.mark.parametrize("N", [1, 2, 3, 7, 2047, 2048, 2049, 4096, 70001, 1 << 20])
def test_systematic_resampling_bit_exact(N):
    rng = np.random.default_rng(N + 1)
    W = rng.gamma(0.2, size=N)
    W[rng.uniform(size=N) < 0.3] = 0.0
    if W.sum() == 0:
        W[0] = 1.0
    W /= W.sum()
    for r64 in (int(rng.integers(0, 2**63)) * 2 + 1, 0, 2**64 - 1):
        q, anc, st = _resample_gpu(W, r64)
        assert st == 0
        S, q_o = oracle.quantise(W)
        np.testing.assert_array_equal(q, q_o)
        T, anc_o = oracle.systematic(q_o, r64)
        np.testing.assert_array_equal(anc, anc_o)


def test_resampling_one_hot_and_degenerate():
    W = np.zeros(5000)
    W[4321] = 1.0
    q, anc, st = _resample_gpu(W, 12345)
    assert st == 0 and np.all(anc == 4321)
    q, anc, st = _resample_gpu(np.zeros(100), 1)
    assert st == -4


# ------------------------------------------------------------- tensor-core path
# Gradient error bounds of the split-BF16 products, relative to the sum of
# absolute summands: BF16 keeps 8 significant bits, so each operand
# x = hi + lo with |x - hi| <= 2^-8 |x| and |x - hi - lo| <= 2^-16 |x|; the
# x3 form (hi*hi + lo*hi + hi*lo, lo*lo dropped) errs by at most about
# 3 x 2^-16 (4.6e-5) per product plus FP32 accumulation, and plain BF16 by
# at most 2 x 2^-8 (7.8e-3); the bounds below sit above these.  The end-point
# log pi is FP32 in every mode.
TC_GRAD_TOL = {1: 6e-5, 2: 2e-2}


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", ["logistic_small", "logistic", "linear", "logistic_d28", "linear_d25",
                                  "logistic_n1700", "gauss10", "gauss100", "illcond100", "gauss_d1",
                                  "gauss_d17", "gauss_d128"])
@pytest.mark.parametrize("N", [1, 45, 300])
def test_tc_target_value_and_gradient(name, N, precision):
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    th = _theta(w, N)
    ld = ((N + 31) // 32) * 32
    D = th.shape[1]
    t_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    t_d[:, :N] = torch.as_tensor(th.T.astype(np.float32)).cuda()
    g_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), precision, stream()), "target")
    lp_g, gr_g = lp_d.cpu().numpy()[:N], g_d.cpu().numpy()[:, :N].T
    lp_o, gr_o = oracle.logpi(t, th)
    gs, ls = _summand_scale(w, th)
    tol = TC_GRAD_TOL[precision]
    assert np.all(np.abs(gr_g - gr_o) <= tol * gs + 1e-6), np.max(np.abs(gr_g - gr_o) / gs)
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls), np.max(np.abs(lp_g - lp_o) / ls)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name,eps,N", [("logistic", 1e-3, 257), ("logistic_small", 0.01, 257),
                                        ("linear", 0.005, 257), ("logistic_d28", 0.002, 257),
                                        ("linear_d25", 1e-3, 257), ("logistic_n1700", 1e-3, 257),
                                        ("logistic", 1e-3, 4096), ("logistic", 1e-3, 20000),
                                        ("gauss10", 0.1, 257), ("gauss100", 0.005, 257),
                                        ("illcond100", 1e-3, 257), ("gauss100", 0.005, 8192),
                                        ("gauss_d1", 0.1, 257), ("gauss_d17", 0.02, 257),
                                        ("gauss_d128", 0.005, 257)])
def test_tc_one_leapfrog_step(name, eps, N, precision):
    """One step: theta_1 = theta_0 + eps (p_0 + eps/2 g_0), p_1 = p_0 + eps/2 (g_0 + g_1);
    a gradient error dg moves p by at most eps*dg and theta by eps^2/2 dg.  At the
    benchmark's particle count and above, a seeded sample of 200 particles is
    checked (every CTA handles the same arithmetic)."""
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    th = _theta(w, N)
    p = f32r(np.random.default_rng(9).standard_normal((N, w["D"])))
    ld = ((N + 31) // 32) * 32
    D = w["D"]
    t_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    t_d[:, :N] = torch.as_tensor(th.T.astype(np.float32)).cuda()
    p_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    p_d[:, :N] = torch.as_tensor(p.T.astype(np.float32)).cuda()
    g_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), precision, stream()), "target")
    s_d = dev(np.ones(N, dtype=np.int32))
    g.check(g.lib().smc_k_leapfrog(dm.h, ptr(t_d), ptr(p_d), ptr(g_d), ptr(lp_d), ptr(s_d), eps, N, ld,
                                   precision, stream()), "leapfrog")
    th_g = t_d.cpu().numpy()[:, :N].T.astype(np.float64)
    p_g = p_d.cpu().numpy()[:, :N].T.astype(np.float64)
    lp_g = lp_d.cpu().numpy()[:N]
    if N > 1000:
        idx = np.sort(np.random.default_rng(N).choice(N, 200, replace=False))
        idx[-1] = N - 1
        th, p, th_g, p_g, lp_g = th[idx], p[idx], th_g[idx], p_g[idx], lp_g[idx]
    th_o, p_o, _, lp_o = oracle.leapfrog(t, th, p, eps, 1)
    gs0, _ = _summand_scale(w, th)
    gs1, ls1 = _summand_scale(w, th_o)
    dg = TC_GRAD_TOL[precision] * np.maximum(gs0, gs1) + 1e-6
    np.testing.assert_array_less(np.abs(p_g - p_o), eps * dg + 1e-5 * (np.abs(p_o) + _rms(p_o)))
    np.testing.assert_array_less(np.abs(th_g - th_o), 0.5 * eps**2 * dg + 1e-5 * (np.abs(th_o) + _rms(th_o)))
    # the end-point energy is exact to FP32 accuracy at the GPU's own end point
    lp_at_g, _ = oracle.logpi(t, th_g)
    assert np.all(np.abs(lp_g - lp_at_g) <= 1e-5 * ls1)


@pytest.mark.parametrize("name,N,eps", [("banana50", 8192, 0.05), ("hier", 278_000, 0.01)])
def test_thread_kernel_trajectories_at_bench_size(name, N, eps):
    """The thread-per-particle kernels at the particle counts the benchmark
    runs (the banana of the preconditioner comparison, the 278 k particles of
    the batched hierarchical workload): ragged step counts 0..12, a seeded
    sample of 150 particles and the last one against the oracle."""
    w = rounded_workload(_workloads()[name])
    t = oracle_target(w)
    dm = _model(w)
    rng = np.random.default_rng(N)
    th = _theta(w, N, seed=N + 7)
    p = f32r(rng.standard_normal((N, w["D"])))
    steps = rng.integers(0, 13, N)
    th_g, p_g, lp_g = _leapfrog_gpu(dm, th, p, steps, eps)
    idx = np.sort(rng.choice(N, 150, replace=False))
    idx[-1] = N - 1
    th_o, p_o, _, lp_o = oracle.leapfrog(t, th[idx], p[idx], eps, steps[idx])
    for a, j in enumerate(idx):
        tol = 1e-5 * max(1, steps[j])
        np.testing.assert_allclose(th_g[j], th_o[a], rtol=tol, atol=tol * _rms(th_o[a]))
        np.testing.assert_allclose(p_g[j], p_o[a], rtol=tol, atol=tol * _rms(p_o[a]))
    _, ls = _summand_scale(w, th_o)
    assert np.all(np.abs(lp_g[idx] - lp_o) <= 1e-5 * steps[idx].clip(1) * ls)
