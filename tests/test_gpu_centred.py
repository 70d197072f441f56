"""GPU parity of the centred tensor-core trajectory kernel (precision 4:
per-move reference point theta_ref = mean of the particles, exact reference
quantities, BF16 products of the deviations only) against the FP64 oracle,
through the C-ABI.

The gradient is compared with the oracle's exact gradient on the FP32 data
within a bound derived from the arithmetic, per component d:
* the deviation d_eta_i = X_i (theta - theta_ref) carries the BF16 rounding of
  the deviation and of X (BF16 keeps 8 significant bits: round to nearest is
  within 2^-8 relative, each, of sum_d |X_id delta_d|), plus
  the FP32 rounding of -log2(e) eta_ref and of the exponential's argument;
* the sigmoid moves by at most 1/4 of that, plus the SFU / FMA-pipe
  reciprocal and exponential errors (below 4e-7 absolute);
* the residual change d_r is rounded to BF16 (2^-8 relative);
* the second product uses BF16 X (2^-8 of sum_i |X_id d_r_i|) and
  accumulates n / 16 partial products in FP32;
* g_ref, G and the prior term are FP32 values added in FP32.
A factor 2 covers the remaining rounding of sums.  The end-point log pi,
which enters the importance weight, is compared with the oracle on the FP32
data (FP32 products, FP64 sums).  Shapes cover ragged 128-observation tiles,
ragged particle tiles, D = 7 .. 128 (one and two 64-dimension atoms), the
linear-Gaussian model, particles spread as the prior and concentrated near
the data-generating coefficients, and the full 1e5-observation,
100-dimensional, 16384-particle launch.
"""
import numpy as np
import pytest

from gpu_util import dev, f32r, need_gpu, oracle_target, ptr, rounded_workload, stream, torch  # noqa: F401
import oracle
import paper_2504_02627_gb300 as g
import workloads
from paper_2504_02627_gb300 import _binding as B

pytestmark = pytest.mark.gpu

PREC = B.PREC_BF16C


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _cases():
    return {
        "logistic": workloads.logistic(),                                     # n=1000 (7 tiles + 104), D=25
        "logistic_mid": workloads.logistic_large(n=3000, D=100),              # 23 tiles + 56, two atoms
        "logistic_d128": workloads.logistic_large(n=500, D=128),              # dk 128
        "linear": workloads.linear_gauss(n=200, D=6),
        "logistic_d7": workloads.logistic(n=300, d_features=6),
    }


def _expit(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def centred_bound(w, th, centre):
    """Per-component bound of |g_gpu - g_exact| (see the module docstring)."""
    X = w["X"]
    n = X.shape[0]
    delta = th - centre[None, :]
    absX = np.abs(X)
    adx = np.abs(delta) @ absX.T                         # [N, n]: sum_d |X_id delta_d|
    eta = th @ X.T
    eta_ref = X @ centre
    e_eta = 2.0**-7 * 1.01 * adx + 2.0**-23 * (np.abs(eta_ref)[None, :] + np.abs(eta))
    if w["kind"] == "logistic":
        s_ref = _expit(eta_ref)
        dr = s_ref[None, :] - _expit(eta)
        dr_err = 0.25 * e_eta + 4e-7 + 2.0**-8 * 1.01 * np.abs(dr)
        gref = X.T @ (w["y"] - s_ref)
        tau2 = w.get("tau", 1.0) ** 2
    else:
        s2 = w["sigma"] ** 2
        dr = -(eta - eta_ref[None, :]) / s2
        dr_err = e_eta / s2 + 2.0**-8 * 1.01 * np.abs(dr)
        gref = X.T @ (w["y"] - eta_ref) / s2
        tau2 = w["tau"] ** 2
    adr = np.abs(dr) @ absX
    G = dr @ X
    err = (1 + 2.0**-8) * (dr_err @ absX) + 2.0**-8 * adr + (n / 16 + 16) * 2.0**-24 * adr
    err += 2.0**-23 * (np.abs(gref)[None, :] + np.abs(G) + np.abs(th) / tau2)
    return 2.0 * err + 1e-6


def _log_scale(w, th):
    eta = th @ w["X"].T
    eta_abs = np.abs(th) @ np.abs(w["X"]).T
    if w["kind"] == "logistic":
        terms = np.abs(w["y"][None, :] * eta) + np.logaddexp(0, eta) + eta_abs
        tau2 = w.get("tau", 1.0) ** 2
    else:
        terms = 0.5 * ((np.abs(w["y"][None, :]) + eta_abs) / w["sigma"]) ** 2
        tau2 = w["tau"] ** 2
    return terms.sum(axis=1) + 0.5 * (th**2).sum(axis=1) / tau2 + 1.0


def _theta(w, N, seed=3, spread=False):
    """Particles around the data-generating coefficients (where a sampler
    spends its time), or spread as the N(0, I) prior (its first iterations)."""
    rng = np.random.default_rng(seed)
    if spread:
        return f32r(rng.standard_normal((N, w["D"])))
    centre = w.get("beta_true", np.zeros(w["D"]))
    return f32r(centre[None, :] + 0.05 * rng.standard_normal((N, w["D"])))


def _dev_state(th, ld):
    N, D = th.shape
    t = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    t[:, :N] = torch.as_tensor(th.T.astype(np.float32)).cuda()
    return t


def _target(dm, th, ld):
    N = th.shape[0]
    t_d = _dev_state(th, ld)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(ld, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), PREC, stream()), "target")
    return lp_d.cpu().numpy()[:N], g_d.cpu().numpy()[:, :N].T.astype(np.float64)


@pytest.mark.parametrize("name", ["logistic", "logistic_mid", "logistic_d128", "linear", "logistic_d7"])
@pytest.mark.parametrize("N", [1, 45, 300])
@pytest.mark.parametrize("spread", [False, True])
def test_centred_target_value_and_gradient(name, N, spread):
    w = rounded_workload(_cases()[name])
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    th = _theta(w, N, spread=spread)
    lp_g, gr_g = _target(dm, th, ((N + 31) // 32) * 32)
    lp_o, gr_o = oracle.logpi(oracle_target(w), th)
    bound = centred_bound(w, th, th.mean(axis=0))
    err = np.abs(gr_g - gr_o) / bound
    assert err.max() <= 1.0, err.max()
    ls = _log_scale(w, th)
    assert np.all(np.abs(lp_g - lp_o) <= 1e-5 * ls), np.max(np.abs(lp_g - lp_o) / ls)
    dm.close()


def test_centred_gradient_beats_the_hi_lo_split_near_the_posterior():
    """Where particles sit near each other, the one-product centred form is
    closer to the exact gradient than the two-product BF16x2 split (whose X
    rounding enters the whole residual), measured on the same particles."""
    w = rounded_workload(_cases()["logistic_mid"])
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    th = _theta(w, 256, seed=21)
    _, gr_c = _target(dm, th, 256)
    t_d = _dev_state(th, 256)
    g_d = torch.zeros_like(t_d)
    lp_d = torch.zeros(256, dtype=torch.float64, device="cuda")
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), 256, 256, ptr(lp_d), ptr(g_d), B.PREC_BF16X2, stream()), "t")
    gr_2 = g_d.cpu().numpy()[:, :256].T.astype(np.float64)
    _, gr_o = oracle.logpi(oracle_target(w), th)
    e_c = np.sqrt(np.mean((gr_c - gr_o) ** 2))
    e_2 = np.sqrt(np.mean((gr_2 - gr_o) ** 2))
    assert e_c < e_2, (e_c, e_2)
    dm.close()


@pytest.mark.parametrize("name,eps", [("logistic", 1e-3), ("logistic_mid", 2e-3), ("linear", 0.005),
                                      ("logistic_d128", 2e-3)])
def test_centred_leapfrog_trajectories(name, eps):
    """Ragged step counts 1..6: positions and momenta against the oracle's
    exact-gradient leapfrog (a gradient error dg moves p by at most S eps dg
    and theta by S^2 eps^2 dg), and the end-point energy against the oracle
    at the GPU's own end points."""
    w = rounded_workload(_cases()[name])
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
    g.check(g.lib().smc_k_target(dm.h, ptr(t_d), N, ld, ptr(lp_d), ptr(g_d), PREC, stream()), "target")
    s_d = dev(S)
    g.check(g.lib().smc_k_leapfrog(dm.h, ptr(t_d), ptr(p_d), ptr(g_d), ptr(lp_d), ptr(s_d), eps, N, ld, PREC,
                                   stream()), "leapfrog")
    th_g = t_d.cpu().numpy()[:, :N].T.astype(np.float64)
    p_g = p_d.cpu().numpy()[:, :N].T.astype(np.float64)
    lp_g = lp_d.cpu().numpy()[:N]
    th_o, p_o, _, _ = oracle.leapfrog(t, th, p, eps, S)
    c = th.mean(axis=0)
    dg = np.maximum(centred_bound(w, th, c), centred_bound(w, th_o, c))
    Sc = S[:, None].astype(np.float64)
    rms = lambda a: np.sqrt(np.mean(a**2))
    tol_p = (Sc + 1) * eps * dg + 1e-5 * Sc * (np.abs(p_o) + rms(p_o))
    tol_t = Sc**2 * eps**2 * dg + 1e-5 * Sc * (np.abs(th_o) + rms(th_o))
    assert np.all(np.abs(p_g - p_o) <= tol_p), np.max(np.abs(p_g - p_o) / tol_p)
    assert np.all(np.abs(th_g - th_o) <= tol_t), np.max(np.abs(th_g - th_o) / tol_t)
    lp_at_g, _ = oracle.logpi(t, th_g)
    assert np.all(np.abs(lp_g - lp_at_g) <= 1e-5 * _log_scale(w, th_g))
    # the cached gradient output is the move's end-point gradient
    _, gr_at_g = oracle.logpi(t, th_g)
    gr_g = g_d.cpu().numpy()[:, :N].T.astype(np.float64)
    assert np.all(np.abs(gr_g - gr_at_g) <= centred_bound(w, th_g, c) + 1e-4 * np.abs(gr_at_g))
    dm.close()


def test_centred_full_size_launch_on_sampled_particles():
    """The launch the benchmark times: n = 1e5 observations, D = 100,
    16384 particles (128 CTAs, 782 tiles of 128 observations).  Gradients and
    log pi of 24 sampled particles against the oracle."""
    w = rounded_workload(workloads.logistic_large())
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 16384
    th = _theta(w, N, seed=7)
    lp, gr = _target(dm, th, N)
    idx = np.sort(np.random.default_rng(11).choice(N, 24, replace=False))
    idx[-1] = N - 1
    _, gr_o = oracle.logpi(oracle_target(w), th[idx])
    lp_o, _ = oracle.logpi(oracle_target(w), th[idx])
    bound = centred_bound(w, th[idx], th.mean(axis=0))
    err = np.abs(gr[idx] - gr_o) / bound
    assert err.max() <= 1.0, err.max()
    assert np.all(np.abs(lp[idx] - lp_o) <= 1e-5 * _log_scale(w, th[idx]))
    dm.close()


def test_centred_eval_is_deterministic_and_tile_independent():
    """Each particle's result depends on its own state and the launch's
    reference point only: the same particles in another order (another tile
    assignment, the same mean) give identical bits."""
    w = rounded_workload(_cases()["logistic_mid"])
    dm = g.DevModel(g.ModelData.from_workload(w), stream())
    N = 300
    th = _theta(w, N, seed=12)
    perm = np.random.default_rng(13).permutation(N)
    out = []
    for order in (np.arange(N), perm):
        lp, gr = _target(dm, th[order], 320)
        a, b = np.empty_like(gr), np.empty_like(lp)
        a[order], b[order] = gr, lp
        out.append((a, b))
    # the mean is summed in a fixed order of the launch's particles, so a
    # permutation may change its last bit; allow exactly that and nothing else
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=0, atol=float(centred_bound(w, th, th.mean(0)).max()))
    np.testing.assert_array_equal(out[0][1], out[1][1])
    lp2, gr2 = _target(dm, th, 320)
    np.testing.assert_array_equal(gr2, out[0][0])
    dm.close()


def _sampler_case():
    lg = workloads.logistic(n=300, d_features=6)
    lg["run"] = dict(n_particles=600, n_iters=8, n_warmup=4, step_size=0.01, traj_len0=0.3,
                     max_steps=60, init_scale=1.0)
    return lg


def test_centred_iterations_keep_exact_weights():
    """Centred tensor-core trajectories in the sampler: resampling and step
    counts bit-exact, and Delta H from the oracle's FP64 log pi at the GPU's
    own end points and momenta matches to FP32 accuracy (the weights stay
    exact whatever the gradient precision); trajectories stay close to the
    exact-gradient ones."""
    w = rounded_workload(_sampler_case())
    run = w["run"]
    t = oracle_target(w)
    seed = 77
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=seed, precision=PREC, **run), stream())
    N, D, K = run["n_particles"], w["D"], run["n_iters"]
    for k in range(1, K + 1):
        pre = {"theta": smp.buffer(B.BUF_THETA).T.astype(np.float64), "logw": smp.buffer(B.BUF_LOGW)}
        lp_pre, _ = oracle.logpi(t, pre["theta"])
        np.testing.assert_allclose(smp.buffer(B.BUF_LOGPI), lp_pre, rtol=1e-6, atol=1e-6 * np.abs(lp_pre).max())
        st = smp.step()[0]
        _, ess, _ = oracle.normalise(pre["logw"])
        assert st["resampled"] == int(ess < 0.5 * N)
        src = np.arange(N)
        if st["resampled"]:
            _, q = oracle.quantise(smp.buffer(B.BUF_W))
            _, src = oracle.systematic(q, oracle.resample_r64(seed, k))
            np.testing.assert_array_equal(smp.buffer(B.BUF_ANCESTORS), src)
        L = smp.runstate()[0]["L_last"]
        S_o = np.array([oracle.step_count(oracle.halton2(j * K + k), L, run["step_size"], run["max_steps"])
                        for j in range(N)])
        np.testing.assert_array_equal(smp.buffer(B.BUF_STEPS), S_o)
        p0 = f32r(np.stack([oracle.normals(seed, oracle.TAG_MOM, k, j, D) for j in range(N)]))
        th1 = smp.buffer(B.BUF_THETA).T.astype(np.float64)
        p1 = smp.buffer(B.BUF_P_FINAL).T.astype(np.float64)
        lp1, _ = oracle.logpi(t, th1)
        dH_o = (0.5 * (p1**2).sum(1) - lp1) - (0.5 * (p0**2).sum(1) - lp_pre[src])
        dH = smp.buffer(B.BUF_DH)
        tol = 1e-5 * (np.abs(lp1) + np.abs(lp_pre[src]) + (p1**2).sum(1) + 1.0)
        assert np.all(np.abs(dH - dH_o) <= tol), np.max(np.abs(dH - dH_o) / tol)
        th1_o, _, _, _ = oracle.leapfrog(t, pre["theta"][src], p0, run["step_size"], S_o)
        rel = np.abs(th1 - th1_o) / (np.abs(th1_o) + np.sqrt(np.mean(th1_o**2)))
        assert np.median(rel) < 1e-3
    smp.close()


def test_centred_ten_run_batch_at_full_size_on_sampled_particles():
    """The batched configuration at full size, in the launch the benchmark
    times: ten runs of 4096 particles of the n = 1000, D = 25 regression in
    one centred handle (320 run-uniform tiles).  Per iteration and run the
    resampling decision, the ancestors and every step count are bit-exact
    against the oracle; on 24 sampled particles the momenta are the oracle's
    Philox normals, Delta H equals the oracle's FP64 energy difference at the
    GPU's own end points to FP32 accuracy (exact weights), and the end points
    stay close to the oracle's exact-gradient trajectories."""
    w = rounded_workload(workloads.logistic())
    run = dict(w["run"])
    t = oracle_target(w)
    R, N, D, K = 10, run["n_particles"], w["D"], run["n_iters"]
    seeds = [5000 + r for r in range(R)]
    smp = g.Sampler(g.ModelData.from_workload(w), [g.make_config(seed=sd, precision=PREC, **run) for sd in seeds],
                    stream())
    pick = np.sort(np.random.default_rng(2).choice(R * N, 24, replace=False))
    for k in range(1, 4):
        th_pre = smp.buffer(B.BUF_THETA).T.astype(np.float64)
        lw_pre = smp.buffer(B.BUF_LOGW)
        lp_pre_s = smp.buffer(B.BUF_LOGPI)
        stats = smp.step()
        W = smp.buffer(B.BUF_W)
        anc = smp.buffer(B.BUF_ANCESTORS)
        steps = smp.buffer(B.BUF_STEPS)
        rs = smp.runstate()
        src = np.arange(R * N)
        for r in range(R):
            sl = slice(r * N, (r + 1) * N)
            _, ess, _ = oracle.normalise(lw_pre[sl])
            assert stats[r]["resampled"] == int(ess < 0.5 * N), (k, r)
            if stats[r]["resampled"]:
                _, q = oracle.quantise(W[sl])
                _, a_o = oracle.systematic(q, oracle.resample_r64(seeds[r], k))
                np.testing.assert_array_equal(anc[sl], a_o)
                src[sl] = r * N + a_o
            L = rs[r]["L_last"]
            S_o = np.array([oracle.step_count(oracle.halton2(j * K + k), L, run["step_size"], run["max_steps"])
                            for j in range(N)])
            np.testing.assert_array_equal(steps[sl], S_o)
        th1 = smp.buffer(B.BUF_THETA).T.astype(np.float64)[pick]
        p1 = smp.buffer(B.BUF_P_FINAL).T.astype(np.float64)[pick]
        dH = smp.buffer(B.BUF_DH)[pick]
        p0 = f32r(np.stack([oracle.normals(seeds[i // N], oracle.TAG_MOM, k, i % N, D) for i in pick]))
        lp0, _ = oracle.logpi(t, th_pre[src[pick]])
        np.testing.assert_allclose(lp_pre_s[src[pick]], lp0, rtol=1e-6, atol=1e-6 * np.abs(lp0).max())
        lp1, _ = oracle.logpi(t, th1)
        dH_o = (0.5 * (p1**2).sum(1) - lp1) - (0.5 * (p0**2).sum(1) - lp0)
        tol = 1e-5 * (np.abs(lp1) + np.abs(lp0) + (p1**2).sum(1) + 1.0)
        assert np.all(np.abs(dH - dH_o) <= tol), (k, np.max(np.abs(dH - dH_o) / tol))
        th1_o, _, _, _ = oracle.leapfrog(t, th_pre[src[pick]], p0, run["step_size"], steps[pick])
        rel = np.abs(th1 - th1_o) / (np.abs(th1_o) + np.sqrt(np.mean(th1_o**2)))
        assert np.median(rel) < 1e-3, (k, np.median(rel))
    smp.close()


def test_centred_batched_runs_equal_single_runs_bit_for_bit():
    """Each run of a batch has its own reference point, so a run gives the
    same bits in a batch as alone."""
    w = _sampler_case()
    run = dict(w["run"])
    sizes = [300, 37, 1025]
    cfgs = [g.make_config(seed=500 + i, precision=PREC, **dict(run, n_particles=n)) for i, n in enumerate(sizes)]
    md = g.ModelData.from_workload(w)
    batch = g.Sampler(md, cfgs, stream())
    batch.run(run["n_iters"])
    th_b, lw_b = batch.particles()
    lz_b = batch.log_evidence()
    off = 0
    for i, n in enumerate(sizes):
        one = g.Sampler(md, cfgs[i], stream())
        one.run(run["n_iters"])
        th1, lw1 = one.particles()
        np.testing.assert_array_equal(th_b[:, off:off + n], th1)
        np.testing.assert_array_equal(lw_b[off:off + n], lw1)
        assert lz_b[i] == one.log_evidence()[0]
        off += n
        one.close()
    batch.close()


def test_centred_sixteen_ragged_runs_equal_single_runs_bit_for_bit():
    """Sixteen runs of sizes around the 128-particle tile (1, 127, 128, 129,
    ...): the run partition gives every tile one run's particles (padded run
    blocks), and each run's particles, weights and evidence are the same bits
    as when the run is alone."""
    w = _sampler_case()
    run = dict(w["run"], n_iters=4, n_warmup=2)
    sizes = [1, 127, 128, 129, 255, 256, 257, 3, 64, 200, 130, 2, 384, 99, 128, 31]
    cfgs = [g.make_config(seed=800 + i, precision=PREC, **dict(run, n_particles=n)) for i, n in enumerate(sizes)]
    md = g.ModelData.from_workload(w)
    batch = g.Sampler(md, cfgs, stream())
    batch.run(run["n_iters"])
    th_b, lw_b = batch.particles()
    lz_b = batch.log_evidence()
    batch.close()
    off = 0
    for i, n in enumerate(sizes):
        one = g.Sampler(md, cfgs[i], stream())
        one.run(run["n_iters"])
        th1, lw1 = one.particles()
        np.testing.assert_array_equal(th_b[:, off:off + n], th1)
        np.testing.assert_array_equal(lw_b[off:off + n], lw1)
        assert lz_b[i] == one.log_evidence()[0]
        off += n
        one.close()


def test_centred_handle_rejects_more_than_16_runs():
    w = _sampler_case()
    run = dict(w["run"], n_particles=64)
    cfgs = [g.make_config(seed=i, precision=PREC, **run) for i in range(17)]
    with pytest.raises(RuntimeError):
        g.Sampler(g.ModelData.from_workload(w), cfgs, stream())
