"""GPU parity of the learned preconditioner (affine-coupling transport map)
against the FP64 oracle, through the C-ABI:

* the training-loss gradient of every parameter (smc_k_flow_loss_grad);
* latent-space trajectories: z0 = T^-1(theta), leapfrog on log pi_z,
  theta' = T(z'), final momenta and the energy error in z
  (smc_k_flow_leapfrog), on ragged step counts;
* whole iterations with the map on (smc_flow_enable), stage by stage from the
  GPU's own state: latent buffers, trajectories, reweighting and the ChEES
  update computed in the latent space;
* one training iteration: the parameters after `epochs` Adam steps;
* the identity map (zero last layer) gives the plain sampler's results;
* a trained map raises acceptance and ESS on an ill-conditioned Gaussian.
"""
import numpy as np
import pytest

from gpu_util import dev, f32r, need_gpu, oracle_target, ptr, rounded_workload, stream, torch  # noqa: F401
import oracle
import paper_2504_02627_gb300 as g
import workloads
from paper_2504_02627_gb300 import _binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _params(D, H, L, seed, scale):
    """He-initialised hidden layers plus a non-zero last layer of size `scale`
    (a map away from the identity), rounded to FP32."""
    rng = np.random.default_rng(seed)
    p = workloads.flow_init(D, H, L, seed=seed)
    Dh = D // 2
    lsz = H * Dh + H + H * H + H + D * H + D
    for l in range(L):
        o = l * lsz + H * Dh + H + H * H + H
        p[o:o + D * H + D] = scale * rng.standard_normal(D * H + D) / np.sqrt(H)
    return f32r(p)


def _targets():
    ban = workloads.banana50()
    ban["eps"] = 0.02
    g10 = workloads.gauss10()
    g10["eps"] = 0.05
    g100 = workloads.gauss100_cond()
    g100["eps"] = 0.002
    return {"banana50": ban, "gauss10": g10, "gauss100": g100}


@pytest.mark.parametrize("D,H,L", [(10, 32, 4), (50, 128, 4), (100, 128, 4), (4, 8, 2)])
def test_loss_gradient_matches_oracle(D, H, L):
    N = 300                                              # 9 full CTAs and a ragged one
    rng = np.random.default_rng(D + H)
    p = _params(D, H, L, seed=D, scale=0.3)
    th = f32r(rng.standard_normal((N, D)) * 1.3)
    W = rng.uniform(0.0, 1.0, N)
    W /= W.sum()
    _, g_o = oracle.flow_loss_grad(oracle.FlowSpec(D, H, L, p), th, W)
    ld = 320
    th_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    th_d[:, :N] = dev(th.T, torch.float32)
    grad = torch.empty(p.size, dtype=torch.float32, device="cuda")
    p_d, W_d = dev(p, torch.float32), dev(W)          # kept alive across the asynchronous calls
    st = B.lib().smc_k_flow_loss_grad(D, H, L, ptr(p_d), ptr(th_d), ptr(W_d), N, ld, ptr(grad), 0, stream())
    assert st == 0
    torch.cuda.synchronize()
    g_gpu = grad.cpu().numpy().astype(np.float64)
    # per parameter block: FP32 sums over 300 particles through L layers
    Dh = D // 2
    sizes = [H * Dh, H, H * H, H, D * H, D]
    o = 0
    for l in range(L):
        for sz in sizes:
            go, gg = g_o[o:o + sz], g_gpu[o:o + sz]
            rms = np.sqrt(np.mean(go**2)) + 1e-12
            err = np.abs(gg - go) / (np.abs(go) + rms)
            assert err.max() < 2e-4, (l, sz, err.max())
            o += sz
    # identical inputs give identical bits (fixed-order reduction)
    grad2 = torch.empty_like(grad)
    assert B.lib().smc_k_flow_loss_grad(D, H, L, ptr(p_d), ptr(th_d), ptr(W_d), N, ld, ptr(grad2), 0,
                                        stream()) == 0
    torch.cuda.synchronize()
    assert torch.equal(grad, grad2)


def _gpu_loss_grad(D, H, L, p, th, W, precision, reps=1):
    """smc_k_flow_loss_grad on N particles (theta padded to a 32-multiple
    leading dimension); returns `reps` gradients of identical calls."""
    N = th.shape[0]
    ld = ((N + 31) // 32) * 32 + 32
    th_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    th_d[:, :N] = dev(th.T, torch.float32)
    p_d, W_d = dev(p, torch.float32), dev(W)
    out = []
    for _ in range(reps):
        grad = torch.empty(p.size, dtype=torch.float32, device="cuda")
        st = B.lib().smc_k_flow_loss_grad(D, H, L, ptr(p_d), ptr(th_d), ptr(W_d), N, ld, ptr(grad), precision,
                                          stream())
        assert st == 0
        out.append(grad)
    torch.cuda.synchronize()
    return [x.cpu().numpy().astype(np.float64) for x in out]


@pytest.mark.parametrize("D,H,L", [(10, 32, 4), (50, 128, 4), (100, 128, 4), (4, 16, 2)])
def test_bf16_loss_gradient_near_oracle(D, H, L):
    """The training gradient with its products on BF16 warp MMAs against the
    FP64 oracle.  A product of two operands rounded to BF16 (unit roundoff
    u = 2^-8) is off by at most 2u relative to its terms, and the gradient of
    a layer-l parameter sits at the end of a chain of at most 6 L such
    products (3 L in the inverse pass, 3 per backward layer up to l, the
    weight-gradient product last).  First order, a block's norm-wise error and
    an element's error relative to |g| + rms(g) are below 12 L u (0.19 at
    L = 4), and with independent roundings the typical block below
    sqrt(6 L) u (1.9e-2 at L = 4); measured, the block medians are 3.5e-3 to
    4.5e-3 (about u), the worst block 7.5e-3 and the worst element 4e-2.  A
    wrong fragment, operand layout or row map gives order one (a lost row:
    about 0.5).  Identical inputs give identical bits."""
    N = 300
    rng = np.random.default_rng(D + H)
    p = _params(D, H, L, seed=D, scale=0.3)
    th = f32r(rng.standard_normal((N, D)) * 1.3)
    W = rng.uniform(0.0, 1.0, N)
    W /= W.sum()
    _, g_o = oracle.flow_loss_grad(oracle.FlowSpec(D, H, L, p), th, W)
    g_gpu, g_again = _gpu_loss_grad(D, H, L, p, th, W, 2, reps=2)
    np.testing.assert_array_equal(g_gpu, g_again)
    Dh = D // 2
    sizes = [H * Dh, H, H * H, H, D * H, D]
    u = 2.0**-8
    bound = 12 * L * u
    o, worst = 0, []
    for l in range(L):
        for sz in sizes:
            go, gg = g_o[o:o + sz], g_gpu[o:o + sz]
            nrm = np.linalg.norm(gg - go) / (np.linalg.norm(go) + 1e-30)
            rel = np.abs(gg - go) / (np.abs(go) + np.sqrt(np.mean(go**2)) + 1e-30)
            worst.append(nrm)
            assert nrm < bound and rel.max() < bound, (l, sz, nrm, rel.max(), bound)
            o += sz
    # the typical block is near the independent-rounding estimate, not the bound
    assert np.median(worst) < 2 * np.sqrt(6 * L) * u, (np.median(worst), max(worst))


@pytest.mark.parametrize("precision", [0, 2])
def test_loss_gradient_at_the_benchmark_size(precision):
    """The training gradient at the benchmark's shape (the 100-d Gaussian's
    map: D = 100, H = 128, L = 4, 8192 particles, 256 CTAs and their
    fixed-order reduction) against the FP64 oracle's full gradient: FP32
    within 2e-4 of the block scale as at 300 particles (the per-CTA partials
    add 256 FP32 terms per parameter), BF16 within the chain-length bound of
    test_bf16_loss_gradient_near_oracle."""
    D, H, L, N = 100, 128, 4, 8192
    rng = np.random.default_rng(77)
    p = _params(D, H, L, seed=3, scale=0.3)
    th = f32r(rng.standard_normal((N, D)))
    W = np.full(N, 1.0 / N)
    _, g_o = oracle.flow_loss_grad(oracle.FlowSpec(D, H, L, p), th, W)
    g_gpu = _gpu_loss_grad(D, H, L, p, th, W, precision)[0]
    Dh = D // 2
    sizes = [H * Dh, H, H * H, H, D * H, D]
    bound = 2e-4 if precision == 0 else 12 * L * 2.0**-8
    o = 0
    for l in range(L):
        for sz in sizes:
            go, gg = g_o[o:o + sz], g_gpu[o:o + sz]
            rel = np.abs(gg - go) / (np.abs(go) + np.sqrt(np.mean(go**2)) + 1e-30)
            nrm = np.linalg.norm(gg - go) / (np.linalg.norm(go) + 1e-30)
            assert rel.max() < bound and nrm < bound, (l, sz, rel.max(), nrm, bound)
            o += sz


def test_bf16_training_from_the_identity_map():
    """From a zero last layer the transposed product W3^T c_o is exactly zero
    in BF16 too, so one BF16-trained Adam step moves only W3 and b3, each by
    lr * sign(gradient) up to Adam's eps, as the FP64 oracle's step; a
    gradient below the BF16 noise may take the other sign."""
    D, H, L, lr = 10, 32, 4, 1e-3
    p_init = f32r(workloads.flow_init(D, H, L, seed=5))
    p_gpu, p_o = _train_case(p_init, 1, lr, train_precision=2)
    Dh = D // 2
    lsz = H * Dh + H + H * H + H + D * H + D
    for l in range(L):
        o = l * lsz
        hid = slice(o, o + H * Dh + 2 * H + H * H)
        np.testing.assert_array_equal(p_gpu[hid], p_init[hid])
        last = slice(o + H * Dh + 2 * H + H * H, o + lsz)
        d = np.abs(p_gpu[last] - p_o[last])
        assert np.all(d <= 2 * lr + 1e-7)
        assert np.mean(d <= 1e-3 * lr) > 0.95, np.mean(d <= 1e-3 * lr)


def oracle_flow_move(f, t, theta, p0, eps, S):
    """Algorithm 1 on log pi_z from z0 = T^-1(theta) with momenta p0 and S_j
    steps, through the oracle's flow_logpi_z; returns theta' = T(z'), p',
    z0, z', log pi(theta'), Delta H in z, grad log pi(theta')."""
    z0, ldi = oracle.flow_inverse(f, theta)
    lpz, gz, x, gx, lpx = oracle.flow_logpi_z(f, t, z0)
    H0 = 0.5 * (p0**2).sum(1) - lpz
    z, p = z0.copy(), p0.copy()
    for s in range(int(S.max())):
        a = S > s
        p[a] += 0.5 * eps * gz[a]
        z[a] += eps * p[a]
        lpz_a, gz_a, x_a, gx_a, lpx_a = oracle.flow_logpi_z(f, t, z[a])
        lpz[a], gz[a], x[a], gx[a], lpx[a] = lpz_a, gz_a, x_a, gx_a, lpx_a
        p[a] += 0.5 * eps * gz[a]
    dH = 0.5 * (p**2).sum(1) - lpz - H0
    return x, p, z0, z, lpx, dH, gx


def _assert_close(a, b, S, what, rel=2e-5):
    scale = np.sqrt(np.mean(b**2)) + 1e-3
    tol = rel * S[:, None] * (np.abs(b) + scale)
    r = np.abs(a - b) / tol
    i, d = np.unravel_index(np.argmax(r), r.shape)
    assert r.max() <= 1.0, (what, r.max(), "particle", i, "dim", d, a[i, d], b[i, d], "steps", S[i],
                            "particles over", int((r.max(1) > 1).sum()))


@pytest.mark.parametrize("name", ["banana50", "gauss10", "gauss100"])
def test_latent_leapfrog_matches_oracle(name):
    w = rounded_workload(_targets()[name])
    D, eps = w["D"], w["eps"]
    t = oracle_target(w)
    H, L = (32, 4) if D <= 10 else (128, 4)
    p = _params(D, H, L, seed=7, scale=0.1)
    f = oracle.FlowSpec(D, H, L, p)
    N = 77                                               # 2 full CTAs and a ragged one
    rng = np.random.default_rng(3)
    Sigma = w.get("Sigma")
    if Sigma is not None:
        th = f32r(rng.standard_normal((N, D)) @ np.linalg.cholesky(Sigma).T)
    else:
        xo = rng.standard_normal((N, D // 2)) * np.sqrt(w["a"])
        xe = rng.standard_normal((N, D // 2)) + w["b"] * (xo**2 - w["a"])
        th = f32r(np.stack([xo, xe], axis=2).reshape(N, D))
    p0 = f32r(rng.standard_normal((N, D)))
    S = rng.integers(1, 9, N).astype(np.int32)
    lp, gr = oracle.logpi(t, th)
    x_o, p_o, z0_o, z1_o, lpx_o, dH_o, gx_o = oracle_flow_move(f, t, th, p0, eps, S)

    m = g.DevModel(g.ModelData.from_workload(w), stream())
    ld = 96
    def buf(a):
        out = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
        out[:, :N] = dev(a.T, torch.float32)
        return out
    th_d, p_d, gr_d = buf(th), buf(p0), buf(f32r(gr))
    lp_d = dev(lp)
    z0_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    z1_d = torch.zeros_like(z0_d)
    dH_d = torch.zeros(N, dtype=torch.float64, device="cuda")
    par_d, S_d = dev(p, torch.float32), dev(S)       # kept alive across the asynchronous call
    st = B.lib().smc_k_flow_leapfrog(m.h, H, L, ptr(par_d), ptr(th_d), ptr(p_d), ptr(gr_d), ptr(lp_d), ptr(S_d),
                                     eps, N, ld, ptr(z0_d), ptr(z1_d), ptr(dH_d), 0, stream())
    assert st == 0
    torch.cuda.synchronize()
    host = lambda a: a[:, :N].cpu().numpy().T.astype(np.float64)
    one = np.ones(N)
    _assert_close(host(z0_d), z0_o, one, "z0")
    _assert_close(host(z1_d), z1_o, S, "z'")
    _assert_close(host(p_d), p_o, S, "p'")
    _assert_close(host(th_d), x_o, S, "theta'")
    _assert_close(host(gr_d), gx_o, S, "grad'")
    lp1 = lp_d.cpu().numpy()
    assert np.all(np.abs(lp1 - lpx_o) <= 2e-5 * S * (np.abs(lpx_o) + 1.0))
    dH = dH_d.cpu().numpy()
    dh_tol = 2e-5 * S * (np.abs(lpx_o) + 0.5 * (p_o**2).sum(1) + 1.0)
    assert np.all(np.abs(dH - dH_o) <= dh_tol), np.max(np.abs(dH - dH_o) / dh_tol)
    m.close()


def _flow_case(name):
    if name == "banana50":
        w = workloads.banana50()
        w["run"] = dict(n_particles=400, n_iters=5, n_warmup=3, step_size=0.02, traj_len0=0.2,
                        max_steps=20, init_scale=1.0)
        return w, (128, 4)
    w = workloads.gauss10()
    w["run"] = dict(n_particles=300, n_iters=6, n_warmup=4, step_size=0.05, traj_len0=0.3,
                    max_steps=20, init_scale=2.0)
    return w, (32, 4)


@pytest.mark.parametrize("name", ["gauss10", "banana50"])
def test_flow_iterations_match_oracle_stage_by_stage(name):
    w, (H, L) = _flow_case(name)
    w = rounded_workload(w)
    run = w["run"]
    t = oracle_target(w)
    D, N, K, eps = w["D"], run["n_particles"], run["n_iters"], run["step_size"]
    params = _params(D, H, L, seed=11, scale=0.1)
    f = oracle.FlowSpec(D, H, L, params)
    seed = 77
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=seed, **run), stream())
    smp.enable_flow(params, H, L, train_every=0, epochs=0)
    ocfg = oracle.SMCConfig(seed=seed, n_particles=N, n_iters=K, n_warmup=run["n_warmup"], step_size=eps,
                            traj_len0=run["traj_len0"], max_steps=run["max_steps"], init_scale=run["init_scale"])
    for k in range(1, K + 1):
        pre = {"theta": smp.buffer(B.BUF_THETA).T.astype(np.float64), "logw": smp.buffer(B.BUF_LOGW),
               "rs": smp.runstate()[0]}
        st = smp.step()[0]
        lse, ess, W_o = oracle.normalise(pre["logw"])
        W = smp.buffer(B.BUF_W)
        np.testing.assert_allclose(W, W_o, rtol=1e-12, atol=1e-300)
        if st["resampled"]:
            _, q = oracle.quantise(W)
            _, src = oracle.systematic(q, oracle.resample_r64(seed, k))
            np.testing.assert_array_equal(smp.buffer(B.BUF_ANCESTORS), src)
        else:
            src = np.arange(N)
        th_start = pre["theta"][src]
        L_k = smp.runstate()[0]["L_last"]
        h = np.array([oracle.halton2(j * K + k) for j in range(N)])
        S = np.array([oracle.step_count(x, L_k, eps, run["max_steps"]) for x in h], dtype=np.int32)
        np.testing.assert_array_equal(smp.buffer(B.BUF_STEPS), S)
        p0 = f32r(np.stack([oracle.normals(seed, oracle.TAG_MOM, k, j, D) for j in range(N)]))
        x_o, p_o, z0_o, z1_o, lpx_o, dH_o, _ = oracle_flow_move(f, t, th_start, p0, eps, S)
        dH = smp.buffer(B.BUF_DH)
        div = ~(np.abs(dH_o) < 50.0)
        assert np.all(~(np.abs(dH[div]) < 30.0)), k
        ok = ~div
        assert ok.mean() > 0.5, (k, ok.mean())
        _assert_close(smp.buffer(B.BUF_Z0).T[ok].astype(np.float64), z0_o[ok], np.ones(ok.sum()), "z0")
        _assert_close(smp.buffer(B.BUF_Z1).T[ok].astype(np.float64), z1_o[ok], S[ok], "z'")
        _assert_close(smp.buffer(B.BUF_P_FINAL).T[ok].astype(np.float64), p_o[ok], S[ok], "p'")
        _assert_close(smp.buffer(B.BUF_THETA).T[ok].astype(np.float64), x_o[ok], S[ok], "theta'")
        dh_tol = 2e-5 * S * (np.abs(lpx_o) + 0.5 * (p_o**2).sum(1) + 1.0)
        assert np.all((np.abs(dH - dH_o) <= dh_tol)[ok]), k
        alpha = smp.buffer(B.BUF_ALPHA)
        base = np.full(N, -np.log(N)) if st["resampled"] else pre["logw"]
        np.testing.assert_allclose(smp.buffer(B.BUF_LOGW), base - dH, rtol=1e-14, atol=1e-12)
        # ChEES in the latent space, from the GPU's latent buffers
        rs = smp.runstate()[0]
        ch = oracle.CheesState(pre["rs"]["log_L"], pre["rs"]["adam_m"], pre["rs"]["adam_v"],
                               int(pre["rs"]["adam_t"]), pre["rs"]["Lbar"])
        if k < run["n_warmup"]:
            z0 = smp.buffer(B.BUF_Z0).T.astype(np.float64)
            z1 = smp.buffer(B.BUF_Z1).T.astype(np.float64)
            p1 = smp.buffer(B.BUF_P_FINAL).T.astype(np.float64)
            ghat, _ = oracle.chees_gradient(z0, z1, p1, h * L_k, alpha)
            if ghat is not None:
                oracle.chees_adam(ch, ghat, ocfg.adam_lr, ocfg.adam_b1, ocfg.adam_b2, ocfg.adam_eps, eps,
                                  run["max_steps"])
            ch.Lbar = 0.9 * ch.Lbar + 0.1 * np.exp(ch.log_L)
        if k == run["n_warmup"] and ch.Lbar > 0:
            ch.log_L = np.log(ch.Lbar)
        assert abs(rs["log_L"] - ch.log_L) <= 1e-9 * max(1.0, abs(ch.log_L)), (k, rs["log_L"], ch.log_L)
    smp.close()


def _train_case(p_init, E, lr, seed=9, train_precision=0):
    """GPU iteration 1 with training on (its products in FP32 or BF16);
    returns the GPU parameters after it and the oracle's parameters after E
    Adam steps on the same particles."""
    w = rounded_workload(workloads.gauss10())
    run = dict(n_particles=512, n_iters=6, n_warmup=4, step_size=0.05, traj_len0=0.3, max_steps=20,
               init_scale=2.0)
    D, H, L = 10, 32, 4
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=seed, **run), stream())
    smp.enable_flow(p_init, H, L, train_every=1, epochs=E, lr=lr, min_ess_frac=0.0, train_precision=train_precision)
    th0 = smp.buffer(B.BUF_THETA).T.astype(np.float64)
    logw0 = smp.buffer(B.BUF_LOGW)
    st = smp.step()[0]
    _, _, W = oracle.normalise(logw0)
    if st["resampled"]:
        _, q = oracle.quantise(smp.buffer(B.BUF_W))
        _, src = oracle.systematic(q, oracle.resample_r64(seed, 1))
        th, Wt = th0[src], np.full(run["n_particles"], 1.0 / run["n_particles"])
    else:
        th, Wt = th0, W
    fs = oracle.new_flow_state(p_init, H, L)
    for e in range(1, E + 1):
        _, gr = oracle.flow_loss_grad(oracle.FlowSpec(D, H, L, fs["params"]), th, Wt)
        oracle.flow_adam(fs["params"], gr, fs["m"], fs["v"], e, lr)
    p_gpu = smp.flow_params()
    smp.close()
    return p_gpu, fs["params"]


def test_training_from_the_identity_map_matches_oracle():
    """From a zero last layer one Adam step moves only W3 and b3 (every other
    gradient is exactly zero), each by lr * sign(gradient) up to Adam's eps;
    a gradient below the FP32 noise may take the other sign."""
    D, H, L, lr = 10, 32, 4, 1e-3
    p_init = f32r(workloads.flow_init(D, H, L, seed=5))
    p_gpu, p_o = _train_case(p_init, 1, lr)
    Dh = D // 2
    lsz = H * Dh + H + H * H + H + D * H + D
    for l in range(L):
        o = l * lsz
        hid = slice(o, o + H * Dh + 2 * H + H * H)
        np.testing.assert_array_equal(p_gpu[hid], p_init[hid])
        last = slice(o + H * Dh + 2 * H + H * H, o + lsz)
        d = np.abs(p_gpu[last] - p_o[last])
        assert np.all(d <= 2 * lr + 1e-7)
        assert np.mean(d <= 1e-3 * lr) > 0.99, np.mean(d <= 1e-3 * lr)


def test_training_epochs_match_oracle_adam():
    """Several Adam steps from a non-identity map.  Adam moves a parameter by
    about lr * sign(gradient) early on, so one whose gradient is below the
    FP32 noise may move the other way; what is unique is compared: almost
    every parameter agrees closely, none is further than 2 * epochs * lr."""
    D, H, L, E, lr = 10, 32, 4, 3, 1e-3
    p_init = _params(D, H, L, seed=12, scale=0.3)
    p_gpu, p_o = _train_case(p_init, E, lr)
    d = np.abs(p_gpu - p_o)
    assert np.all(d <= 2 * E * lr + 1e-6)
    close = d <= 1e-2 * lr * E + 1e-7
    assert np.mean(close) > 0.995, np.mean(close)


def test_training_gate_skips_a_degenerate_weighted_set():
    """Iteration 1 of the 10-d Gaussian starts from N(0, 4 I): its tested ESS
    is far below 0.9 J, so with min_ess_frac = 0.9 the map must not move."""
    w = rounded_workload(workloads.gauss10())
    run = dict(n_particles=512, n_iters=6, n_warmup=4, step_size=0.05, traj_len0=0.3, max_steps=20,
               init_scale=2.0)
    p_init = _params(10, 32, 4, seed=12, scale=0.3)
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=9, **run), stream())
    smp.enable_flow(p_init, 32, 4, train_every=1, epochs=5, lr=1e-3, min_ess_frac=0.9)
    st = smp.step()[0]
    assert st["ess_pre"] < 0.9 * run["n_particles"]
    np.testing.assert_array_equal(smp.flow_params(), p_init)
    smp.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_identity_map_gives_the_plain_sampler(precision):
    """With a zero last layer and no training, T is the identity (s = 0,
    t = 0 exactly, in BF16 too), so the preconditioned sampler must reproduce
    the plain one: identical decisions and step counts, trajectories within FP32."""
    w = rounded_workload(workloads.gauss10())
    run = dict(n_particles=256, n_iters=8, n_warmup=4, step_size=0.05, traj_len0=0.3, max_steps=20,
               init_scale=2.0)
    plain = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=5, **run), stream())
    flow = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=5, **run), stream())
    flow.enable_flow(f32r(workloads.flow_init(10, 32, 4)), 32, 4, train_every=0, epochs=0, precision=precision)
    for k in range(run["n_iters"]):
        sp, sf = plain.step()[0], flow.step()[0]
        assert sp["resampled"] == sf["resampled"]
        np.testing.assert_array_equal(plain.buffer(B.BUF_STEPS), flow.buffer(B.BUF_STEPS))
        np.testing.assert_allclose(flow.buffer(B.BUF_THETA), plain.buffer(B.BUF_THETA), rtol=2e-4, atol=2e-4)
        np.testing.assert_allclose(flow.buffer(B.BUF_DH), plain.buffer(B.BUF_DH), rtol=1e-3, atol=2e-4)
        src = flow.buffer(B.BUF_ANCESTORS) if sf["resampled"] else np.arange(run["n_particles"])
        np.testing.assert_array_equal(flow.buffer(B.BUF_Z0), flow.buffer(B.BUF_THETA_PREV)[:, src])
    plain.close()
    flow.close()


@pytest.mark.parametrize("precision,train_precision", [(0, 0), (2, 0), (2, 2)])
def test_trained_map_raises_acceptance_and_ess(precision, train_precision):
    """Ill-conditioned 4-d Gaussian (variances 0.01 .. 4) at a step size the
    stiff direction barely tolerates (the oracle's pin of the same claim):
    training the map on the particles whitens the target (with the map's
    products in FP32 or BF16, and its training products in FP32 or BF16)."""
    tgt = workloads._gauss_from_spectrum(np.array([0.01, 0.1, 1.0, 4.0]), 11)
    w = rounded_workload(tgt)
    run = dict(n_particles=512, n_iters=16, n_warmup=12, step_size=0.18, traj_len0=1.0, max_steps=500,
               init_scale=1.0, adapt=0)
    md = g.ModelData.from_workload(w)
    plain = g.Sampler(md, g.make_config(seed=21, **run), stream())
    flow = g.Sampler(md, g.make_config(seed=21, **run), stream())
    flow.enable_flow(f32r(workloads.flow_init(4, 32, 4, seed=5)), 32, 4, train_every=1, epochs=60, lr=3e-3,
                     precision=precision, train_precision=train_precision)
    sp = [plain.step()[0] for _ in range(run["n_iters"])]
    sf = []
    for k in range(run["n_iters"]):
        try:
            sf.append(flow.step()[0])
        except RuntimeError as e:
            p = flow.flow_params()
            raise AssertionError((k, str(e), "finite params", bool(np.isfinite(p).all()),
                                  [(x["ess"], x["mean_alpha"]) for x in sf])) from e
    last = lambda s, key: np.mean([x[key] for x in s[-4:]])
    assert last(sf, "mean_alpha") > last(sp, "mean_alpha") + 0.1, (last(sf, "mean_alpha"), last(sp, "mean_alpha"))
    assert last(sf, "ess") > 1.3 * last(sp, "ess"), (last(sf, "ess"), last(sp, "ess"))
    plain.close()
    flow.close()


def test_flow_rejects_unsupported_configurations():
    w = rounded_workload(workloads.logistic(n=100, d_features=5))
    w["run"] = dict(n_particles=64, n_iters=4, n_warmup=2, step_size=0.01, traj_len0=0.1, max_steps=10,
                    init_scale=1.0)
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=1, **w["run"]), stream())
    with pytest.raises(RuntimeError):
        smp.enable_flow(np.zeros(B.lib().smc_flow_num_params(6, 32, 4)), 32, 4)
    smp.close()
    w = rounded_workload(workloads.gauss10())
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=1, n_particles=64, n_iters=4, n_warmup=2,
                                                                step_size=0.05), stream())
    with pytest.raises(RuntimeError):
        smp.enable_flow(np.zeros(B.lib().smc_flow_num_params(10, 30, 4)), 30, 4)     # H not a multiple of 4
    with pytest.raises(RuntimeError):                                                  # BF16: H not a multiple of 16
        smp.enable_flow(np.zeros(B.lib().smc_flow_num_params(10, 40, 4)), 40, 4, precision=2)
    with pytest.raises(RuntimeError):                                                  # BF16 training: the same
        smp.enable_flow(np.zeros(B.lib().smc_flow_num_params(10, 40, 4)), 40, 4, train_precision=2)
    with pytest.raises(RuntimeError):                                                  # no such training precision
        smp.enable_flow(np.zeros(B.lib().smc_flow_num_params(10, 32, 4)), 32, 4, train_precision=1)
    # the kernel-level training gradient: precision FP32 or BF16 only, BF16 with hidden a multiple of 16
    g_d = torch.empty(B.lib().smc_flow_num_params(10, 40, 4), dtype=torch.float32, device="cuda")
    assert B.lib().smc_k_flow_loss_grad(10, 40, 4, ptr(g_d), None, None, 0, 0, ptr(g_d), 1, stream()) == B.SMC_E_INVAL
    assert B.lib().smc_k_flow_loss_grad(10, 40, 4, ptr(g_d), None, None, 0, 0, ptr(g_d), 2, stream()) == B.SMC_E_INVAL
    smp.step()
    with pytest.raises(RuntimeError):                                                  # after the first iteration
        smp.enable_flow(np.zeros(B.lib().smc_flow_num_params(10, 32, 4)), 32, 4)
    smp.close()


# ------------------------------------------------------------- BF16 conditioner products
def _gpu_flow_move(w, H, L, p, th, p0, S, eps, precision):
    """smc_k_flow_leapfrog on the given particles; returns host arrays
    (theta', p', z0, z', grad', log pi', dH) and the starting log pi, grad."""
    D = w["D"]
    N = th.shape[0]
    t = oracle_target(w)
    lp, gr = oracle.logpi(t, th)
    m = g.DevModel(g.ModelData.from_workload(w), stream())
    ld = ((N + 31) // 32) * 32

    def buf(a):
        out = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
        out[:, :N] = dev(a.T, torch.float32)
        return out
    th_d, p_d, gr_d = buf(th), buf(p0), buf(f32r(gr))
    lp_d = dev(lp)
    z0_d = torch.zeros((D, ld), dtype=torch.float32, device="cuda")
    z1_d = torch.zeros_like(z0_d)
    dH_d = torch.zeros(N, dtype=torch.float64, device="cuda")
    par_d, S_d = dev(p, torch.float32), dev(S)
    st = B.lib().smc_k_flow_leapfrog(m.h, H, L, ptr(par_d), ptr(th_d), ptr(p_d), ptr(gr_d), ptr(lp_d), ptr(S_d),
                                     eps, N, ld, ptr(z0_d), ptr(z1_d), ptr(dH_d), precision, stream())
    assert st == 0
    torch.cuda.synchronize()
    host = lambda a: a[:, :N].cpu().numpy().T.astype(np.float64)
    out = (host(th_d), host(p_d), host(z0_d), host(z1_d), host(gr_d), lp_d.cpu().numpy(), dH_d.cpu().numpy())
    m.close()
    return out, lp, gr


def _start_points(w, N, seed):
    rng = np.random.default_rng(seed)
    D = w["D"]
    Sigma = w.get("Sigma")
    if Sigma is not None:
        th = f32r(rng.standard_normal((N, D)) @ np.linalg.cholesky(Sigma).T)
    else:
        xo = rng.standard_normal((N, D // 2)) * np.sqrt(w["a"])
        xe = rng.standard_normal((N, D // 2)) + w["b"] * (xo**2 - w["a"])
        th = f32r(np.stack([xo, xe], axis=2).reshape(N, D))
    return th, f32r(rng.standard_normal((N, D)))


@pytest.mark.parametrize("name", ["banana50", "gauss10", "gauss100"])
def test_bf16_transport_round_trip_is_exact(name):
    """The BF16 map is a deterministic affine coupling, so T(T^-1(theta)) =
    theta up to the FP32 affine arithmetic and the energy of a particle that
    does not move is unchanged: the property that keeps the preconditioned
    sampler exact with reduced-precision conditioners."""
    w = rounded_workload(_targets()[name])
    D, eps = w["D"], w["eps"]
    H, L = (32, 4) if D <= 10 else (128, 4)
    p = _params(D, H, L, seed=7, scale=0.3)
    N = 77
    th, p0 = _start_points(w, N, 3)
    S = np.random.default_rng(4).integers(1, 5, N).astype(np.int32)
    S[::2] = 0                                            # half the particles stay at z0
    (th1, p1, z0, z1, gr1, lp1, dH), lp, gr = _gpu_flow_move(w, H, L, p, th, p0, S, eps, 2)
    for a in (th1, p1, z0, z1, gr1, lp1, dH):
        assert np.all(np.isfinite(a))
    still = S == 0
    scale = np.sqrt(np.mean(th**2))
    np.testing.assert_allclose(th1[still], th[still], rtol=1e-4, atol=1e-4 * scale)
    np.testing.assert_array_equal(z1[still], z0[still])
    np.testing.assert_array_equal(p1[still], p0[still])
    gs = np.sqrt(np.mean(gr**2))
    np.testing.assert_allclose(gr1[still], gr[still], rtol=1e-3, atol=1e-3 * gs)
    np.testing.assert_allclose(lp1[still], lp[still], rtol=1e-5, atol=1e-4)
    assert np.all(np.abs(dH[still]) <= 2e-3 + 1e-6 * np.abs(lp[still])), np.abs(dH[still]).max()


@pytest.mark.parametrize("name,N", [("banana50", 77), ("gauss10", 77), ("gauss100", 77), ("gauss100", 8192)])
def test_bf16_latent_leapfrog_near_oracle(name, N):
    """One latent leapfrog step with BF16 conditioner products against the FP64
    oracle map.  BF16 rounds weights and activations (unit roundoff 2^-8): the map
    (z0, theta') carries errors of about 2e-3 of its scale (bound 2e-2), and the
    latent gradient, whose vector-Jacobian products pass through the twelve
    BF16 products of the four layers twice, up to 5e-2 of the gradient scale
    (median 4e-3; bound 0.1).  A wrong fragment or operand layout gives order
    one.  At the benchmark's 8192 particles a seeded sample of 100 is checked."""
    w = rounded_workload(_targets()[name])
    D, eps = w["D"], w["eps"]
    t = oracle_target(w)
    H, L = (32, 4) if D <= 10 else (128, 4)
    p = _params(D, H, L, seed=7, scale=0.1)
    f = oracle.FlowSpec(D, H, L, p)
    th, p0 = _start_points(w, N, 5)
    S = np.ones(N, dtype=np.int32)
    (th1, p1, z0, z1, gr1, lp1, dH), _, _ = _gpu_flow_move(w, H, L, p, th, p0, S, eps, 2)
    idx = np.arange(N) if N <= 100 else np.sort(np.random.default_rng(N).choice(N, 100, replace=False))
    x_o, p_o, z0_o, z1_o, lpx_o, dH_o, gx_o = oracle_flow_move(f, t, th[idx], p0[idx], eps, S[idx])
    rel = lambda a, b: np.abs(a - b) / (np.abs(b) + np.sqrt(np.mean(b**2)) + 1e-6)
    assert rel(z0[idx], z0_o).max() < 2e-2, rel(z0[idx], z0_o).max()
    assert rel(th1[idx], x_o).max() < 2e-2, rel(th1[idx], x_o).max()
    # p' = p0 + eps/2 (g0 + g1): the latent gradients carry the conditioner error
    _, g0_o, _, _, _ = oracle.flow_logpi_z(f, t, z0_o)
    _, g1_o, _, _, _ = oracle.flow_logpi_z(f, t, z1_o)
    gscale = np.abs(g0_o) + np.abs(g1_o) + np.sqrt(np.mean(g0_o**2))
    assert np.all(np.abs(p1[idx] - p_o) <= 0.5 * eps * 0.1 * gscale + 1e-5 * (np.abs(p_o) + 1.0))
    assert rel(lp1[idx], lpx_o).max() < 2e-2
