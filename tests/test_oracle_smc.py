"""Pins for the whole oracle sampler (Algorithm 3 with the ChEES-HMC proposal).

Closed forms, over R = 30 seeds (the log-evidence estimate is skewed, so fewer seeds
understate its spread), within 3 Monte Carlo standard errors
(MCSE = sd across seeds / sqrt(R)):
* conjugate Gaussian N(mu, Sigma): weighted mean and variance, and the
  log evidence (D/2) log 2 pi + 1/2 log det Sigma of exp(-1/2 (t-mu)'P(t-mu));
* Bayesian linear-Gaussian regression: the evidence N(y; 0, s^2 I + t^2 XX').
The evidence estimator is only as good as the initial importance step (it is
the product of that step's estimate with per-iteration factors of mean one),
so these targets keep q_init close to the posterior.
Structural invariants: step counts without jitter, the resampling rule,
evidence bookkeeping, the accept-reject variant, and the degenerate status.
The paper's Table 1 (1-d Halton, 5-d Gaussian: 8.01 gradient evaluations per
particle) is a loose statistical check only: the Adam constants are unpinned.
"""
import json
import os

import numpy as np
from scipy import stats

import oracle
import workloads

R = 30


def _runs(t, **kw):
    out = []
    for s in range(workloads.RUN_SEEDS[0], workloads.RUN_SEEDS[0] + R):
        cfg = oracle.SMCConfig(seed=s, **kw)
        r = oracle.smc_run(t, cfg)
        assert r["status"] == 0
        m, v = oracle.moments(r["theta"], r["logw"])
        out.append((r["log_z"], m, v, r["stats"]))
    return out


def _within_3_mcse(samples, truth):
    samples = np.asarray(samples)
    mcse = samples.std(axis=0, ddof=1) / np.sqrt(samples.shape[0])
    return np.abs(samples.mean(axis=0) - truth) <= 3.0 * mcse + 1e-12


def test_gaussian_moments_and_evidence():
    mu = np.array([0.5, -0.3, 0.2])
    var = np.array([0.5, 1.0, 2.0])
    t = oracle.TargetSpec.gauss_dense(mu, np.diag(1.0 / var))
    res = _runs(t, n_particles=512, n_iters=12, n_warmup=6, step_size=0.1, traj_len0=2.0,
                init_scale=1.5)
    log_z_true = 0.5 * 3 * np.log(2 * np.pi) + 0.5 * np.log(var).sum()
    assert _within_3_mcse([r[0] for r in res], log_z_true)
    assert np.all(_within_3_mcse([r[1] for r in res], mu))
    assert np.all(_within_3_mcse([r[2] for r in res], var))


def test_linear_gaussian_evidence():
    lin = workloads.linear_gauss(n=5, D=3, sigma=1.0, tau=1.0)
    t = oracle.TargetSpec.linear_gauss(lin["X"], lin["y"], 1.0, 1.0)
    res = _runs(t, n_particles=1024, n_iters=8, n_warmup=4, step_size=0.1, traj_len0=1.0,
                init_scale=1.0)
    X, y = lin["X"], lin["y"]
    truth = stats.multivariate_normal(np.zeros(5), np.eye(5) + X @ X.T).logpdf(y)
    assert _within_3_mcse([r[0] for r in res], truth)
    A = X.T @ X + np.eye(3)
    post_mean = np.linalg.solve(A, X.T @ y)
    post_var = np.diag(np.linalg.inv(A))
    assert np.all(_within_3_mcse([r[1] for r in res], post_mean))
    assert np.all(_within_3_mcse([r[2] for r in res], post_var))


def test_bookkeeping_invariants():
    g = workloads.gauss10()
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    cfg = oracle.SMCConfig(n_particles=64, n_iters=6, n_warmup=3, step_size=0.1,
                           traj_len0=0.75, jitter=0, adapt=0, init_scale=2.0, seed=5)
    st = oracle.smc_init(t, cfg)
    st["chees"] = oracle.initial_chees_state(cfg)
    lz = st["log_z"]
    for k in range(1, 7):
        pre_w = st["logw"].copy()
        out = oracle.smc_iteration(t, cfg, k, st)
        s = out["stats"]
        assert np.all(out["steps"] == 8)                      # ceil(0.75 / 0.1)
        assert s["grad_evals"] == 64 * 8
        _, ess_pre, _ = oracle.normalise(pre_w)
        assert s["resampled"] == int(ess_pre < 32)
        assert abs(s["ess_pre"] - ess_pre) < 1e-9 * ess_pre
        if not s["resampled"]:
            assert np.all(out["ancestors"] == np.arange(64))
            np.testing.assert_allclose(st["logw"], pre_w - out["dH"])
        lz += s["log_z_inc"]
        assert abs(st["log_z"] - lz) < 1e-12
        np.testing.assert_allclose(out["alpha"], np.minimum(1.0, np.exp(-out["dH"])))
    # momentum comes from the (seed, MOM, k, j) stream
    np.testing.assert_array_equal(out["p0"][3], oracle.normals(5, oracle.TAG_MOM, 6, 3, 10))


def test_accept_reject_variant_keeps_weights():
    g = workloads.gauss10()
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    cfg = oracle.SMCConfig(n_particles=128, n_iters=4, n_warmup=2, step_size=0.3,
                           traj_len0=2.0, accept_reject=1, init_scale=0.3, seed=9)
    r = oracle.smc_run(t, cfg)
    assert r["status"] == 0
    assert all(s["log_z_inc"] == 0.0 for s in r["stats"])


def test_degenerate_target_reports_status():
    t = oracle.TargetSpec.gauss_dense(np.zeros(2), np.eye(2), c=float("nan"))
    r = oracle.smc_run(t, oracle.SMCConfig(n_particles=16, n_iters=3, n_warmup=1))
    assert r["status"] == -4


def test_table1_shape_gaussian_1d_halton():
    """Sec. 4 'Gaussian' with 1-d Halton: the paper prints 8.01 gradient
    evaluations per particle and J_eff per evaluation 0.125 (Table 1).  The
    Adam constants are not given by the paper; over Adam rates 0.025 to 0.25,
    both readings of the J x K Halton index order, Adam descent and the
    printed initial momentum in the ChEES estimate, none brings the adapted
    trajectory down to the paper's (this oracle gives about 19 gradients per
    particle at the default rate 0.025), so the check only bounds the ratio
    (statistical; parity unpinned for the constants)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1_1d_halton.json")) as f:
        gold = json.load(f)
    ge_paper = gold["grad_evals_per_particle"]["gaussian_5d"]
    ej_paper = gold["ess_per_grad_eval"]["gaussian_5d"]
    g = workloads.paper_gauss5()
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    ge, ej = [], []
    for s in workloads.RUN_SEEDS[:3]:
        r = oracle.smc_run(t, oracle.SMCConfig(seed=s, **g["run"]))
        ge.append(np.mean([x["grad_evals"] / 1000 + 1 for x in r["stats"]]))
        ej.append(np.mean([x["ess"] / (x["grad_evals"] + 1000) for x in r["stats"]]))
    assert ge_paper / 3 < np.mean(ge) < ge_paper * 3
    assert ej_paper / 3 < np.mean(ej) < ej_paper * 3


def test_multinomial_scheme_moments_evidence_and_draws():
    """resample_scheme = 1 (multinomial, the paper's choice): the same closed
    forms within 3 MCSE; the per-output uniforms are the Philox blocks
    (1, i, k, RESAMPLE) -- uniform by a chi-square test on their top bits and
    distinct from the systematic draw (0, 0, k, RESAMPLE); with the sampler's
    resampled ancestors matching the stand-alone multinomial rule on those
    uniforms."""
    mu = np.array([0.5, -0.3, 0.2])
    var = np.array([0.5, 1.0, 2.0])
    t = oracle.TargetSpec.gauss_dense(mu, np.diag(1.0 / var))
    kw = dict(n_particles=512, n_iters=12, n_warmup=6, step_size=0.1, traj_len0=2.0, init_scale=1.5,
              resample_scheme=1)
    res = _runs(t, **kw)
    log_z_true = 0.5 * 3 * np.log(2 * np.pi) + 0.5 * np.log(var).sum()
    assert _within_3_mcse([r[0] for r in res], log_z_true)
    assert np.all(_within_3_mcse([r[1] for r in res], mu))
    assert np.all(_within_3_mcse([r[2] for r in res], var))
    assert any(s["resampled"] for r in res for s in r[3])
    # the uniforms
    u = np.array([oracle.multinomial_u64(77, 3, i) for i in range(20000)], dtype=np.uint64)
    top = (u >> np.uint64(60)).astype(np.int64)
    _, p = stats.chisquare(np.bincount(top, minlength=16))
    assert p > 1e-4
    assert oracle.resample_r64(77, 3) not in set(u.tolist())
    # one resampling iteration of the sampler against the stand-alone rule
    cfg = oracle.SMCConfig(seed=91, **dict(kw, n_iters=3, init_scale=3.0))
    st = oracle.smc_init(t, cfg)
    st["chees"] = oracle.initial_chees_state(cfg)
    lw = st["logw"].copy()
    out = oracle.smc_iteration(t, cfg, 1, st)
    assert out["stats"]["resampled"] == 1
    _, _, W = oracle.normalise(lw)
    _, q = oracle.quantise(W)
    uu = np.array([oracle.multinomial_u64(91, 1, i) for i in range(cfg.n_particles)], dtype=np.uint64)
    np.testing.assert_array_equal(out["ancestors"], oracle.multinomial(q, uu))


def test_mcmc_mode_chains_reach_the_target():
    """mcmc = 1 (Algorithm 2 as J independent chains): no weights (ESS = J
    every iteration, nothing resampled, log Z = 0), and started far off
    (q_init = N(0, 3^2 I)) the chains' ensemble mean and variance after
    warm-up match the conjugate Gaussian's within 4 standard errors."""
    mu = np.array([0.5, -0.3, 0.2])
    var = np.array([0.5, 1.0, 2.0])
    t = oracle.TargetSpec.gauss_dense(mu, np.diag(1.0 / var))
    J = 2048
    cfg = oracle.SMCConfig(n_particles=J, n_iters=30, n_warmup=15, step_size=0.2, traj_len0=1.5,
                           init_scale=3.0, seed=5, mcmc=1)
    r = oracle.smc_run(t, cfg)
    assert r["status"] == 0
    assert r["log_z"] == 0.0
    assert all(s["resampled"] == 0 and abs(s["ess"] - J) <= 1e-9 * J and s["log_z_inc"] == 0.0 for s in r["stats"])
    th = r["theta"]
    se_m = np.sqrt(var / J)
    assert np.all(np.abs(th.mean(0) - mu) <= 4 * se_m)
    se_v = var * np.sqrt(2.0 / (J - 1))
    assert np.all(np.abs(th.var(0, ddof=1) - var) <= 4 * se_v)
    # without the Metropolis select (mcmc off, SMC weights) the same seed gives a
    # different, weighted ensemble
    r2 = oracle.smc_run(t, oracle.SMCConfig(**{**cfg.__dict__, "mcmc": 0}))
    assert r2["log_z"] != 0.0


def test_accept_reject_keeps_the_target_invariant():
    """The Metropolis select (accept_reject = 1) makes each move leave the
    target invariant: started exactly at N(0, I) (q_init = the target, so the
    initial weights are uniform) with a step size large enough that many
    proposals are rejected, the ensemble stays N(0, I): mean within 4 SE and
    variance within 4 SE after every iteration."""
    D, J = 3, 4096
    t = oracle.TargetSpec.gauss_dense(np.zeros(D), np.eye(D))
    cfg = oracle.SMCConfig(n_particles=J, n_iters=8, n_warmup=0, step_size=1.5, traj_len0=4.0, max_steps=50,
                           init_scale=1.0, seed=17, accept_reject=1, adapt=0, jitter=1, ess_frac=0.0)
    st = oracle.smc_init(t, cfg)
    st["chees"] = oracle.initial_chees_state(cfg)
    rejected = 0
    for k in range(1, cfg.n_iters + 1):
        out = oracle.smc_iteration(t, cfg, k, st)
        assert out["status"] == 0
        rejected += int(np.sum(out["alpha"] < 0.5))
        th = st["theta"]
        assert np.all(np.abs(th.mean(0)) <= 4 * np.sqrt(1.0 / J)), (k, th.mean(0))
        assert np.all(np.abs(th.var(0, ddof=1) - 1.0) <= 4 * np.sqrt(2.0 / (J - 1))), (k, th.var(0, ddof=1))
    assert rejected > J      # the step size really does reject proposals
