"""Pins for the oracle's general Gaussian initial distribution q_init = N(m, L L^T).

The paper leaves the initial distribution to the user (its experiments draw
theta_0 from N(0, I), Sec. 4) and weights the first population by
w_1 = pi(theta_0) / q_init(theta_0) (Algorithm 3).  The pins:
* with q_init equal to a Gaussian target up to its normaliser, every initial
  log-weight equals the target's closed-form log normaliser -- a transposed
  L, a dropped mean or a wrong sign of the log-determinant makes the weights
  vary or shifts them;
* L = s I given explicitly, or only a mean given, reproduces the isotropic
  draw (the same standard normals, shifted);
* the upper triangle of L is never read;
* the sample mean and covariance of theta_0 match m and L L^T;
* the whole sampler started from a Gaussian q_init still estimates the
  closed-form evidence and moments of a conjugate Gaussian within 3 MCSE.
"""
import numpy as np

import oracle


def _spd(D, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((D, D))
    return A @ A.T / D + 0.3 * np.eye(D)


def _target(D=6, seed=3, c=0.7):
    rng = np.random.default_rng(seed + 1)
    mu = rng.standard_normal(D)
    P = _spd(D, seed)
    return mu, P, oracle.TargetSpec.gauss_dense(mu, P, c=c), c


def test_initial_weights_are_the_log_normaliser_when_q_init_is_the_target():
    D = 6
    mu, P, t, c = _target(D)
    Sigma = np.linalg.inv(P)
    L = np.linalg.cholesky(Sigma)
    cfg = oracle.SMCConfig(n_particles=512, seed=11, init_mean=mu, init_chol=L)
    st = oracle.smc_init(t, cfg)
    log_norm = c + 0.5 * D * np.log(2 * np.pi) - 0.5 * np.linalg.slogdet(P)[1]
    np.testing.assert_allclose(st["logw"], log_norm, rtol=0, atol=1e-10)
    assert abs(st["log_z"] - log_norm) < 1e-10
    # the transposed factor gives the wrong covariance: the weights then vary
    st_t = oracle.smc_init(t, oracle.SMCConfig(n_particles=512, seed=11, init_mean=mu, init_chol=np.tril(L.T)))
    assert np.std(st_t["logw"]) > 1e-3


def test_explicit_isotropic_factor_and_mean_only_reproduce_the_isotropic_draw():
    D, s = 5, 0.7
    _, _, t, _ = _target(D, seed=5)
    base = oracle.smc_init(t, oracle.SMCConfig(n_particles=300, seed=4, init_scale=s))
    expl = oracle.smc_init(t, oracle.SMCConfig(n_particles=300, seed=4, init_chol=s * np.eye(D)))
    np.testing.assert_array_equal(expl["theta"], base["theta"])
    np.testing.assert_allclose(expl["logw"], base["logw"], rtol=0, atol=1e-12)
    m = np.linspace(-1.0, 2.0, D)
    shift = oracle.smc_init(t, oracle.SMCConfig(n_particles=300, seed=4, init_scale=s, init_mean=m))
    np.testing.assert_array_equal(shift["theta"], base["theta"] + m)
    # log q is that of the isotropic draw at the unshifted point: only log pi changes
    lq_base = base["logpi"] - base["logw"]
    lq_shift = shift["logpi"] - shift["logw"]
    np.testing.assert_allclose(lq_shift, lq_base, rtol=0, atol=1e-9)


def test_upper_triangle_is_not_read():
    D = 6
    mu, P, t, _ = _target(D, seed=8)
    L = np.linalg.cholesky(np.linalg.inv(P))
    junk = L + np.triu(np.full((D, D), 37.0), 1)
    a = oracle.smc_init(t, oracle.SMCConfig(n_particles=64, seed=2, init_mean=mu, init_chol=L))
    b = oracle.smc_init(t, oracle.SMCConfig(n_particles=64, seed=2, init_mean=mu, init_chol=junk))
    np.testing.assert_array_equal(a["theta"], b["theta"])
    np.testing.assert_array_equal(a["logw"], b["logw"])


def test_initial_draw_has_the_requested_mean_and_covariance():
    D, N = 4, 40000
    rng = np.random.default_rng(9)
    m = rng.standard_normal(D)
    L = np.linalg.cholesky(_spd(D, 12))
    t = oracle.TargetSpec.gauss_dense(np.zeros(D), np.eye(D))
    th = oracle.smc_init(t, oracle.SMCConfig(n_particles=N, seed=77, init_mean=m, init_chol=L))["theta"]
    S = L @ L.T
    se_mean = np.sqrt(np.diag(S) / N)
    assert np.all(np.abs(th.mean(0) - m) < 4 * se_mean)
    C = np.cov(th.T)
    # SE of a sample covariance entry: sqrt((S_ii S_jj + S_ij^2) / N)
    se_cov = np.sqrt((np.outer(np.diag(S), np.diag(S)) + S**2) / N)
    assert np.all(np.abs(C - S) < 4 * se_cov)


def test_sampler_from_a_gaussian_q_init_keeps_the_closed_form_evidence():
    D = 3
    mu = np.array([0.5, -0.3, 0.2])
    var = np.array([0.5, 1.0, 2.0])
    t = oracle.TargetSpec.gauss_dense(mu, np.diag(1.0 / var))
    log_z_true = 0.5 * D * np.log(2 * np.pi) + 0.5 * np.log(var).sum()
    L = np.diag([1.2, 0.5, 2.0])          # a Gaussian q_init unlike the target
    m = np.array([1.0, 0.0, -1.0])
    lz, means = [], []
    for s in range(30):
        r = oracle.smc_run(t, oracle.SMCConfig(n_particles=512, n_iters=8, n_warmup=4, step_size=0.2,
                                               traj_len0=1.5, seed=700 + s, init_mean=m, init_chol=L))
        assert r["status"] == 0
        lz.append(r["log_z"])
        W = np.exp(r["logw"] - r["logw"].max())
        means.append((W / W.sum()) @ r["theta"])
    lz, means = np.asarray(lz), np.asarray(means)
    assert abs(lz.mean() - log_z_true) < 3 * lz.std(ddof=1) / np.sqrt(len(lz))
    assert np.all(np.abs(means.mean(0) - mu) < 3 * means.std(0, ddof=1) / np.sqrt(len(lz)) + 1e-3)
