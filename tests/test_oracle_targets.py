"""Pins for the oracle's log-targets (Sec. 2 and Sec. 4).

* gradients against central finite differences of log pi;
* the hierarchical model's sufficient-statistic form against the raw-data
  likelihood written with scipy.stats;
* normalising constants: the banana integrates to one (2-d quadrature), the
  linear-Gaussian evidence equals the marginal N(y; 0, s^2 I + t^2 X X') from
  scipy, the logistic log-likelihood at theta = 0 is -n log 2 plus the prior.
"""
import numpy as np
import pytest
from scipy import integrate, stats

import oracle
import workloads


def _fd_grad(t, theta, h=1e-6):
    g = np.empty_like(theta)
    for d in range(theta.size):
        e = np.zeros_like(theta)
        e[d] = h
        lp_p, _ = oracle.logpi(t, theta + e)
        lp_m, _ = oracle.logpi(t, theta - e)
        g[d] = (lp_p[0] - lp_m[0]) / (2 * h)
    return g


def _targets():
    g10 = workloads.gauss10()
    lg = workloads.logistic(n=60, d_features=4)
    lin = workloads.linear_gauss(n=40, D=5)
    hi = workloads.hier(groups=6, obs=5)
    return {
        "gauss": oracle.TargetSpec.gauss_dense(g10["mu"] + 0.3, g10["P"], c=1.7),
        "logistic": oracle.TargetSpec.logistic(lg["X"], lg["y"], tau=1.5),
        "linear": oracle.TargetSpec.linear_gauss(lin["X"], lin["y"], 0.5, 2.0),
        "hier": oracle.TargetSpec.hier_normal(hi["ybar"], hi["n_g"], hi["ss"], 1.3),
        "banana": oracle.TargetSpec.banana(6, 10.0, 0.1),
    }


@pytest.mark.parametrize("name", ["gauss", "logistic", "linear", "hier", "banana"])
def test_gradient_matches_finite_differences(name):
    t = _targets()[name]
    rng = np.random.default_rng(11)
    for _ in range(3):
        th = rng.standard_normal(t.D) * 0.7
        _, g = oracle.logpi(t, th)
        fd = _fd_grad(t, th)
        np.testing.assert_allclose(g[0], fd, rtol=1e-6, atol=1e-6)


def test_hier_matches_raw_data_likelihood():
    hi = workloads.hier(groups=7, obs=5)
    t = oracle.TargetSpec.hier_normal(hi["ybar"], hi["n_g"], hi["ss"], hi["sigma"])
    rng = np.random.default_rng(5)
    for _ in range(3):
        th = rng.standard_normal(t.D)
        mu, logtau, eta = th[0], th[1], th[2:]
        b = mu + np.exp(logtau) * eta
        direct = (stats.norm.logpdf(hi["y_raw"], loc=b[:, None], scale=hi["sigma"]).sum()
                  + stats.norm.logpdf(mu) + stats.norm.logpdf(logtau)
                  + stats.norm.logpdf(eta).sum())
        lp, _ = oracle.logpi(t, th)
        assert abs(lp[0] - direct) < 1e-9 * max(1.0, abs(direct))


def test_banana_is_normalised():
    t = oracle.TargetSpec.banana(2, 100.0, 0.03)
    f = lambda x2, x1: np.exp(oracle.logpi(t, np.array([x1, x2]))[0][0])
    # x2 centred at 0.03 (x1^2 - 100); integrate a +-10 sd window around it.
    val, _ = integrate.dblquad(f, -80.0, 80.0, lambda x1: 0.03 * (x1 * x1 - 100) - 10,
                               lambda x1: 0.03 * (x1 * x1 - 100) + 10, epsabs=1e-10)
    assert abs(val - 1.0) < 1e-6


def test_linear_gauss_evidence_closed_form():
    lin = workloads.linear_gauss(n=30, D=4, sigma=0.7, tau=1.3)
    t = oracle.TargetSpec.linear_gauss(lin["X"], lin["y"], 0.7, 1.3)
    X, y = lin["X"], lin["y"]
    # posterior precision A and mode m; Gaussian integral of exp(log pi)
    A = X.T @ X / 0.7**2 + np.eye(4) / 1.3**2
    m = np.linalg.solve(A, X.T @ y / 0.7**2)
    lp_m, g = oracle.logpi(t, m)
    assert np.max(np.abs(g)) < 1e-9
    logZ = lp_m[0] + 0.5 * 4 * np.log(2 * np.pi) - 0.5 * np.linalg.slogdet(A)[1]
    marg = stats.multivariate_normal(np.zeros(30), 0.7**2 * np.eye(30) + 1.3**2 * X @ X.T)
    assert abs(logZ - marg.logpdf(y)) < 1e-8


def test_logistic_at_origin():
    lg = workloads.logistic(n=50, d_features=3)
    t = oracle.TargetSpec.logistic(lg["X"], lg["y"], tau=1.0)
    lp, g = oracle.logpi(t, np.zeros(4))
    expect = -50 * np.log(2.0) + stats.norm.logpdf(np.zeros(4)).sum()
    assert abs(lp[0] - expect) < 1e-10
    np.testing.assert_allclose(g[0], lg["X"].T @ (lg["y"] - 0.5), rtol=1e-12)


def test_gauss_dense_value():
    g10 = workloads.gauss10()
    t = oracle.TargetSpec.gauss_dense(g10["mu"], g10["P"], c=0.25)
    lp, g = oracle.logpi(t, g10["mu"])
    assert lp[0] == 0.25 and np.all(g[0] == 0.0)
    x = np.arange(10) * 0.1
    lp, _ = oracle.logpi(t, x)
    assert abs(lp[0] - (0.25 + stats.multivariate_normal(np.zeros(10), g10["Sigma"]).logpdf(x)
                        + 0.5 * 10 * np.log(2 * np.pi) + 0.5 * np.log(g10["eigvals"]).sum())) < 1e-8
