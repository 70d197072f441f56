"""Pins for the oracle's leapfrog integrator (Sec. 2.1, Algorithm 1).

* reversibility: integrate S steps, negate p, integrate S steps -> start;
* energy error of a fixed-time trajectory scales as eps^2 (second order);
* on a Gaussian target the leapfrog map is linear: in each eigendirection of
  the precision (frequency w) one step is the 2x2 matrix
  [[1 - e^2 w^2/2, e], [-e w^2 (1 - e^2 w^2/4), 1 - e^2 w^2/2]] acting on (q, p),
  so S steps are its S-th matrix power.
"""
import numpy as np
import pytest

import oracle
import workloads


def _logistic_small():
    lg = workloads.logistic(n=80, d_features=5)
    return oracle.TargetSpec.logistic(lg["X"], lg["y"])


@pytest.mark.parametrize("which", ["logistic", "banana", "hier"])
def test_leapfrog_reversible(which):
    if which == "logistic":
        t = _logistic_small()
    elif which == "banana":
        t = oracle.TargetSpec.banana(4, 10.0, 0.1)
    else:
        h = workloads.hier(groups=5, obs=4)
        t = oracle.TargetSpec.hier_normal(h["ybar"], h["n_g"], h["ss"])
    rng = np.random.default_rng(1)
    th0 = rng.standard_normal((4, t.D)) * 0.3
    p0 = rng.standard_normal((4, t.D))
    th1, p1, _, _ = oracle.leapfrog(t, th0, p0, 0.01, 37)
    th2, p2, _, _ = oracle.leapfrog(t, th1, -p1, 0.01, 37)
    np.testing.assert_allclose(th2, th0, atol=1e-11)
    np.testing.assert_allclose(-p2, p0, atol=1e-10)


def test_energy_error_is_second_order():
    t = _logistic_small()
    rng = np.random.default_rng(2)
    th0 = rng.standard_normal((8, t.D)) * 0.2
    p0 = rng.standard_normal((8, t.D))
    lp0, _ = oracle.logpi(t, th0)
    errs = []
    for eps in (0.02, 0.01, 0.005):
        steps = int(round(0.4 / eps))
        _, p1, _, lp1 = oracle.leapfrog(t, th0, p0, eps, steps)
        dH = [oracle.hamiltonian(p1[j], lp1[j]) - oracle.hamiltonian(p0[j], lp0[j])
              for j in range(8)]
        errs.append(np.sqrt(np.mean(np.square(dH))))
    slope = np.polyfit(np.log([0.02, 0.01, 0.005]), np.log(errs), 1)[0]
    assert abs(slope - 2.0) < 0.15, (errs, slope)


def test_leapfrog_on_gaussian_is_matrix_power():
    g = workloads.gauss10()
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    lam = g["eigvals"]                       # covariance eigenvalues
    Q = workloads.haar_orthogonal(10)        # same eigenvectors as P
    rng = np.random.default_rng(4)
    th0 = rng.standard_normal(10)
    p0 = rng.standard_normal(10)
    eps, S = 0.05, 23
    th1, p1, _, _ = oracle.leapfrog(t, th0, p0, eps, S)
    q0, r0 = Q.T @ th0, Q.T @ p0
    q1, r1 = np.empty(10), np.empty(10)
    for i in range(10):
        w2 = 1.0 / lam[i]
        a = 1.0 - 0.5 * eps**2 * w2
        M = np.array([[a, eps], [-eps * w2 * (1.0 - 0.25 * eps**2 * w2), a]])
        q1[i], r1[i] = np.linalg.matrix_power(M, S) @ np.array([q0[i], r0[i]])
    np.testing.assert_allclose(th1[0], Q @ q1, atol=1e-10)
    np.testing.assert_allclose(p1[0], Q @ r1, atol=1e-10)
