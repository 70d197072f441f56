"""Pins for the oracle's ChEES adaptation (Sec. 2.3, Algorithm 2).

The per-particle estimate g_c = l (|t1_c - mean t1|^2 - |t0_c - mean t0|^2)
(t1_c - mean t1)' p_c is the derivative, in log trajectory time, of the sample
criterion 1/4 mean_c (|t1_c - mean t1|^2 - |t0_c - mean t0|^2)^2 -- exactly so
when the population mean of the final momenta is zero.  Pinned by a central
finite difference in log t along the exact Hamiltonian flow of a standard
normal target (theta(t) = theta0 cos t + p sin t), which needs no integrator:
* a symmetric population (pairs +x, -x) has zero mean momentum: the oracle's
  mean estimate equals the finite difference;
* a general population: it equals the finite difference plus the term
  t mean_c Delta_c (t1_c - mean t1)' mean(p) that the estimate leaves out;
* the initial-momentum reading fails the same check.
Adam is pinned by its closed forms: a constant gradient g gives bias-corrected
moments exactly g and g^2, so each step moves log L by lr g / (|g| + eps_A).
"""
import numpy as np

import oracle


def _flow(th0, p0, t):
    return th0 * np.cos(t) + p0 * np.sin(t), -th0 * np.sin(t) + p0 * np.cos(t)


def _criterion(th0, th1):
    d0 = np.sum((th0 - th0.mean(0)) ** 2, axis=1)
    d1 = np.sum((th1 - th1.mean(0)) ** 2, axis=1)
    return 0.25 * np.mean((d1 - d0) ** 2)


def _fd_log_t(th0, p0, t, h=1e-5):
    up = _criterion(th0, _flow(th0, p0, t * np.exp(h))[0])
    dn = _criterion(th0, _flow(th0, p0, t * np.exp(-h))[0])
    return (up - dn) / (2 * h)


def test_chees_gradient_symmetric_population_equals_fd():
    rng = np.random.default_rng(0)
    half_t, half_p = rng.standard_normal((4, 2)), rng.standard_normal((4, 2))
    th0 = np.concatenate([half_t, -half_t])
    p0 = np.concatenate([half_p, -half_p])
    for t in (0.3, 0.9, 1.7):
        th1, p1 = _flow(th0, p0, t)
        ghat, _ = oracle.chees_gradient(th0, th1, p1, np.full(8, t), np.ones(8))
        fd = _fd_log_t(th0, p0, t)
        assert abs(ghat - fd) < 1e-7 * max(1.0, abs(fd)), (t, ghat, fd)


def test_chees_gradient_general_population_matches_fd_plus_mean_momentum_term():
    rng = np.random.default_rng(1)
    th0 = rng.standard_normal((8, 2)) + 0.5
    p0 = rng.standard_normal((8, 2))
    t = 0.8
    th1, p1 = _flow(th0, p0, t)
    ghat, _ = oracle.chees_gradient(th0, th1, p1, np.full(8, t), np.ones(8))
    d0 = np.sum((th0 - th0.mean(0)) ** 2, axis=1)
    d1 = np.sum((th1 - th1.mean(0)) ** 2, axis=1)
    missing = t * np.mean((d1 - d0) * ((th1 - th1.mean(0)) @ p1.mean(0)))
    fd = _fd_log_t(th0, p0, t)
    assert abs(ghat - (fd + missing)) < 1e-7 * max(1.0, abs(fd))
    # reading check: the initial momentum does not give the derivative
    g_init, _ = oracle.chees_gradient(th0, th1, p0, np.full(8, t), np.ones(8))
    assert abs(g_init - (fd + missing)) > 1e-3


def test_chees_gradient_acceptance_weighting_and_degenerate():
    rng = np.random.default_rng(2)
    th0, th1, p = (rng.standard_normal((6, 3)) for _ in range(3))
    l = rng.uniform(0.1, 1.0, 6)
    a = np.array([1.0, 0.0, 0.5, 0.25, 1.0, 0.0])
    ghat, per = oracle.chees_gradient(th0, th1, p, l, a)
    assert abs(ghat - np.sum(a * per) / a.sum()) < 1e-12
    # no accepted mass -> no update
    g0, _ = oracle.chees_gradient(th0, th1, p, l, np.zeros(6))
    assert g0 is None


def test_adam_constant_gradient_closed_form():
    for g in (3.0, -0.2):
        st = oracle.CheesState(np.log(1.0), 0.0, 0.0, 0, 0.0)
        logs = []
        for _ in range(5):
            oracle.chees_adam(st, g, 0.025, 0.9, 0.999, 1e-8, 0.01, 10**6)
            logs.append(st.log_L)
        step = 0.025 * g / (abs(g) + 1e-8)
        np.testing.assert_allclose(np.diff([0.0] + logs), step, rtol=1e-12)
        assert st.t == 5


def test_adam_clamps_to_step_range():
    st = oracle.CheesState(np.log(0.02), 0.0, 0.0, 0, 0.0)
    for _ in range(10):
        oracle.chees_adam(st, -1.0, 0.5, 0.9, 0.999, 1e-8, 0.01, 100)
    assert st.log_L == np.log(0.01)
    for _ in range(40):
        oracle.chees_adam(st, 1.0, 0.5, 0.9, 0.999, 1e-8, 0.01, 100)
    assert st.log_L == np.log(100 * 0.01)
