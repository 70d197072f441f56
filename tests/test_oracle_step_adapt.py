"""Pins for the oracle's optional step-size rule (not in the paper, which
fixes epsilon per experiment and leaves its adaptation to future work,
Sec. 5): during warm-up, after the ChEES update, log eps moves by
rate * (a_h - target) with a_h the harmonic mean of the acceptance
probabilities and target 0.651.

* the harmonic mean agrees with scipy's, and is 0 when some alpha is 0;
* the update agrees with scipy's harmonic mean put through the rule, and
  all-accepting particles give the closed form eps exp(rate (1 - target));
* rate 0 reproduces the fixed-step sampler exactly;
* a step that is too large shrinks and one that is too small grows, and
  after warm-up the harmonic-mean acceptance sits near the target, on a
  5-d Gaussian whose stable leapfrog range is known (eps < 2 for unit
  variances);
* epsilon is frozen from M_warmup on.
"""
import ctypes as C

import numpy as np
import pytest

import oracle

scipy_stats = pytest.importorskip("scipy.stats")


def test_harmonic_mean_matches_scipy_and_zero_case():
    rng = np.random.default_rng(3)
    a = rng.uniform(0.05, 1.0, 257)
    assert abs(oracle.harmonic_mean_alpha(a) - scipy_stats.hmean(a)) <= 1e-14
    a[17] = 0.0
    assert oracle.harmonic_mean_alpha(a) == 0.0


def test_update_against_scipy_and_closed_form():
    rng = np.random.default_rng(4)
    a = rng.uniform(0.2, 1.0, 100)
    e1 = oracle.step_size_update(0.3, a, 0.7, 0.651)
    assert abs(np.log(e1 / 0.3) - 0.7 * (scipy_stats.hmean(a) - 0.651)) <= 1e-13
    e2 = oracle.step_size_update(0.25, np.ones(64), 0.5, 0.651)
    assert abs(e2 - 0.25 * np.exp(0.5 * 0.349)) <= 1e-15


def _gauss5():
    return oracle.TargetSpec.gauss_dense(np.zeros(5), np.eye(5))


def _run_steps(cfg, K):
    t = _gauss5()
    st = oracle.smc_init(t, cfg)
    st["chees"] = oracle.initial_chees_state(cfg)
    st["eps"] = C.c_double(cfg.step_size)
    eps, ah = [], []
    for k in range(1, K + 1):
        out = oracle.smc_iteration(t, cfg, k, st)
        assert out["status"] == 0
        ah.append(oracle.harmonic_mean_alpha(out["alpha"]))
        eps.append(st["eps"].value)
    return np.array(eps), np.array(ah), st


def test_rate_zero_reproduces_fixed_step():
    base = dict(n_particles=128, n_iters=6, n_warmup=4, step_size=0.4, traj_len0=1.0, seed=11)
    a = oracle.smc_run(_gauss5(), oracle.SMCConfig(**base))
    b = oracle.smc_run(_gauss5(), oracle.SMCConfig(**base, step_adapt_rate=0.0))
    assert a["log_z"] == b["log_z"]
    np.testing.assert_array_equal(a["theta"], b["theta"])
    # a positive rate changes the run
    c = oracle.smc_run(_gauss5(), oracle.SMCConfig(**base, step_adapt_rate=0.5))
    assert c["log_z"] != a["log_z"]


@pytest.mark.parametrize("eps0,direction", [(1.9, -1), (0.02, +1)])
def test_adaptation_moves_toward_target_and_freezes(eps0, direction):
    K, M = 40, 30
    cfg = oracle.SMCConfig(n_particles=256, n_iters=K, n_warmup=M, step_size=eps0, traj_len0=1.0,
                           max_steps=200, seed=21, step_adapt_rate=0.5)
    eps, ah, _ = _run_steps(cfg, K)
    assert direction * (eps[M - 2] - eps0) > 0
    # near the target once adapted (a loose band: a_h is a noisy statistic)
    assert abs(np.median(ah[M - 8:M]) - 0.651) < 0.12, ah[M - 8:M]
    # the last update is at iteration M_warmup - 1; frozen from M_warmup on
    assert eps[M - 2] != eps[M - 3]
    assert np.all(eps[M - 2:] == eps[M - 2])
    assert 0.1 < eps[M - 2] < 2.0
