"""Pins for the oracle's affine-coupling transport map (learned preconditioner).

* the zero last layer gives the identity map, and then the preconditioned
  sampler is bit-identical to the plain one;
* T(T^-1(x)) = x and the inverse log-determinant is minus the forward one;
* log|det dT/dz| against the log-determinant of a central-difference Jacobian;
* the latent-space gradient of log pi(T(z)) + log|det dT/dz| against central
  finite differences;
* the training-loss gradient (weighted NLL under the flow density) against
  central finite differences, for parameters of every block of every layer;
* training on an ill-conditioned Gaussian raises the HMC acceptance at a fixed
  step size (what the learned map buys).
"""
import numpy as np
import pytest

import oracle
import workloads

D, H, L = 4, 8, 4


def _random_flow(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    p = workloads.flow_init(D, H, L, seed=seed)
    p = p + scale * rng.standard_normal(p.size)        # non-trivial last layers too
    return oracle.FlowSpec(D, H, L, p)


def test_zero_last_layer_is_identity():
    f = oracle.FlowSpec(D, H, L, workloads.flow_init(D, H, L))
    z = np.random.default_rng(1).standard_normal((5, D))
    x, ld = oracle.flow_forward(f, z)
    np.testing.assert_array_equal(x, z)
    assert np.all(ld == 0.0)


def test_inverse_round_trip_and_logdet_sign():
    f = _random_flow()
    x = np.random.default_rng(2).standard_normal((6, D)) * 1.5
    z, ldi = oracle.flow_inverse(f, x)
    x2, ld = oracle.flow_forward(f, z)
    np.testing.assert_allclose(x2, x, atol=1e-12)
    np.testing.assert_allclose(ld, -ldi, atol=1e-12)


def test_logdet_matches_finite_difference_jacobian():
    f = _random_flow(3)
    z0 = np.random.default_rng(4).standard_normal(D)
    _, ld = oracle.flow_forward(f, z0)
    J = np.empty((D, D))
    h = 1e-6
    for k in range(D):
        e = np.zeros(D)
        e[k] = h
        xp, _ = oracle.flow_forward(f, z0 + e)
        xm, _ = oracle.flow_forward(f, z0 - e)
        J[:, k] = (xp[0] - xm[0]) / (2 * h)
    assert abs(np.linalg.slogdet(J)[1] - ld[0]) < 1e-7


@pytest.mark.parametrize("target", ["banana", "gauss"])
def test_latent_gradient_matches_finite_differences(target):
    f = _random_flow(5)
    if target == "banana":
        t = oracle.TargetSpec.banana(D, 10.0, 0.1)
    else:
        g = workloads._gauss_from_spectrum(np.array([0.1, 0.5, 1.0, 3.0]), 7)
        t = oracle.TargetSpec.gauss_dense(g["mu"] + 0.2, g["P"])
    z0 = np.random.default_rng(6).standard_normal(D) * 0.5
    lpz, gz, _, _, _ = oracle.flow_logpi_z(f, t, z0)
    fd = np.empty(D)
    h = 1e-6
    for k in range(D):
        e = np.zeros(D)
        e[k] = h
        fd[k] = (oracle.flow_logpi_z(f, t, z0 + e)[0][0] - oracle.flow_logpi_z(f, t, z0 - e)[0][0]) / (2 * h)
    np.testing.assert_allclose(gz[0], fd, rtol=1e-6, atol=1e-6)


def test_training_loss_gradient_matches_finite_differences():
    f = _random_flow(8, scale=0.2)
    rng = np.random.default_rng(9)
    th = rng.standard_normal((7, D))
    W = rng.uniform(0.1, 1.0, 7)
    W /= W.sum()
    loss, grad = oracle.flow_loss_grad(f, th, W)
    Dh = D // 2
    lsz = H * Dh + H + H * H + H + D * H + D
    offs = [0, H * Dh, H * Dh + H, H * Dh + H + H * H, H * Dh + 2 * H + H * H, lsz - D]   # one per block
    idx = [l * lsz + o + 1 for l in range(L) for o in offs]
    h = 1e-6
    for i in idx:
        p0 = f.params[i]
        f.params[i] = p0 + h
        lp, _ = oracle.flow_loss_grad(f, th, W)
        f.params[i] = p0 - h
        lm, _ = oracle.flow_loss_grad(f, th, W)
        f.params[i] = p0
        fd = (lp - lm) / (2 * h)
        assert abs(grad[i] - fd) < 1e-6 * max(1.0, abs(fd)), (i, grad[i], fd)


def test_zero_flow_without_training_equals_plain_sampler_bit_for_bit():
    g = workloads.gauss10()
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    cfg = oracle.SMCConfig(n_particles=64, n_iters=5, n_warmup=3, step_size=0.1, traj_len0=1.0,
                           init_scale=2.0, seed=3, flow_epochs=0)
    plain = oracle.smc_run(t, cfg)
    flow = oracle.smc_run_flow(t, cfg, workloads.flow_init(10, 16, 4), 16, 4)
    np.testing.assert_array_equal(flow["theta"], plain["theta"])
    np.testing.assert_array_equal(flow["logw"], plain["logw"])
    assert flow["log_z"] == plain["log_z"]


def test_trained_flow_raises_acceptance_on_an_ill_conditioned_target():
    """A 4-d Gaussian with variances 0.01..4 at a step size the stiff direction
    barely tolerates: after training on the particles the map whitens the
    target and the mean acceptance of the move rises."""
    g = workloads._gauss_from_spectrum(np.array([0.01, 0.1, 1.0, 4.0]), 11)
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    cfg = oracle.SMCConfig(n_particles=512, n_iters=16, n_warmup=12, step_size=0.18, traj_len0=1.0,
                           init_scale=1.0, seed=21, adapt=0, flow_train_every=1, flow_epochs=60,
                           flow_lr=3e-3)
    plain = oracle.smc_run(t, cfg)
    flow = oracle.smc_run_flow(t, cfg, workloads.flow_init(4, 32, 4, seed=5), 32, 4)
    last = lambda r, key: np.mean([s[key] for s in r["stats"][-4:]])
    assert last(flow, "mean_alpha") > last(plain, "mean_alpha") + 0.1
    assert last(flow, "ess") > 1.3 * last(plain, "ess")


def test_zero_weight_particles_are_left_out_of_training():
    """A particle of zero weight (the end of a divergent trajectory, possibly
    non-finite) changes neither the loss nor its gradient."""
    f = _random_flow(13, scale=0.2)
    rng = np.random.default_rng(14)
    th = rng.standard_normal((6, D))
    W = rng.uniform(0.1, 1.0, 6)
    W /= W.sum()
    loss, grad = oracle.flow_loss_grad(f, th, W)
    th2 = np.vstack([th[:3], np.full((1, D), np.nan), th[3:]])
    W2 = np.concatenate([W[:3], [0.0], W[3:]])
    loss2, grad2 = oracle.flow_loss_grad(f, th2, W2)
    assert loss2 == loss
    np.testing.assert_array_equal(grad2, grad)


def test_training_gate_on_the_tested_ess():
    """With flow_min_ess = 1 no weighted set qualifies (J_eff < J whenever the
    weights are uneven), so the map never trains and stays the identity."""
    g = workloads.gauss10()
    t = oracle.TargetSpec.gauss_dense(g["mu"], g["P"])
    p0 = workloads.flow_init(10, 16, 4)
    cfg = oracle.SMCConfig(n_particles=64, n_iters=4, n_warmup=3, step_size=0.1, traj_len0=1.0,
                           init_scale=2.0, seed=3, flow_train_every=1, flow_epochs=5, flow_min_ess=1.0)
    r = oracle.smc_run_flow(t, cfg, p0, 16, 4)
    np.testing.assert_array_equal(r["flow"]["params"], p0)
    assert r["flow"]["t"].value == 0
    cfg.flow_min_ess = 0.0
    r = oracle.smc_run_flow(t, cfg, p0, 16, 4)
    assert r["flow"]["t"].value == 2 * 5          # k = 1, 2 train (k < M_warmup = 3)
