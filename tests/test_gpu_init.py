"""GPU parity of the general Gaussian initial distribution q_init = N(m, L L^T)
(Algorithm 3's first weighting w_1 = pi / q_init) against the FP64 oracle,
through the C-ABI: the initial particles bit for bit (both sides sum
m_d + L_d0 z_0 + ... + L_dd z_d in FP64 in the same order, without
contraction, then round to FP32), the initial log-weights within the
tolerance of the isotropic draw's test, batched runs with different initial
distributions, q_init equal to a Gaussian target (constant weights, the
closed-form evidence at step 1 and after a run), and the argument checks.
"""
import numpy as np
import pytest

from gpu_util import f32r, need_gpu, oracle_target, rounded_workload, stream, torch  # noqa: F401
import oracle
import paper_2504_02627_gb300 as g
import workloads
from paper_2504_02627_gb300 import _binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _chol(D, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((D, D))
    return np.linalg.cholesky(A @ A.T / D + 0.2 * np.eye(D))


def _oracle_init(w, run, seed, mean, chol):
    t = oracle_target(w)
    cfg = oracle.SMCConfig(seed=seed, n_particles=run["n_particles"], n_iters=run["n_iters"],
                           n_warmup=run["n_warmup"], step_size=run["step_size"],
                           traj_len0=run["traj_len0"], max_steps=run["max_steps"],
                           init_scale=run["init_scale"], init_mean=mean, init_chol=chol)
    return oracle.smc_init(t, cfg)


def _check_run(w, th_gpu, lw_gpu, run, seed, mean, chol):
    """theta bit for bit against the oracle's draw; log w = log pi - log q at
    the GPU's (FP32) particles within the isotropic test's tolerance."""
    D = w["D"]
    o = _oracle_init(w, run, seed, mean, chol)
    np.testing.assert_array_equal(th_gpu, f32r(o["theta"]))
    N = run["n_particles"]
    z = np.stack([oracle.normals(seed, oracle.TAG_INIT, 0, j, D) for j in range(N)])
    logdet = np.sum(np.log(np.diag(chol))) if chol is not None else D * np.log(run["init_scale"])
    lq = -0.5 * (z**2).sum(1) - (0.5 * D * np.log(2 * np.pi) + logdet)
    lp_o, _ = oracle.logpi(oracle_target(w), th_gpu)
    np.testing.assert_allclose(lw_gpu, lp_o - lq, rtol=1e-6, atol=1e-6 * np.abs(lp_o).max())


@pytest.mark.parametrize("case", ["mean_and_chol", "mean_only", "chol_only"])
def test_initial_draw_matches_oracle(case):
    w = rounded_workload(workloads.gauss10())
    D = w["D"]
    run = dict(w["run"], n_particles=777, init_scale=0.6)
    mean = np.linspace(-1.5, 1.0, D) if case != "chol_only" else None
    chol = _chol(D, 21) if case != "mean_only" else None
    seed = 4321
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=seed, init_mean=mean, init_chol=chol, **run),
                    stream())
    th = smp.buffer(B.BUF_THETA).T.astype(np.float64)
    lw = smp.buffer(B.BUF_LOGW)
    smp.close()
    _check_run(w, th, lw, run, seed, mean, chol)


def test_batched_runs_keep_their_own_initial_distributions():
    w = rounded_workload(workloads.hier(groups=10, obs=8))
    D = w["D"]
    base = dict(n_iters=6, n_warmup=3, step_size=0.01, traj_len0=0.3, max_steps=40, init_scale=1.0)
    specs = [(500, np.full(D, 0.3), _chol(D, 5)), (333, None, None), (129, None, 0.5 * _chol(D, 6)),
             (640, -np.arange(D) / D, None)]
    cfgs, runs = [], []
    for r, (n, m, L) in enumerate(specs):
        run = dict(base, n_particles=n)
        runs.append(run)
        cfgs.append(g.make_config(seed=900 + r, init_mean=m, init_chol=L, **run))
    smp = g.Sampler(g.ModelData.from_workload(w), cfgs, stream())
    th = smp.buffer(B.BUF_THETA).T.astype(np.float64)
    lw = smp.buffer(B.BUF_LOGW)
    # a reset redraws from the same distributions (the handle's own copies)
    smp.reset(900)
    th_r = smp.buffer(B.BUF_THETA).T.astype(np.float64)
    smp.close()
    off = 0
    for r, ((n, m, L), run) in enumerate(zip(specs, runs)):
        _check_run(w, th[off:off + n], lw[off:off + n], run, 900 + r, m, L)
        off += n
    # reset(900) gives every run seed 900: run 0's draw is reproduced exactly
    np.testing.assert_array_equal(th_r[:specs[0][0]], th[:specs[0][0]])


def test_q_init_equal_to_the_target_gives_the_closed_form_evidence():
    w = rounded_workload(workloads.gauss10())
    D = w["D"]
    P = w["P"]
    Sigma = np.linalg.inv(P)
    L = np.linalg.cholesky(Sigma)
    log_norm = 0.5 * D * np.log(2 * np.pi) - 0.5 * np.linalg.slogdet(P)[1] + w.get("c", 0.0)
    run = dict(w["run"], n_particles=4096)
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=5, init_mean=w["mu"], init_chol=L, **run),
                    stream())
    lw = smp.buffer(B.BUF_LOGW)
    # the weights are constant up to the FP32 rounding of the particles
    assert np.max(np.abs(lw - log_norm)) < 1e-4
    smp.close()
    lz = []
    cfgs = [g.make_config(seed=60 + r, init_mean=w["mu"], init_chol=L, **w["run"]) for r in range(16)]
    bat = g.Sampler(g.ModelData.from_workload(w), cfgs, stream())
    bat.run(w["run"]["n_iters"])
    lz = np.asarray(bat.log_evidence())
    bat.close()
    mcse = lz.std(ddof=1) / np.sqrt(len(lz))
    assert abs(lz.mean() - log_norm) < 3 * mcse + 1e-3


@pytest.mark.parametrize("bad", ["nan_mean", "zero_diag", "negative_diag", "inf_lower"])
def test_invalid_initial_distribution_is_rejected(bad):
    w = workloads.gauss10()
    D = w["D"]
    m, L = np.zeros(D), np.eye(D)
    if bad == "nan_mean":
        m[3] = np.nan
    elif bad == "zero_diag":
        L[2, 2] = 0.0
    elif bad == "negative_diag":
        L[4, 4] = -1.0
    else:
        L[5, 1] = np.inf
    with pytest.raises(Exception):
        g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=1, init_mean=m, init_chol=L, **w["run"]), stream())
