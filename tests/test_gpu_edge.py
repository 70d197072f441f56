"""Degenerate and empty cases through the C-ABI on the GPU:

* a zero-step trajectory is the identity for every kernel family and
  precision: positions and momenta unchanged bit for bit, log pi equal to the
  target evaluation's, the gradient that evaluation's (mixed with particles
  that do move, so each kernel's per-particle step masks are exercised);
* empty launches (N = 0) succeed and write nothing;
* a one-particle sampler runs (J_eff = 1 never falls below J/2), in the SMC
  and the independent-chain form.
"""
import numpy as np
import pytest

from gpu_util import dev, need_gpu, ptr, rounded_workload, stream, torch  # noqa: F401
import paper_2504_02627_gb300 as g
import workloads
from paper_2504_02627_gb300 import _binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


CASES = [("gauss10", 0), ("gauss10", 1), ("gauss100", 0), ("gauss100", 1), ("gauss100", 2),
         ("logistic", 0), ("logistic", 1), ("logistic", 2), ("hier", 0), ("banana50", 0)]


def _workload(name):
    return {"gauss10": workloads.gauss10, "gauss100": workloads.gauss100_cond,
            "logistic": lambda: workloads.logistic(n=400, d_features=6),
            "hier": lambda: workloads.hier(groups=10, obs=8), "banana50": workloads.banana50}[name]()


@pytest.mark.parametrize("name,precision", CASES)
def test_zero_steps_is_identity(name, precision):
    w = rounded_workload(_workload(name))
    D, N = w["D"], 333
    s = stream()
    dm = B.DevModel(B.ModelData.from_workload(w), s)
    rng = np.random.default_rng(5)
    th0 = (0.05 * rng.standard_normal((D, N))).astype(np.float32)
    p0 = rng.standard_normal((D, N)).astype(np.float32)
    th, p = dev(th0), dev(p0)
    gr = torch.zeros((D, N), dtype=torch.float32, device="cuda")
    lp = torch.zeros(N, dtype=torch.float64, device="cuda")
    lib = B.lib()
    B.check(lib.smc_k_target(dm.h, ptr(th), N, N, ptr(lp), ptr(gr), precision, s), "smc_k_target")
    lp_eval, gr_eval = lp.cpu().numpy().copy(), gr.cpu().numpy().copy()
    steps = np.where(np.arange(N) % 3 == 0, 3, 0).astype(np.int32)     # a third of them move
    st = dev(steps)
    B.check(lib.smc_k_leapfrog(dm.h, ptr(th), ptr(p), ptr(gr), ptr(lp), ptr(st), 1e-3, N, N, precision, s),
            "smc_k_leapfrog")
    still = steps == 0
    np.testing.assert_array_equal(th.cpu().numpy()[:, still], th0[:, still])
    np.testing.assert_array_equal(p.cpu().numpy()[:, still], p0[:, still])
    np.testing.assert_array_equal(lp.cpu().numpy()[still], lp_eval[still])
    np.testing.assert_array_equal(gr.cpu().numpy()[:, still], gr_eval[:, still])
    assert np.any(th.cpu().numpy()[:, ~still] != th0[:, ~still])
    dm.close()


def test_empty_launches():
    w = rounded_workload(workloads.gauss10())
    s = stream()
    dm = B.DevModel(B.ModelData.from_workload(w), s)
    lib = B.lib()
    t = torch.zeros(4, device="cuda")
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert lib.smc_k_target(dm.h, ptr(t), 0, 0, ptr(d), ptr(t), 0, s) == 0
    assert lib.smc_k_leapfrog(dm.h, ptr(t), ptr(t), ptr(t), ptr(d), ptr(i), 0.1, 0, 0, 0, s) == 0
    assert lib.smc_k_jitter(3, 1, 0, 10, 1, ptr(d), s) == 0
    assert lib.smc_k_steps(0, 10, 1, 1.0, 0.1, 10, 1, None, ptr(i), s) == 0
    torch.cuda.synchronize()
    assert float(d.abs().sum()) == 0.0 and int(i.abs().sum()) == 0
    dm.close()


@pytest.mark.parametrize("mcmc", [0, 1])
def test_single_particle_sampler(mcmc):
    w = rounded_workload(workloads.gauss10())
    run = dict(w["run"], n_particles=1, n_iters=5, n_warmup=2)
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=3, mcmc=mcmc, **run), stream())
    st = smp.run(5, with_stats=True)
    assert all(x["resampled"] == 0 and x["ess"] == 1.0 for x in st)
    assert np.isfinite(smp.log_evidence()[0])
    th, lw = smp.particles()
    assert np.all(np.isfinite(th))
    smp.close()
