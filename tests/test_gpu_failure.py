"""Failure detection without a GPU fault: the resampling scan's bounded
look-back wait, made to run out on the GPU by a predecessor tile that nothing
ever publishes (smc_k_lookback_wait_check).  The wait must give up after its
poll limit, report -5 (the status the sampler turns into SMC_E_TIMEOUT), and
leave the context usable: an ordinary resampling call afterwards still runs
and gives the allocating entry's result.  The argument checks run on the
host before any CUDA call, so they are tested without a GPU.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, need_gpu, ptr, stream, torch  # noqa: F401
import paper_2504_02627_gb300 as g


@pytest.mark.gpu
@pytest.mark.parametrize("limit", [1, 1000, 100000])
def test_lookback_wait_gives_up_and_reports_timeout(limit):
    need_gpu()
    lib = g.lib()
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    scratch = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert lib.smc_k_lookback_wait_check(limit, ptr(st), ptr(scratch), stream()) == 0
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == -5
    # the context still works: a real resampling call after the timeout
    N = 3000
    W = np.random.default_rng(4).gamma(0.5, size=N)
    W /= W.sum()
    W_d = dev(W)
    q = torch.empty(N, dtype=torch.int64, device="cuda")
    anc = torch.empty(N, dtype=torch.int32, device="cuda")
    st2 = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    sc = torch.empty(lib.smc_k_resample_scratch_bytes(N), dtype=torch.uint8, device="cuda")
    assert lib.smc_k_resample(ptr(W_d), N, 12345, ptr(q), ptr(anc), ptr(st2), ptr(sc), stream()) == 0
    torch.cuda.synchronize()
    assert int(st2.cpu()[0]) == 0
    a = anc.cpu().numpy()
    assert a.min() >= 0 and a.max() < N and np.all(np.diff(a) >= 0)


def test_lookback_wait_check_rejects_bad_arguments():
    # checked on the host before any CUDA call: no GPU needed
    lib = g.lib()
    one = ctypes.c_void_p(16)
    assert lib.smc_k_lookback_wait_check(0, one, one, None) == -1
    assert lib.smc_k_lookback_wait_check(1 << 41, one, one, None) == -1
    assert lib.smc_k_lookback_wait_check(10, None, one, None) == -1
    assert lib.smc_k_lookback_wait_check(10, one, None, None) == -1
