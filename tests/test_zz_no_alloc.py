"""smc_k_resample_noalloc: the resampling entry point for callers that cannot
allocate device memory where they resample.  It must give exactly what
smc_k_resample gives (bit-exact fixed-point weights, ancestors and status),
on two calls in a row (the fixed scratch keeps the previous call's contents),
and refuse sizes beyond its fixed scratch without touching the GPU.

This file is collected last on purpose, so a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, need_gpu, ptr, stream, torch  # noqa: F401
import paper_2504_02627_gb300 as g
from paper_2504_02627_gb300 import _binding as B


def _weights(N, seed):
    rng = np.random.default_rng(seed)
    W = rng.gamma(0.3, size=N)
    W[rng.uniform(size=N) < 0.2] = 0.0
    W[0] += 1e-3
    return W / W.sum()


def _run(entry, W, r64):
    N = W.size
    W_d = dev(W)
    q_d = torch.full((N,), -1, dtype=torch.int64, device="cuda")
    a_d = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    st_d = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    if entry == "noalloc":
        rc = g.lib().smc_k_resample_noalloc(ptr(W_d), N, r64, ptr(q_d), ptr(a_d), ptr(st_d), stream())
    else:
        scratch = torch.empty(g.lib().smc_k_resample_scratch_bytes(N), dtype=torch.uint8, device="cuda")
        rc = g.lib().smc_k_resample(ptr(W_d), N, r64, ptr(q_d), ptr(a_d), ptr(st_d), ptr(scratch), stream())
    assert rc == 0
    torch.cuda.synchronize()
    return q_d.cpu().numpy(), a_d.cpu().numpy(), int(st_d.cpu().numpy()[0])


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_on_two_calls_in_a_row():
    need_gpu()
    # the second call is smaller than the first, so stale descriptors of the
    # first call remain in the fixed scratch when it runs; the third is larger
    # than the second, and the last one uses the whole advertised maximum
    for N, seed, r64 in ((70001, 1, 0x9E3779B97F4A7C15), (5000, 2, 12345), (300007, 3, 2**63 + 7),
                         (B.NOALLOC_MAX_N, 4, 987654321)):
        W = _weights(N, seed)
        q0, a0, s0 = _run("alloc", W, r64)
        q1, a1, s1 = _run("noalloc", W, r64)
        assert s0 == 0 and s1 == 0
        np.testing.assert_array_equal(q1, q0)
        np.testing.assert_array_equal(a1, a0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # argument checks run before any CUDA call, so this needs no GPU
    lib = g.lib()
    one = ctypes.c_void_p(8)
    assert lib.smc_k_resample_noalloc(one, B.NOALLOC_MAX_N + 1, 1, one, one, one, None) == -1
    assert lib.smc_k_resample_noalloc(one, 0, 1, one, one, one, None) == -1


def test_noalloc_scratch_holds_the_advertised_maximum():
    # the fixed array is 64 KiB; the layout the scan uses must fit it for every
    # N up to the maximum (a host-side size query, no GPU needed)
    lib = g.lib()
    assert lib.smc_k_resample_scratch_bytes(B.NOALLOC_MAX_N) <= 65536
    assert lib.smc_k_resample_scratch_bytes(B.NOALLOC_MAX_N + 1) >= lib.smc_k_resample_scratch_bytes(B.NOALLOC_MAX_N)
