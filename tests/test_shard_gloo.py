"""The exchange step of particle-sharded resampling over gloo ranks on the
CPU (4 ranks, uneven slices, one empty): the ancestors every rank computes for
its output slots equal, bit for bit, those of one device resampling all
particles (the oracle's fixed-point systematic rule); the exchanged rows are
those of the ancestors; and the normalisation partials give every rank the
same log-sum-exp and ESS, equal to one device's to FP64 rounding."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2504_02627_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SIZES = [37, 0, 64, 29]      # one rank with no particles


def _case(seed):
    rng = np.random.default_rng(seed)
    N = sum(SIZES)
    W = rng.gamma(0.3, size=N)
    W[rng.choice(N, 20, replace=False)] = 0.0      # some zero weights
    W /= W.sum()
    _, q = oracle.quantise(W)
    theta = rng.standard_normal((N, 3))
    return q, theta, int(rng.integers(0, 2**63)) * 2 + 1


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for seed in (1, 2, 3):
            q, theta, r64 = _case(seed)
            lo = int(np.sum(SIZES[:rank]))
            sl = slice(lo, lo + SIZES[rank])
            anc = shard.systematic_shard(q[sl], r64, dist)
            rows = shard.gather_rows(theta[sl], anc, dist)
            lw = np.log(np.random.default_rng(seed + 100).gamma(0.3, size=sum(SIZES))) * 3.0
            lse, ess, W = shard.normalise_shard(lw[sl], dist)
            res.append((anc.tolist(), rows.tolist(), lse, ess, W.tolist()))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_sharded_systematic_matches_single_device():
    world = len(SIZES)
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for i, seed in enumerate((1, 2, 3)):
        q, theta, r64 = _case(seed)
        _, anc_ref = oracle.systematic(q, r64)
        anc = np.concatenate([np.array(res[r][i][0], dtype=np.int64) for r in range(world)])
        np.testing.assert_array_equal(anc, anc_ref)
        rows = np.concatenate([np.array(res[r][i][1]).reshape(-1, 3) for r in range(world)])
        np.testing.assert_array_equal(rows, theta[anc_ref])
        # the normalisation partials: every rank gets the same LSE and ESS, equal
        # to one device's to FP64 rounding, and the slices of W
        lw = np.log(np.random.default_rng(seed + 100).gamma(0.3, size=sum(SIZES))) * 3.0
        lse_o, ess_o, W_o = oracle.normalise(lw)
        assert len({res[r][i][2] for r in range(world)}) == 1 and len({res[r][i][3] for r in range(world)}) == 1
        assert abs(res[0][i][2] - lse_o) <= 1e-12 * abs(lse_o) and abs(res[0][i][3] - ess_o) <= 1e-10 * ess_o
        W = np.concatenate([np.array(res[r][i][4]) for r in range(world)])
        np.testing.assert_allclose(W, W_o, rtol=1e-12, atol=0)
