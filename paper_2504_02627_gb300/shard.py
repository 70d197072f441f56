"""Particle-sharded resampling across ranks: the exchange step a multi-GPU
SMC iteration would need (host logic, any torch.distributed backend).

Ranks own contiguous slices of the particles (rank r: global indices
[off_r, off_r + n_r)) and, after resampling, the same slices of the output
slots.  Systematic resampling in fixed point (Sec. 3: the resampling step
of Algorithm 3) needs only two scalars per rank to be exchanged -- its
particle count and its total fixed-point weight T_r -- because output slot o
takes the particle j whose inclusive prefix satisfies
cnt(C_{j-1}) <= o < cnt(C_j), cnt(C) = min(N, ceil((N C - U) / T)),
U = floor(r64 T / 2^64), and a rank's prefixes are its own cumulative sums
plus the totals of the ranks before it.  Each rank emits (slot, ancestor)
pairs for its own particles, the pairs go to the slots' owners, and the
ancestors' rows are fetched from the ranks that hold them.  All arithmetic is
on integers, so the ancestors are bit-identical to one device resampling all
particles at once.

On one GPU per box the library runs independent replicas instead; this
module is the tested design of the exchange (the normalisation partials,
an all-gather of two integers, one all-to-all of pairs, one all-to-all of
row requests and one of rows: a rank receives only what is addressed to it).
"""
from __future__ import annotations

import numpy as np


def _count(C: int, N: int, T: int, U: int) -> int:
    """Output slots i with i T + U < N C, clipped to [0, N]."""
    v = N * C - U
    if v <= 0:
        return 0
    return min(N, -(-v // T))


def _layout(n_local: int, t_local: int, dist):
    import torch
    world = dist.get_world_size()
    info = torch.tensor([n_local, t_local], dtype=torch.int64)
    allinfo = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allinfo, info)
    ns = [int(a[0]) for a in allinfo]
    ts = [int(a[1]) for a in allinfo]
    return ns, ts


def normalise_shard(logw_local, dist):
    """Global log-sum-exp and ESS (Eqs. for W and J_eff) of log-weights spread
    over the ranks: each rank contributes (max, sum exp(lw - max),
    sum exp(2 (lw - max))) of its slice; the partials are gathered and
    combined in rank order, so every rank gets the same bits.  Returns
    (lse, ess, W_local) with W_local = exp(lw - lse) for this rank's slice."""
    import torch
    world = dist.get_world_size()
    lw = np.asarray(logw_local, dtype=np.float64)
    m = lw.max() if lw.size and np.isfinite(lw.max()) else -np.inf
    if np.isfinite(m):
        e = np.exp(lw - m)
        part = [m, float(e.sum()), float((e * e).sum())]
    else:
        part = [-np.inf, 0.0, 0.0]
    t = torch.tensor(part, dtype=torch.float64)
    parts = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, t)
    M = max(float(p[0]) for p in parts)
    if not np.isfinite(M):
        raise ValueError("all weights are zero")
    s1 = s2 = 0.0
    for p in parts:                                     # rank order
        if np.isfinite(float(p[0])):
            f = np.exp(float(p[0]) - M)
            s1 += float(p[1]) * f
            s2 += float(p[2]) * f * f
    lse = M + np.log(s1)
    return lse, s1 * s1 / s2, np.exp(lw - lse)


def systematic_shard(q_local, r64: int, dist) -> np.ndarray:
    """Global ancestor index of every output slot this rank owns, from its
    slice of the fixed-point weights q (each < 2^62, their global sum T < 2^63)
    and the iteration's 64-bit uniform r64."""
    world, rank = dist.get_world_size(), dist.get_rank()
    q_local = [int(x) for x in np.asarray(q_local, dtype=np.uint64)]
    ns, ts = _layout(len(q_local), sum(q_local), dist)
    N, T = sum(ns), sum(ts)
    if T == 0:
        raise ValueError("all weights are zero")
    p_off, c_off = sum(ns[:rank]), sum(ts[:rank])
    out_lo = np.cumsum([0] + ns)                       # rank r owns slots [out_lo[r], out_lo[r + 1])
    U = (r64 * T) >> 64
    pairs = [[] for _ in range(world)]
    C = c_off
    for j, qj in enumerate(q_local):
        lo = _count(C, N, T, U)
        C += qj
        hi = _count(C, N, T, U)
        for o in range(lo, hi):
            r = int(np.searchsorted(out_lo, o, side="right") - 1)
            pairs[r].append((o, p_off + j))
    flat = [np.asarray(pr, dtype=np.int64).reshape(-1, 2) for pr in pairs]
    got = _all_to_all(flat, 2, np.int64, dist)          # the pairs of the slots this rank owns
    mine = got[np.argsort(got[:, 0], kind="stable")]
    anc = mine[:, 1].copy()
    assert len(anc) == ns[rank] and np.array_equal(mine[:, 0], out_lo[rank] + np.arange(ns[rank]))
    return anc


def _all_to_all(blocks, width, dtype, dist):
    """Point-to-point exchange: blocks[r] ([k_r, width] rows) goes to rank r;
    returns the rows every rank sent to this one, in sender order.  One
    all-to-all of the row counts, then one of the rows themselves, so a rank
    receives only what is addressed to it."""
    import torch
    world = dist.get_world_size()
    send_counts = torch.tensor([len(b) for b in blocks], dtype=torch.int64)
    recv_counts = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(recv_counts, send_counts)
    rc = [int(x) for x in recv_counts]
    send = torch.from_numpy(np.concatenate([np.asarray(b, dtype=dtype).reshape(-1, width) for b in blocks])
                            .reshape(-1).copy())
    recv = torch.empty(sum(rc) * width, dtype=send.dtype)
    dist.all_to_all_single(recv, send, [c * width for c in rc], [len(b) * width for b in blocks])
    return recv.numpy().reshape(-1, width)


def gather_rows(rows_local: np.ndarray, anc: np.ndarray, dist) -> np.ndarray:
    """rows_local [n_local, D] of this rank's particles; returns the rows of
    the global indices `anc` (this rank's ancestors), fetched from the ranks
    that own them."""
    world, rank = dist.get_world_size(), dist.get_rank()
    ns, _ = _layout(len(rows_local), 0, dist)
    lo = np.cumsum([0] + ns)
    owner = np.searchsorted(lo, anc, side="right") - 1
    want = [np.unique(anc[owner == r]).astype(np.int64) for r in range(world)]
    asks = _all_to_all([w.reshape(-1, 1) for w in want], 1, np.int64, dist)[:, 0]   # indices others need from me
    # the asked rows, in the order the asks arrived (sender by sender)
    recv_counts = _ask_counts(want, dist)
    off = np.cumsum([0] + recv_counts)
    D = rows_local.shape[1] if rows_local.ndim == 2 else 0
    give = [rows_local[asks[off[r]:off[r + 1]] - lo[rank]] for r in range(world)]
    rows = _all_to_all(give, D, rows_local.dtype, dist)   # sender order = owner order, each sorted as asked
    table = {}
    k = 0
    for r in range(world):
        for i in want[r]:
            table[int(i)] = rows[k]
            k += 1
    return np.stack([table[int(a)] for a in anc]) if len(anc) else rows_local[:0]


def _ask_counts(want, dist):
    """How many rows each rank asked this one for (the counts of the ask exchange)."""
    import torch
    world = dist.get_world_size()
    send = torch.tensor([len(w) for w in want], dtype=torch.int64)
    recv = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(recv, send)
    return [int(x) for x in recv]
