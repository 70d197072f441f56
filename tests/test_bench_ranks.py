"""The multi-rank path of bench.py on CPU: independent replicas (no data
exchange) combined by one all-reduce of their timing and counts, with the
gloo backend and world size 2 (the benchmark runs the same code over NCCL,
one rank per GPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 100 + 10 r ms of device time, 1000 (r + 1) gradients, 5 (r + 1) ESS
        got = bench.aggregate_ranks(torch, dist, 100.0 + 10.0 * rank, 1000 * (rank + 1), 5.0 * (rank + 1), "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time and the summed work
    for r in range(world):
        assert res[r] == (110.0, 3000.0, 15.0)


def test_single_process_keeps_its_own_numbers():
    assert bench.aggregate_ranks(torch, None, 12.5, 40, 2.0, "cpu") == (12.5, 40.0, 2.0)
