"""The multi-rank bookkeeping of bench.py, run as world_size-2 gloo process groups on the CPU.

Replica runs report, on rank 0, the slowest rank's span and the steps of all ranks; the
reference arm runs on rank 0 only and the other ranks leave without work.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _combine_worker(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r took 1000 + 500 r ms for 1e9 (r + 1) path-steps
        span, steps, value = bench.combine_ranks(1000.0 + 500.0 * rank, 1e9 * (rank + 1), ws, "cpu")
        out[rank] = (span, steps, value)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_combine_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        span, steps, value = res[rank]
        assert span == 1500.0                    # the slower rank
        assert steps == 3e9                      # both ranks' work
        assert value == pytest.approx(3e9 / 1.5)


def test_combine_ranks_single_rank_exchanges_nothing():
    import bench
    assert bench.combine_ranks(2000.0, 4e9, 1, None) == (2000.0, 4e9, 2e9)


def _reference_worker(rank, ws, out):
    import bench
    os.environ.update(WORLD_SIZE=str(ws), RANK=str(rank), LOCAL_RANK=str(rank))
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": ws})()
    if rank != 0:
        bench.run_reference(args)          # must return at once, without touching the oracle
        out[rank] = "returned"


def test_reference_arm_other_ranks_do_no_work():
    with mp.Manager() as mgr:
        out = mgr.dict()
        ctx = mp.get_context("spawn")
        p = ctx.Process(target=_reference_worker, args=(1, 2, out))
        p.start()
        p.join(60)
        assert p.exitcode == 0
        assert dict(out) == {1: "returned"}
