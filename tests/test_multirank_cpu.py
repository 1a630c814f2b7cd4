"""bench.py's replica path (one image per rank, weak scaling) on CPU ranks.

Two gloo processes stand in for two GPUs: the step time is the maximum over
ranks, the whole-job value counts every rank's pixels, only rank 0 prints the
JSON line, and the reference arm does its CPU work on rank 0 alone.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        ms = [4.0, 7.5][rank]  # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, dist)
        value = bench.replica_value(1024, world, worst)
        buf = io.StringIO()
        with redirect_stdout(buf):
            printed = bench.emit({"value": value, "n_gpus": world}, rank)
        # the reference arm returns at once on every rank but 0
        ref_out = io.StringIO()
        if rank != 0:
            with redirect_stdout(ref_out):
                bench.run_reference(_ref_args())
        q.put((rank, worst, value, printed, buf.getvalue(), ref_out.getvalue()))
    finally:
        dist.destroy_process_group()


def _ref_args():
    import argparse
    return argparse.Namespace(steps=2, warmup=1, levels=5, size=16384, gpus=2, scheme="reduced")


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, worst, value, printed, out, ref_out in res:
        assert worst == 7.5  # the maximum over ranks, on every rank
        assert value == pytest.approx(1024 * 1024 * 2 / 7.5e-3 / 1e9)
        assert printed == (rank == 0)
        if rank == 0:
            assert json.loads(out)["n_gpus"] == 2
        else:
            assert out == "" and ref_out == ""
