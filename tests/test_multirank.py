"""The benchmark's multi-rank host logic on CPU, as gloo ranks (world size 2):
the barrier, the max-over-ranks step time, the whole-job value, and the
reference arm's rule that only rank 0 works and prints.  (The state vector does
not shard; under torchrun every rank runs an independent replica.)"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import io
    import contextlib
    import types
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)
        value = bench.whole_job_value(world, 1.0e9, ms)
        printed = ""
        if rank != 0:
            buf = io.StringIO()
            args = types.SimpleNamespace(n=4, depth=1, warmup=0, steps=1, gpus=world)
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args, world, rank, dist)
            printed = buf.getvalue()
        bench.barrier(dist)
        out.put((rank, ms, value, printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, printed in res:
        assert ms == 15.0                       # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 1.0e9 / 15.0e-3)
        assert printed == ""                    # only rank 0 runs the reference arm
