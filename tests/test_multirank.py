"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank times its own copy of
the workload (weak scaling, no data-path collective); the timings are reduced to the slowest
rank, the job's throughput counts every rank's nodes, and only rank 0 reports.  The
reference arm does no work on ranks other than 0."""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    C = bench.Ctx(torch, None, dist, torch.device("cpu"), world)
    C.barrier()
    t_dev, t_e2e = C.max_over_ranks(1.0 + rank, 3.0 - rank)        # rank 1 slower on the first
    value = bench.job_rhs(1000, 4, world) / t_dev / 1e6
    args = types.SimpleNamespace(warmup=1, steps=2, gpus=world, workload="vortex256", scheme=2)
    buf = io.StringIO()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(args, rank)              # returns at once on ranks other than 0
    dist.destroy_process_group()
    out.put((rank, t_dev, t_e2e, value, buf.getvalue()))


def test_two_ranks_reduce_to_the_slowest_and_count_every_rank():
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed unavailable")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_dev, t_e2e, value, printed in res:
        assert (t_dev, t_e2e) == (2.0, 3.0)                  # max over the ranks, on every rank
        assert value == pytest.approx(1000 * 3 * 4 * 2 / 2.0 / 1e6)
        assert printed == ""
