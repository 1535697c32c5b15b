"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2).

The benchmark runs independent replicas per rank; the only cross-rank steps
are the barrier around the timed region and the max over ranks of the
elapsed time.  Those run here with the gloo backend on 127.0.0.1.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    m = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    bench.barrier(world)
    q.put((rank, m))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_barrier_and_max_over_ranks_gloo():
    if torch.cuda.is_available():
        pytest.skip("the CPU (gloo) variant runs on CPU-only hosts")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=100) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert got == {0: 3.0, 1: 3.0}
