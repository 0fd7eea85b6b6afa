"""The bench's multi-GPU path on CPU: two gloo ranks run its rendezvous,
barrier and max-over-ranks timing (the replicas share nothing else), and the
reference arm runs on rank 0 only."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    # each rank reports its own time; the job's time is the slowest rank's
    t = bench.allreduce_max(10.0 * (r + 1), w)
    bench.barrier(w)
    # the reference arm: ranks other than 0 return at once without output
    if r != 0:
        assert bench.run_reference(types.SimpleNamespace(), w, r) is None
    q.put((r, w, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2, 20.0), (1, 2, 20.0)]
