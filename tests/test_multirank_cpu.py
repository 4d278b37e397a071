"""The multi-GPU bench path is replicas only: every rank solves its own system and the ranks meet
only at a barrier and a MAX over the per-rank step times.  That host logic runs here on CPU with
the gloo backend and two ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.rank_barrier(dist)
    step_time = 0.25 + 0.5 * rank                  # the slow replica sets the job time
    t = bench.rank_max(step_time, dist)
    n = bench.rank_sum(1.0, dist)
    bench.rank_barrier(dist)
    q.put((rank, t, n))
    dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(abs(o[1] - 0.75) < 1e-15 for o in out)
    assert all(o[2] == 2.0 for o in out)


def test_single_process_helpers_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(1.5, None) == 1.5 and bench.rank_sum(2.0, None) == 2.0
    bench.rank_barrier(None)
