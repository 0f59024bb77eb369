"""bench.py's N > 1 path (one replica per GPU): barrier and max-over-ranks timing,
exercised as two gloo ranks on the CPU. The sort itself has no collective: the
workload does not shard (replicas only)."""
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, lr = bench.dist_env()
    rep = bench.Replicas(w, r, lr, "gloo")
    rep.barrier()
    m = rep.max(1.5 + rank)  # each rank's elapsed time; the job's is the max
    rep.barrier()
    rep.close()
    out.put((rank, w, m))


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas(1, 0, 0, "gloo")
    assert rep.max(3.0) == 3.0
    rep.barrier()
    rep.close()
