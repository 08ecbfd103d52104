"""The N > 1 benchmark path on the CPU: two gloo ranks count disjoint
colourings (no data exchange) and the job time is the slowest rank's."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    trials = bench.rank_trials(rank, 5)
    import torch
    gathered = [None] * world
    dist.all_gather_object(gathered, trials)
    slowest = bench.max_over_ranks(10.0 + rank, dist)
    q.put((rank, gathered, slowest))
    dist.destroy_process_group()


def test_two_ranks_disjoint_trials_and_max_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slowest in out:
        a, b = set(gathered[0]), set(gathered[1])
        assert len(a) == len(b) == 5 and not (a & b)
        assert slowest == 11.0
