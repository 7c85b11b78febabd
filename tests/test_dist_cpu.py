"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): whole-job
time is the maximum over ranks and lattice updates are summed; batched
instances are split over ranks without overlap and balanced by size."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t, u = bench.job_totals(1.0 + rank, 10 * (rank + 1), ws, "cpu")
    out.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_job_totals_single_rank_is_identity():
    import bench
    assert bench.job_totals(0.5, 7, 1, "cpu") == (0.5, 7.0)


@pytest.mark.parametrize("ws", [1, 2, 3, 8])
def test_shard_instances_partition(ws):
    import bench
    from paper_1403_1937_gb300 import workloads as wl
    sizes = [i.n for i in wl.config4(count=64, side=(64, 256))]
    parts = bench.shard_instances(sizes, ws)
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(sizes)))          # every instance exactly once
    loads = [sum(sizes[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)    # greedy balance bound
    assert parts == bench.shard_instances(sizes, ws)   # deterministic
