"""The multi-GPU form of the benchmark runs independent replicas (weak scaling, no
collective on the data path); its only collectives are the barrier and the max over
ranks of the timed region.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    elapsed = [2.0, 3.5][rank]
    dist.barrier()
    m = bench.reduce_max(elapsed, dist, torch.device("cpu"))
    q.put((rank, m, bench.replica_rate(world, 4, 10, 1e12, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    import torch.multiprocessing as mp

    ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = ROOT + os.pathsep + os.environ.get("PYTHONPATH", "")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [3.5, 3.5]
    # 2 replicas x 4 steps x 10 vectors x 1e12 flop in 3.5 s
    assert got[0][2] == pytest.approx(2 * 4 * 10 * 1e12 / 3.5 / 1e12)
