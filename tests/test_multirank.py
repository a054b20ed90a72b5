"""The N-rank bench path on the CPU: two gloo ranks (no GPU).  Each rank owns a disjoint shard of
independent knots, and the timing is the maximum over ranks; nothing else is exchanged."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    curves, cfg, indep = bench.workload("knots8x4096", rank)
    local_time = 1.0 + rank          # rank 1 is the slow one
    tmax = bench.max_over_ranks(local_time, dist, "cpu")
    out[rank] = (cfg["workload"], float(curves.gamma[0, 0]), tmax, indep)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_and_max_timing():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (w0, g0, t0, i0), (w1, g1, t1, i1) = res[0], res[1]
    assert w0.endswith("seeds1-8") and w1.endswith("seeds9-16")   # disjoint units of work
    assert g0 != g1
    assert t0 == t1 == 2.0                                        # max over ranks on every rank
    assert i0 == i1 == 1


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
