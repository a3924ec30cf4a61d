"""The multi-process bench path on CPU: two gloo ranks agree on the max-over-ranks
step time and on the whole-job throughput (independent replicas, no collective on
the data path; only the timing reduction is a collective)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    ms = 10.0 + 5.0 * rank                   # rank 1 is the slow one
    got = bench.max_over_ranks(ms, world, device=torch.device("cpu"))
    n_per_rank = 1000
    value = n_per_rank * world / (got / 1e3)
    out[rank] = (got, value)
    dist.destroy_process_group()


def test_two_rank_max_over_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    assert out[0][0] == 15.0
    assert abs(out[0][1] - 2000 / 0.015) < 1e-6


def test_replica_seeds_differ():
    """Each rank draws its own system (seed + 1000 * rank): replicas, not copies."""
    from paper_2005_12351_gb300 import synth
    a = synth.make_system(100, 1, "uniform", 20260001)[0]
    b = synth.make_system(100, 1, "uniform", 20260001 + 1000)[0]
    assert not (a == b).all()
