"""bench.py's multi-rank plumbing on CPU: world_size 2 over gloo, the step
time is the max over ranks and the work units the sum (weak scaling of
independent replicas; no data-path collective)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      BENCH_BACKEND="gloo")
    import bench
    r, w = bench.dist_init()
    assert (r, w) == (rank, world)
    bench.barrier(w)
    t, u = bench.reduce_max_sum(w, 1.0 + rank, 10.0 * (rank + 1), device="cpu")
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_max_time_and_summed_units_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == (2.0, 30.0) and res[1] == (2.0, 30.0)


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_max_sum(1, 3.5, 7.0) == (3.5, 7.0)
