"""The multi-rank host logic of bench.py (replicas only: a barrier and the maximum of the
per-rank timings, whole-job throughput summed over the replicas), on CPU with gloo ranks."""
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


def _rank_main(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r timed (1 + r) s for the filter and (3 - r) s for the whole step
        t_filter, t_step = bench.max_over_ranks([1.0 + rank, 3.0 - rank], dist, "cpu")
        value = bench.weak_value(world, 2560, t_filter)
        q.put((rank, t_filter, t_step, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_value_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_filter, t_step, value in res:
        assert t_filter == 2.0 and t_step == 3.0      # the slowest rank decides
        assert value == 2 * 2560 / 2.0               # both replicas' work over the max time


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
    assert bench.weak_value(1, 100, 2.0) == 50.0
