"""N > 1 host logic of bench.py on CPU (gloo, world size 2): replicas are
timed by the slowest rank and their DOF-updates add up."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
        dofs_local = 1000.0 * (rank + 1)
        ms, step_ms, value = bench.reduce_time_and_value(ms_local, dofs_local, 10, world)
        out[rank] = (ms, step_ms, value)
    finally:
        dist.destroy_process_group()


def test_replicas_max_time_and_summed_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, step_ms, value = res[r]
        assert ms == 150.0
        assert step_ms == 15.0
        assert value == pytest.approx(3000.0 * 1e3 / 15.0)


def test_single_rank_passthrough():
    import bench
    ms, step_ms, value = bench.reduce_time_and_value(20.0, 500.0, 4, 1)
    assert (ms, step_ms) == (20.0, 5.0) and value == pytest.approx(500.0 * 1e3 / 5.0)


@pytest.mark.parametrize("n,world", [(256, 2), (256, 8), (7, 4), (3, 4)])
def test_ensemble_sharding_is_a_partition(n, world):
    """every instance belongs to exactly one rank; rank loads differ by at
    most one instance"""
    import bench
    parts = [bench.shard_instances(n, world, r) for r in range(world)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def test_cpu_baseline_reports_the_threads_it_used(oracle_mod):
    """the CPU baseline's core count is the oracle's thread count, not the
    machine's"""
    import bench
    from paper_1904_08684_gb300 import inputs as I
    sample = bench._oracle_sample(I.hump_p1_32(n=8))
    sample[0].set_threads(1)
    dofs, el, reps = bench._time_sample(sample, 0.05)
    assert sample[0].threads() == 1 and reps >= 1 and dofs == 3 * 3 * len(sample[4]) * reps
    sample[0].set_threads(0)
    assert sample[0].threads() >= 1
