"""The multi-GPU path of bench.py runs independent replicas (the solve does not shard here): every rank solves
the same workload and the job's time is the slowest rank's. Checked on CPU with world_size-2 gloo process groups."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")     # rank 1 is the slowest replica
        r, w, local = bench._env_rank()
        q.put((rank, got, r, w, local))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [x[1] for x in res] == [15.0, 15.0]
    assert [(x[2], x[3], x[4]) for x in res] == [(0, 2, 0), (1, 2, 1)]


def test_max_over_ranks_without_a_group_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    import workloads as wl
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        warmup, steps, ref_iters = 1, 1, 1
    assert bench.run_reference(A, wl.GRID16_K64) == 0
    assert capsys.readouterr().out == ""
