"""The N > 1 path of bench.py on CPU: replicas (one lattice per rank, no data-path collective) meet
only in the barrier and the max-over-ranks timing; the whole-job value counts every rank's bytes.
Two gloo ranks on 127.0.0.1."""
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
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    w, r, local = bench.dist_setup()
    dist.init_process_group("gloo", rank=r, world_size=w)
    dist.barrier()
    mine = [1.0 + r, 10.0 - r]  # rank 0 is slower in the second timing, rank 1 in the first
    got = bench.max_over_ranks(mine, dist, "cpu")
    value = bench.whole_job_gbs(w, 2_000_000_000, 5, got[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, got, value))


def test_two_gloo_ranks_take_the_max_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, got, value in out:
        assert w == world
        assert got == [2.0, 10.0]  # max over ranks, elementwise
        assert value == pytest.approx(2 * 2_000_000_000 * 5 / 2.0 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    res, rank = bench.run_reference(type("A", (), {"warmup": 3, "steps": 1})())
    assert res is None and rank == 1
