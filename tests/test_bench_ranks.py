"""Host logic of bench.py's multi-process run (one process per GPU, replicas
only): the step time is the maximum over the ranks, and only rank 0 of the
reference arm does any work.  Run as two gloo processes on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, bench.max_over_ranks(1.5 + rank, world, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_maximum_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 2.5, 1: 2.5}


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    called = []
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "build_matrix", lambda: called.append(1))
    assert bench.run_reference(None) is None
    assert called == []
