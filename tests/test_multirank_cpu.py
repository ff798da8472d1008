"""The N > 1 host logic of bench.py on CPU with gloo ranks: the slowest
rank's time sets the whole-job rate, every rank contributes its own
instance (weak scaling), and the reference arm does no work off rank 0."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    m = bench.max_over_ranks(ms, dist)
    rate = bench.aggregate_rate(1000, 4, world, m)
    q.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert all(abs(o[2] - 2 * 1000 * 4 / 0.015) < 1e-6 for o in out)


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.aggregate_rate(10, 2, 1, 1.0) == 20000.0


def test_reference_arm_only_runs_on_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")

    class Args:
        ref_n = 8
        steps = 1
        warmup = 0
        gpus = 2
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
