"""The multi-rank parts of bench.py on the CPU: max-over-ranks timing through a
world_size-2 gloo group, the whole-job aggregate, and the reference arm printing
on rank 0 only.  No GPU, no oracle run."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.0, 30.0][rank]  # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    value, ms_step = bench.aggregate(ms, 10, world, 1000)
    out.put((rank, ms, value, ms_step))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(out.get() for _ in range(world))
    for rank, ms, value, ms_step in res:
        assert ms == 30.0  # every rank sees the slowest rank's time
        assert ms_step == 3.0
        assert value == pytest.approx(2 * 1000 / 3.0e-3 / 1e9)  # both ranks' keys in that time


def test_single_rank_needs_no_group():
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    value, ms_step = bench.aggregate(20.0, 4, 1, 2 ** 25)
    assert ms_step == 5.0 and value == pytest.approx(2 ** 25 / 5e-3 / 1e9)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    args = bench.parse()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
