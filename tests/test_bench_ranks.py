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


def test_reference_arm_line_has_the_contract_keys(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the bench contract's
    keys, its CPU baseline and an end-to-end block that moves no bytes."""
    import json
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"])
    args = bench.parse()
    assert bench.run_reference(args) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and "workload" in line["config"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_every_bench_row_has_an_oracle_case():
    """Each row the bench can report finds its oracle sample (a renamed row would
    otherwise lose the timing beside it)."""
    names = ["partition_w32_n65536", "partition_w32_n65536_eager", "partition_w32_n65536_lemma1",
             "partition_w32_n65536_unbalanced", "permute_kv_2pow24", "permute_kv_scatter_2pow24",
             "permute_kv_fused_2pow24", "permute_keys_2pow24", "permute_keys_scatter_2pow24",
             "tile_permute_scatter_2pow24", "tile_permute_coloured_2pow24",
             "tile_permute_coloured_sorted_finish_2pow24", "permute_kv_2pow26", "permute_kv_scatter_2pow26",
             "sort_kv_2pow26_uniform", "sort_kv_2pow26_zipf", "sort_kv_2pow26_24bit",
             "partition_splitters_255_2pow26", "partition_w256_2pow26", "partition_w256_2pow26_lemma1",
             "tile_sort_lemma1_2pow24", "segmented_sort_batched_10k", "segmented_partition_batched_10k",
             "autograd_sort_by_key_64x65536", "autograd_permute_rows_64x65536"]
    rows = {n: {"gkeys_s": 1.0} for n in names}
    info = bench.oracle_rows(rows)
    assert info["kind"] == "oracle"
    for n in names:
        assert rows[n]["oracle_gkeys_s"] > 0 and rows[n]["gpu_vs_oracle"] > 0, n
