"""GPU: every sweep tile configuration gives the oracle's result, and the
autotuner picks a configuration per size and caches it per device."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bcf():
    import paper_1507_01391_b300 as m
    m.lib()
    yield m
    for op in (m.OP_SORT, m.OP_PARTITION):
        for k in range(64):
            m.lib().bcf_tune_set(op, k, -1)


@pytest.mark.parametrize("n", [1, 1000, 1023, 1024, 1025, 3 * 8192 + 17, 100_000])
def test_every_config_sorts_and_partitions(bcf, n):
    from paper_1507_01391_b300 import tune
    k = (n - 1).bit_length() if n > 1 else 0
    keys = synth.uniform_keys(n, seed=n)
    vals = synth.index_payload(n)
    rk, rv = oracle.sort_kv(keys, vals)
    lab = synth.random_labels(n, 200, seed=n + 1)
    pk, pv = oracle.partition_kv(lab, vals, 200)
    for c in range(len(tune.configs())):
        tune.set_config("sort", k, c)
        tune.set_config("partition", k, c)
        assert tune.get_config("sort", n) == c
        ko, vo = bcf.sort(dev(keys), dev(vals))
        assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv), c
        ko, vo = bcf.partition(dev(lab), dev(vals), 200)
        assert bits_equal(host(ko, np.uint32), pk) and bits_equal(host(vo, np.uint32), pv), c
    assert bcf.get_status() == bcf.OK


def test_autotune_and_cache(bcf, tmp_path):
    from paper_1507_01391_b300 import tune
    res = tune.autotune(ops=("sort", "partition"), log2_sizes=[14, 18], reps=2)
    for op in ("sort", "partition"):
        for k in (14, 18):
            best, times = res[op][k]
            assert best == min(times, key=times.get)
            assert tune.get_config(op, 1 << k) == best
    path = tune.save(res, str(tmp_path / "tune.txt"))
    for op in ("sort", "partition"):
        tune.set_config(op, 14, -1)
    assert tune.load(path)
    assert tune.get_config("sort", 1 << 14) == res["sort"][14][0]


def test_autotune_batched_sort(bcf, tmp_path):
    """The batched sort's entries: only its two 4096-key counts + scan forms are
    timed, the fastest is kept, saved and loaded back."""
    from paper_1507_01391_b300 import tune
    assert tune.candidates("segmented_sort") == [4, 8]
    res = tune.autotune(ops=("segmented_sort",), log2_sizes=[16], reps=2)
    best, times = res["segmented_sort"][16]
    assert set(times) == {4, 8} and best == min(times, key=times.get)
    assert tune.get_config("segmented_sort", 1 << 16) == best
    path = tune.save(res, str(tmp_path / "tune.txt"))
    tune.set_config("segmented_sort", 16, -1)
    assert tune.get_config("segmented_sort", 1 << 16) == 4
    assert tune.load(path) and tune.get_config("segmented_sort", 1 << 16) == best
    tune.set_config("segmented_sort", 16, -1)


def test_tune_cache_keeps_other_devices(bcf, tmp_path):
    """bcf_tune_save rewrites only this device's lines of the cache file."""
    from paper_1507_01391_b300 import tune
    path = tmp_path / "tune.txt"
    path.write_text("bcf-tune 1\nOther GPU/7sm\t0\t20\t2\n")
    tune.set_config("sort", 20, 3)
    tune.save(path=str(path))
    lines = path.read_text().splitlines()
    assert lines[0] == "bcf-tune 1" and "Other GPU/7sm\t0\t20\t2" in lines
    mine = [ln for ln in lines[1:] if not ln.startswith("Other GPU")]
    assert any(ln.endswith("\t0\t20\t3") for ln in mine)
    tune.set_config("sort", 20, -1)
    assert tune.load(str(path)) and tune.get_config("sort", 1 << 20) == 3
    tune.set_config("sort", 20, -1)
