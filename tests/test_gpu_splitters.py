"""GPU parity: w-way partition by w - 1 splitters (bucket = number of splitters <=
key) through the C ABI, bit-exact against the CPU oracle (keys and payloads), on
sizes that span several tiles and end in ragged tails, with duplicate-heavy keys,
equal splitters, the balanced form, in-place calls and the error paths."""
import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu

TILE = 4096


@pytest.fixture(scope="module")
def bcf():
    import paper_1507_01391_b300 as m
    m.lib()
    return m


def _case(bcf, keys, vals, spl, balanced=False, in_place=False):
    kd = dev(keys)
    vd = None if vals is None else dev(vals)
    sd = dev(np.asarray(spl, dtype=np.uint32)) if len(spl) else dev(np.zeros(4, np.uint32))[:0]
    if in_place:
        ko, vo = bcf.partition_splitters(kd, vd, sd, balanced=balanced, keys_out=kd, vals_out=vd)
    else:
        ko, vo = bcf.partition_splitters(kd, vd, sd, balanced=balanced)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.partition_splitters(keys, vals, spl, balanced=balanced)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


def _sample_splitters(keys, nsplit, seed):
    """Sample-sort pivots: nsplit order statistics of a random sample."""
    g = synth.rng(seed)
    sample = np.sort(keys[g.integers(0, keys.size, size=max(16 * nsplit, 1))])
    return sample[(np.arange(1, nsplit + 1) * sample.size) // (nsplit + 1)].astype(np.uint32)


@pytest.mark.parametrize("n", [1, 33, TILE - 1, TILE, TILE + 1, 4 * TILE, 4 * TILE + 7, 100_001, 300_001])
@pytest.mark.parametrize("nsplit", [0, 1, 31, 255])
def test_partition_splitters_sizes(bcf, n, nsplit):
    keys = synth.uniform_keys(n, seed=n + nsplit)
    spl = _sample_splitters(keys, nsplit, seed=n) if nsplit else np.zeros(0, np.uint32)
    _case(bcf, keys, synth.index_payload(n), spl)


@pytest.mark.parametrize("vb", [0, 4, 8])
def test_partition_splitters_payload_widths(bcf, vb):
    n = 5 * TILE + 123
    keys = synth.uniform_keys(n, seed=vb)
    vals = None if vb == 0 else (synth.float_bits_payload(n, seed=1) if vb == 4
                                 else synth.uniform_keys(2 * n, seed=2).view(np.uint64))
    _case(bcf, keys, vals, _sample_splitters(keys, 100, seed=3))


def test_partition_splitters_duplicates_and_equal_splitters(bcf):
    """Zipf keys (heavy duplicates) with splitters that repeat and sit on key values."""
    n = 8 * TILE + 5
    keys = synth.zipf_keys(n, seed=4)
    spl = np.sort(np.concatenate([keys[:50], keys[:10], np.array([0, 0xFFFFFFFF], np.uint32)])).astype(np.uint32)
    _case(bcf, keys, synth.index_payload(n), spl)


@pytest.mark.parametrize("key_bits", [1, 8, 13, 20, 31])
@pytest.mark.parametrize("nsplit", [1, 2, 255])
def test_partition_splitters_narrow_key_ranges(bcf, key_bits, nsplit):
    """Keys confined to [0, 2^key_bits) (offset away from 0 for some widths), so the
    splitters span a narrow window of values, and splitters that share values or
    fall outside the keys' range."""
    n = 6 * TILE + 77
    offset = np.uint32(0 if key_bits % 2 else 0x9E3779B9 >> key_bits)
    keys = (synth.uniform_keys(n, seed=key_bits) >> np.uint32(32 - key_bits)) + offset
    spl = _sample_splitters(keys, nsplit, seed=nsplit)
    if nsplit == 255:  # a splitter above every key and one below
        spl[0], spl[-1] = 0, 0xFFFFFFFF
        spl = np.sort(spl).astype(np.uint32)
    _case(bcf, keys.astype(np.uint32), synth.index_payload(n), spl)


def test_partition_splitters_balanced_and_in_place(bcf):
    n, w = 16 * TILE, 64
    keys = (synth.random_perm(n, seed=5) * 7).astype(np.uint32)  # distinct keys
    spl = np.sort(keys)[np.arange(1, w) * (n // w)]  # exactly n/w keys per bucket
    _case(bcf, keys, synth.index_payload(n), spl, balanced=True)
    _case(bcf, keys, synth.index_payload(n), spl, balanced=False, in_place=True)


def test_partition_splitters_reports_errors(bcf):
    n = 3 * TILE
    keys = synth.uniform_keys(n, seed=6)
    bcf.partition_splitters(dev(keys), None, dev(np.array([10, 5, 20], np.uint32)))
    assert bcf.get_status() == bcf.E_BAD_KEY  # descending neighbours
    spl = np.sort(keys)[[n // 4]]  # 1/4 below, 3/4 at or above: not balanced
    bcf.partition_splitters(dev(keys), None, dev(spl), balanced=True)
    assert bcf.get_status() == bcf.E_NOT_BALANCED
    L = bcf.lib()
    import ctypes
    sz = ctypes.c_size_t(0)
    assert L.bcf_partition_splitters_workspace_size(100, 256, 4, 0, ctypes.byref(sz)) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_splitters_workspace_size(100, -1, 4, 0, ctypes.byref(sz)) == bcf.E_INVAL


@pytest.mark.slow
def test_partition_splitters_full_size_2pow26(bcf):
    """Sample-sort bucketing of 2^26 uniform keys into 256 buckets."""
    n = 1 << 26
    keys = synth.uniform_keys(n, seed=0x2D)
    _case(bcf, keys, synth.index_payload(n), _sample_splitters(keys, 255, seed=7))
