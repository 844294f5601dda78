"""GPU parity: radix sort and w-way partition through the C ABI, bit-exact against
the CPU oracle (keys and payloads), on seeded inputs that span several tiles and
a ragged tail, plus the full-size workloads and the device-side error paths."""
import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu

TILE = 4096
SIZES = [1, 2, 31, 32, 33, 1000, TILE - 1, TILE, TILE + 1, 3 * TILE + 5, 50_001]
# Inputs up to 2^18 keys take the single-launch look-back sweeps, larger ones the
# tile counts + scan + sweep passes: both sides of the boundary.
SMALL_MAX = 1 << 18
BOUNDARY = [SMALL_MAX - 1, SMALL_MAX, SMALL_MAX + 1, 700_001]


@pytest.fixture(scope="module")
def bcf():
    import paper_1507_01391_b300 as m
    m.lib()
    return m


def _sort_case(bcf, keys, vals, key_bits=32, in_place=False):
    kd = dev(keys)
    vd = None if vals is None else dev(vals)
    if in_place:
        ko, vo = bcf.sort(kd, vd, key_bits=key_bits, keys_out=kd, vals_out=vd)
    else:
        ko, vo = bcf.sort(kd, vd, key_bits=key_bits)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


@pytest.mark.parametrize("n", SIZES)
def test_sort_uniform_kv(bcf, n):
    _sort_case(bcf, synth.uniform_keys(n, seed=n), synth.index_payload(n))


@pytest.mark.parametrize("n", BOUNDARY)
@pytest.mark.parametrize("key_bits", [8, 32])
def test_sort_small_large_boundary(bcf, n, key_bits):
    _sort_case(bcf, synth.uniform_keys(n, seed=n + key_bits, bits=key_bits), synth.index_payload(n),
               key_bits=key_bits)


@pytest.mark.parametrize("kind", ["equal", "sorted", "reverse", "few", "zipf"])
def test_sort_structured(bcf, kind):
    n = 2 * TILE + 77
    if kind == "equal":
        keys = np.full(n, 0xDEADBEEF, np.uint32)
    elif kind == "sorted":
        keys = np.sort(synth.uniform_keys(n, seed=1))
    elif kind == "reverse":
        keys = np.sort(synth.uniform_keys(n, seed=2))[::-1].copy()
    elif kind == "few":
        keys = synth.random_labels(n, 3, seed=3)
    else:
        keys = synth.zipf_keys(n, seed=4)
    _sort_case(bcf, keys, synth.index_payload(n))


@pytest.mark.parametrize("vb", [0, 4, 8])
@pytest.mark.parametrize("key_bits", [1, 7, 8, 9, 20, 31, 32])
def test_sort_widths_and_key_bits(bcf, vb, key_bits):
    n = 2 * TILE + 333
    keys = synth.uniform_keys(n, seed=key_bits, bits=key_bits)
    vals = None
    if vb == 4:
        vals = synth.float_bits_payload(n, seed=5)  # NaN / -0.0 bit patterns
    elif vb == 8:
        vals = synth.uniform_keys(2 * n, seed=6).view(np.uint64)
    _sort_case(bcf, keys, vals, key_bits=key_bits)


@pytest.mark.parametrize("key_bits", [8, 20, 32])
def test_sort_in_place(bcf, key_bits):
    n = 3 * TILE + 1
    _sort_case(bcf, synth.uniform_keys(n, seed=9, bits=key_bits), synth.index_payload(n),
               key_bits=key_bits, in_place=True)


def test_sort_empty(bcf):
    import torch
    k = torch.empty(0, dtype=torch.int32, device="cuda")
    ko, _ = bcf.sort(k, None)
    assert ko.numel() == 0


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["uniform", "zipf"])
def test_sort_full_size_2pow26(bcf, kind):
    """The 2^26 key-value sort workload, compared in full with the oracle."""
    n = 1 << 26
    keys = synth.uniform_keys(n, seed=0x2A) if kind == "uniform" else synth.zipf_keys(n, seed=0x2B)
    _sort_case(bcf, keys, synth.index_payload(n))


# ---------------------------------------------------------------- partition
def _partition_case(bcf, keys, vals, w, balanced, in_place=False):
    kd = dev(keys)
    vd = None if vals is None else dev(vals)
    if in_place:
        ko, vo = bcf.partition(kd, vd, w, balanced=balanced, keys_out=kd, vals_out=vd)
    else:
        ko, vo = bcf.partition(kd, vd, w, balanced=balanced)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=balanced)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


def test_partition_w32_n65536_balanced(bcf):
    """The w = 32, n = 65536 workload: 2048 copies of each label."""
    n, w = 65536, 32
    _partition_case(bcf, synth.partition_keys(n, w, seed=0x1507), synth.index_payload(n), w, True)


@pytest.mark.parametrize("w", [1, 2, 5, 31, 32, 33, 64, 100, 255, 256])
@pytest.mark.parametrize("balanced", [True, False])
def test_partition_widths(bcf, w, balanced):
    n = w * (3 * TILE // w + 7)
    keys = synth.partition_keys(n, w, seed=w) if balanced else synth.random_labels(n, w, seed=w)
    _partition_case(bcf, keys, synth.index_payload(n), w, balanced)


@pytest.mark.parametrize("n", [1, 33, TILE + 1, 3 * TILE + 5])
@pytest.mark.parametrize("vb", [0, 8])
def test_partition_ragged_and_widths(bcf, n, vb):
    w = 7
    keys = synth.random_labels(n, w, seed=n)
    vals = None if vb == 0 else synth.uniform_keys(2 * n, seed=1).view(np.uint64)
    _partition_case(bcf, keys, vals, w, False)


@pytest.mark.parametrize("n", BOUNDARY)
@pytest.mark.parametrize("w", [32, 256])
@pytest.mark.parametrize("balanced", [True, False])
def test_partition_small_large_boundary(bcf, n, w, balanced):
    if balanced:
        n -= n % w
    keys = synth.partition_keys(n, w, seed=n + w) if balanced else synth.random_labels(n, w, seed=n + w)
    _partition_case(bcf, keys, synth.index_payload(n), w, balanced)


def test_partition_in_place(bcf):
    n, w = 4 * TILE, 64
    _partition_case(bcf, synth.partition_keys(n, w, seed=3), synth.index_payload(n), w, True, in_place=True)


@pytest.mark.slow
def test_partition_full_size_w256(bcf):
    n, w = 1 << 26, 256
    _partition_case(bcf, synth.partition_keys(n, w, seed=0x2C), synth.index_payload(n), w, True)


def test_partition_reports_bad_label(bcf):
    n, w = 2 * TILE, 16
    keys = synth.random_labels(n, w, seed=1)
    keys[777] = 16
    kd = dev(keys)
    bcf.partition(kd, None, w)
    assert bcf.get_status() == bcf.E_BAD_KEY
    assert bcf.get_status() == bcf.OK  # reading clears the word


def test_partition_reports_unbalanced(bcf):
    n, w = 2 * TILE, 16
    keys = synth.partition_keys(n, w, seed=2)
    keys[5] = (keys[5] + 1) % w  # one label too many, another too few
    bcf.partition(dev(keys), None, w, balanced=True)
    assert bcf.get_status() == bcf.E_NOT_BALANCED


# ------------------------------------------------- Lemma 1 tile partition
@pytest.mark.parametrize("w,balanced,n", [(32, True, 65536), (32, False, 3 * 4096 + 5), (256, True, 1 << 16),
                                          (7, False, 1000), (1, True, 4096), (200, False, 1 << 20)])
def test_partition_lemma1_schedule(bcf, w, balanced, n):
    if balanced:
        n -= n % w
    keys = synth.partition_keys(n, w, seed=w + n) if balanced else synth.random_labels(n, w, seed=w + n)
    vals = synth.float_bits_payload(n, seed=3)
    ko, vo = bcf.partition(dev(keys), dev(vals), w, balanced=balanced, flags=bcf.PARTITION_LEMMA1)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=balanced)
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.float32), rv)


def test_partition_lemma1_reports_bad_label(bcf):
    keys = synth.random_labels(5000, 16, seed=1)
    keys[123] = 40
    bcf.partition(dev(keys), None, 16, flags=bcf.PARTITION_LEMMA1)
    assert bcf.get_status() == bcf.E_BAD_KEY


# ------------------------------------------- direct write-out (w <= 32)
@pytest.mark.parametrize("w,balanced,n", [(32, True, 65536), (32, False, 3 * 4096 + 5), (1, True, 4096),
                                          (7, False, 1000), (16, True, 1 << 18), (32, False, (1 << 18) + 77),
                                          (31, False, 700_001), (32, True, 1 << 20)])
@pytest.mark.parametrize("vb", [0, 4, 8])
def test_partition_direct_write_out(bcf, w, balanced, n, vb):
    """Keys stored from registers straight to their global places: the same
    stable partition, on both sides of the single-launch / counts + scan boundary,
    ragged tails, every payload width."""
    if balanced:
        n -= n % w
    keys = synth.partition_keys(n, w, seed=w + n) if balanced else synth.random_labels(n, w, seed=w + n)
    vals = {0: None, 4: synth.float_bits_payload(n, seed=3),
            8: synth.uniform_keys(2 * n, seed=4).view(np.uint64)}[vb]
    ko, vo = bcf.partition(dev(keys), None if vals is None else dev(vals), w, balanced=balanced,
                           flags=bcf.PARTITION_DIRECT)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=balanced)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


def test_partition_direct_index_payload_and_bad_label(bcf):
    """Position payloads (vals NULL with 4-byte payloads) and a bad label."""
    n, w = 3 * 4096 + 1, 24
    keys = synth.random_labels(n, w, seed=11)
    L = bcf.lib()
    kd, ko, vo = dev(keys), dev(np.zeros(n, np.uint32)), dev(np.zeros(n, np.uint32))
    ws = bcf.workspace(bcf.partition_workspace_size(n, w, 4, bcf.PARTITION_DIRECT))
    import ctypes
    P = ctypes.c_void_p
    assert L.bcf_partition(P(kd.data_ptr()), None, P(ko.data_ptr()), P(vo.data_ptr()), n, w, 4,
                           bcf.PARTITION_DIRECT, P(ws.data_ptr()), ws.numel(), None) == bcf.OK
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.partition_kv(keys, synth.index_payload(n), w)
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv)
    keys[4242] = w
    bcf.partition(dev(keys), None, w, flags=bcf.PARTITION_DIRECT)
    assert bcf.get_status() == bcf.E_BAD_KEY


# ------------------------------------------------------ bounded look-back waits
@pytest.mark.parametrize("op", ["partition", "sort"])
def test_lookback_wait_gives_up(bcf, op):
    """A tile that never publishes its status makes the next tiles' waits run out:
    the call ends with BCF_E_TIMEOUT after a bounded number of polls instead of
    hanging, and the library works normally afterwards."""
    n, w = 65536, 32  # <= 2^18 keys: one look-back sweep per pass, several tiles
    keys = synth.partition_keys(n, w, seed=77) if op == "partition" else synth.uniform_keys(n, seed=78)
    vals = synth.index_payload(n)
    L = bcf.lib()
    assert L.bcf_debug_lookback(3, 0) == bcf.E_INVAL
    assert L.bcf_debug_lookback(3, 4096) == bcf.OK
    try:
        if op == "partition":
            bcf.partition(dev(keys), dev(vals), w, balanced=True)
        else:
            bcf.sort(dev(keys), dev(vals))
        assert bcf.get_status() == bcf.E_TIMEOUT
    finally:
        assert L.bcf_debug_lookback(-1, 0) == bcf.OK
    if op == "partition":
        _partition_case(bcf, keys, vals, w, True)
    else:
        _sort_case(bcf, keys, vals)


@pytest.mark.slow
def test_sort_largest_size_by_properties(bcf):
    """The largest sort the library takes (n < 2^30; here 2^30 - 4099 keys, a ragged
    last tile), too large for the oracle, checked by what determines a stable sort's
    output at any size: the keys come out ascending (as uint32), the returned
    permutation is a permutation and carries every key from its input position, and
    equal keys keep their input order."""
    import torch
    n = (1 << 30) - 4099
    g = torch.Generator(device="cuda").manual_seed(0x51)
    keys = torch.randint(-(1 << 31), 1 << 31, (n,), dtype=torch.int32, device="cuda", generator=g)
    keys[: n // 8] &= 0xFFFF  # an eighth of the keys below 2^16: long runs of equal keys
    ko, perm = bcf.sort(keys, None, index_payload=True)
    assert bcf.get_status() == bcf.OK
    s = ko ^ torch.tensor(-(1 << 31), dtype=torch.int32, device="cuda")  # uint32 order as int32 order
    assert bool((s[1:] >= s[:-1]).all())
    assert bool((perm >= 0).all()) and bool((perm < n).all())
    seen = torch.zeros(n, dtype=torch.uint8, device="cuda")
    seen[perm.long()] = 1
    assert bool(seen.all())  # n indices, every one hit: a permutation
    del seen
    assert torch.equal(keys[perm.long()], ko)
    tie = s[1:] == s[:-1]
    assert bool((perm[1:][tie] > perm[:-1][tie]).all())


@pytest.mark.slow
def test_partition_largest_size_by_properties(bcf):
    """A 256-way partition of 2^30 - 4099 labels with index payloads (n < 2^30, the
    largest the library takes), checked by the properties that make a stable
    partition unique: labels non-decreasing, payloads a permutation that carries
    every label from its input position, equal labels in input order."""
    import torch
    n = (1 << 30) - 4099
    g = torch.Generator(device="cuda").manual_seed(0x52)
    keys = torch.randint(0, 256, (n,), dtype=torch.int32, device="cuda", generator=g)
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    ko, perm = bcf.partition(keys, idx, 256)
    assert bcf.get_status() == bcf.OK
    assert bool((ko[1:] >= ko[:-1]).all())
    seen = torch.zeros(n, dtype=torch.uint8, device="cuda")
    seen[perm.long()] = 1
    assert bool(seen.all())
    del seen
    assert torch.equal(keys[perm.long()], ko)
    tie = ko[1:] == ko[:-1]
    assert bool((perm[1:][tie] > perm[:-1][tie]).all())
