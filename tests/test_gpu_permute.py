"""GPU parity: permutation scatter, gather and tile-local permutation through the C
ABI, bit-exact against the CPU oracle, including NaN / -0.0 payload bits, ragged
tails, the full-size 2^24 workload and the bad-permutation error path."""
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
    return m


@pytest.mark.parametrize("n", [1, 3, 4, 5, 31, 1000, 4097, 100_003])
def test_permute_kv_float_payload(bcf, n):
    keys = synth.uniform_keys(n, seed=n)
    vals = synth.float_bits_payload(n, seed=n + 1)
    pi = synth.random_perm(n, seed=n + 2)
    ko, vo = bcf.permute_kv(dev(keys), dev(vals), dev(pi), check=True)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))
    assert bits_equal(host(vo, np.float32), oracle.permute(vals, pi))


@pytest.mark.parametrize("n", [7, 4096, 65_537])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_permute_and_gather_elements(bcf, n, dtype):
    x = synth.uniform_keys(n * (np.dtype(dtype).itemsize // 4), seed=3).view(dtype)
    pi = synth.random_perm(n, seed=4)
    y = bcf.permute(dev(x), dev(pi))
    assert bits_equal(host(y, dtype), oracle.permute(x, pi))
    z = bcf.gather(y, dev(pi))
    assert bits_equal(host(z, dtype), oracle.gather(oracle.permute(x, pi), pi))
    assert bits_equal(host(z, dtype), x)
    assert bcf.get_status() == bcf.OK


def test_permute_keys_only(bcf):
    n = 12_345
    keys = synth.uniform_keys(n, seed=8)
    pi = synth.random_perm(n, seed=9)
    ko, vo = bcf.permute_kv(dev(keys), None, dev(pi))
    assert vo is None
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))


@pytest.mark.slow
def test_permute_full_size_2pow24(bcf):
    n = 1 << 24
    keys = synth.uniform_keys(n, seed=0x1A)
    vals = synth.float_bits_payload(n, seed=0x1B)
    pi = synth.random_perm(n, seed=0x1C)
    ko, vo = bcf.permute_kv(dev(keys), dev(vals), dev(pi))
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))
    assert bits_equal(host(vo, np.float32), oracle.permute(vals, pi))


def test_permute_reports_non_bijection(bcf):
    n = 1000
    pi = synth.random_perm(n, seed=1)
    pi[10] = pi[11]
    bcf.permute(dev(synth.uniform_keys(n, seed=2)), dev(pi), check=True)
    assert bcf.get_status() == bcf.E_BAD_PERM
    pi = synth.random_perm(n, seed=1)
    pi[3] = n + 5  # out of range: never written, always reported
    bcf.permute(dev(synth.uniform_keys(n, seed=2)), dev(pi))
    assert bcf.get_status() == bcf.E_BAD_PERM


def test_gather_reports_out_of_range(bcf):
    idx = np.array([0, 1, 99, 2], dtype=np.uint32)
    bcf.gather(dev(np.arange(4, dtype=np.uint32)), dev(idx))
    assert bcf.get_status() == bcf.E_BAD_PERM


# ------------------------------------------------------------ tile-local
SCHEDULES = [(False, "greedy"), (True, "greedy"), (True, "sorted")]


@pytest.mark.parametrize("coloured,finish", SCHEDULES)
@pytest.mark.parametrize("tile", [1024, 2048, 4096])
@pytest.mark.parametrize("n_tiles,extra", [(1, 0), (3, 0), (5, 77), (0, 33)])
def test_permute_tiles(bcf, coloured, finish, tile, n_tiles, extra):
    n = n_tiles * tile + extra
    src = synth.uniform_keys(n, seed=n + tile)
    lpi = synth.tile_local_perms(n, tile, seed=n)
    out = bcf.permute_tiles(dev(src), dev(lpi), tile=tile, coloured=coloured, finish=finish)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(out, np.uint32), oracle.permute_tiles(src, lpi, tile))


@pytest.mark.parametrize("coloured,finish", SCHEDULES)
def test_permute_tiles_structured(bcf, coloured, finish):
    """Adversarial labels for the colouring: identity, reversal, a transpose of
    the 32 x 128 bank matrix (every row sends all its items to one bank), and all
    items of a row aimed at one slot column."""
    tile, m = 4096, 128
    q = np.arange(tile)
    cases = [q, q[::-1], (q % 32) * m + q // 32, ((q % 32) * 32 + (q // 32) % 32 + 1024 * ((q // 32) // 32)) % tile]
    for lab in cases:
        lpi = np.asarray(lab, dtype=np.uint16)
        assert len(np.unique(lpi)) == tile
        src = synth.uniform_keys(tile, seed=5)
        out = bcf.permute_tiles(dev(src), dev(lpi), tile=tile, coloured=coloured, seed=123, finish=finish)
        assert bits_equal(host(out, np.uint32), oracle.permute_tiles(src, lpi, tile))
    assert bcf.get_status() == bcf.OK


@pytest.mark.slow
@pytest.mark.parametrize("coloured,finish", SCHEDULES)
def test_permute_tiles_full_size(bcf, coloured, finish):
    n, tile = 1 << 24, 4096
    src = synth.uniform_keys(n, seed=0x1D)
    lpi = synth.tile_local_perms(n, tile, seed=0x1E)
    out = bcf.permute_tiles(dev(src), dev(lpi), tile=tile, coloured=coloured, finish=finish)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(out, np.uint32), oracle.permute_tiles(src, lpi, tile))


def test_permute_tiles_reports_bad_label(bcf):
    tile = 1024
    lpi = synth.tile_local_perms(tile + 100, tile, seed=1)
    lpi[tile + 5] = 500  # outside the 100-item ragged tile
    for coloured, finish in SCHEDULES:
        bcf.permute_tiles(dev(synth.uniform_keys(tile + 100, seed=2)), dev(lpi), tile=tile, coloured=coloured,
                          finish=finish)
        assert bcf.get_status() == bcf.E_BAD_PERM


# ------------------------------------------------------------ bucketed form
# Two coalesced passes: group by destination block (4096 to 53248 positions,
# sized so that the blocks fill whole waves of SMs), then place each block in
# shared memory.  Sizes span several 8192-element tiles and blocks and end in
# ragged tails (n not a multiple of 4, 8 or 8192).
BLOCK = 1 << 15


@pytest.mark.parametrize("n", [1, 5, 8191, 8192, 8193, BLOCK - 3, BLOCK, BLOCK + 1, 3 * BLOCK + 4099, 300_001])
@pytest.mark.parametrize("with_vals", [False, True])
def test_permute_bucketed(bcf, n, with_vals):
    keys = synth.uniform_keys(n, seed=n + 11)
    vals = synth.float_bits_payload(n, seed=n + 12)
    pi = synth.random_perm(n, seed=n + 13)
    if with_vals:
        ko, vo = bcf.permute_kv(dev(keys), dev(vals), dev(pi), bucketed=True)
        assert bits_equal(host(vo, np.float32), oracle.permute(vals, pi))
    else:
        ko = bcf.permute(dev(keys), dev(pi), bucketed=True)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))


@pytest.mark.parametrize("kind", ["identity", "reverse", "rotate", "transpose", "one_block_per_tile"])
def test_permute_bucketed_structured(bcf, kind):
    """Permutations that load blocks unevenly over time: the identity sends every
    tile to one block, a transpose sends consecutive elements to far-apart blocks."""
    n = 5 * BLOCK + 128
    i = np.arange(n, dtype=np.int64)
    if kind == "identity":
        pi = i
    elif kind == "reverse":
        pi = n - 1 - i
    elif kind == "rotate":
        pi = (i + 12_345) % n
    elif kind == "transpose":  # n = 64 * (n // 64): i = r * 64 + c -> c * (n // 64) + r
        pi = (i % 64) * (n // 64) + i // 64
    else:  # tile t of 8192 elements -> block (t * 7) mod blocks, shuffled inside
        pi = synth.random_perm(n, seed=3).astype(np.int64)
        pi = np.sort(pi)[np.argsort(np.argsort((i // 8192 * 7919 + i % 8192) % n, kind="stable"), kind="stable")]
    pi = pi.astype(np.uint32)
    assert len(np.unique(pi)) == n
    keys = synth.uniform_keys(n, seed=4)
    vals = synth.float_bits_payload(n, seed=5)
    ko, vo = bcf.permute_kv(dev(keys), dev(vals), dev(pi), bucketed=True, check=True)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))
    assert bits_equal(host(vo, np.float32), oracle.permute(vals, pi))


def test_permute_bucketed_rows(bcf):
    """Row-local permutations (row_len > 0) through the bucketed form."""
    rows, row_len = 6, 70_001
    n = rows * row_len
    pi = np.concatenate([synth.random_perm(row_len, seed=r) for r in range(rows)])
    keys = synth.uniform_keys(n, seed=7)
    vals = synth.float_bits_payload(n, seed=8)
    ko, vo = bcf.permute_kv(dev(keys), dev(vals), dev(pi), row_len=row_len, bucketed=True)
    assert bcf.get_status() == bcf.OK
    glob = (np.arange(n) // row_len * row_len + pi).astype(np.uint32)
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, glob))
    assert bits_equal(host(vo, np.float32), oracle.permute(vals, glob))


def test_permute_bucketed_more_than_512_blocks(bcf):
    """Above 512 destination blocks (740 blocks of 45344 on 148 SMs) the pass-1
    kernel keeps 2048 block counters."""
    n = (1 << 25) + 7
    keys = synth.uniform_keys(n, seed=9)
    pi = synth.random_perm(n, seed=10)
    ko = bcf.permute(dev(keys), dev(pi), bucketed=True)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))


@pytest.mark.parametrize("n", [3 * BLOCK + 5, (1 << 22) + 3])  # blocks of 4096; of 28,344 (148 SMs)
def test_permute_bucketed_reports_non_bijection(bcf, n):
    keys = dev(synth.uniform_keys(n, seed=2))
    for a, b in [(10, 11), (7, 3 * BLOCK)]:  # same block; different blocks (one over-full)
        pi = synth.random_perm(n, seed=1)
        pi[a] = pi[b]
        bcf.permute(keys, dev(pi), check=True, bucketed=True)
        assert bcf.get_status() == bcf.E_BAD_PERM
    pi = synth.random_perm(n, seed=1)
    pi[3] = n + 5  # out of range: never written, always reported
    bcf.permute(keys, dev(pi), bucketed=True)
    assert bcf.get_status() == bcf.E_BAD_PERM


def test_permute_bucketed_not_applicable_runs_scatter(bcf):
    """8-byte payloads are outside the bucketed form: the flag falls back to the
    one-pass scatter and the result is the same."""
    n = 50_000
    keys = synth.uniform_keys(n, seed=1)
    vals = synth.uniform_keys(2 * n, seed=2).view(np.uint64)
    pi = synth.random_perm(n, seed=3)
    ko, vo = bcf.permute_kv(dev(keys), dev(vals), dev(pi), bucketed=True)
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))
    assert bits_equal(host(vo, np.uint64), oracle.permute(vals, pi))
