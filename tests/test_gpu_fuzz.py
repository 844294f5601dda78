"""GPU parity over many seeded random configurations: sizes from 0 to a few hundred
thousand (both sides of the single-launch limit and of every tile size), key
widths, payload widths, balanced and unbalanced partitions (sweep, Lemma 1 tiles,
direct write-out), splitters, permutation forms and in-place calls -- each
compared bit-exact with the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu

N_CASES = 60


@pytest.fixture(scope="module")
def bcf():
    import paper_1507_01391_b300 as m
    m.lib()
    return m


def _payload(g, n, vb):
    if vb == 0:
        return None
    if vb == 4:
        return synth.float_bits_payload(n, seed=int(g.integers(1 << 30)))
    return synth.uniform_keys(2 * n, seed=int(g.integers(1 << 30))).view(np.uint64)


def _size(g):
    return int(g.choice([0, 1, 7, 1023, 1024, 4097, 70_000, 262_143, 262_144, 262_145, 400_000])
               if g.random() < 0.4 else g.integers(0, 300_000))


@pytest.mark.parametrize("case", range(N_CASES))
def test_fuzz_sort(bcf, case):
    g = synth.rng(1000 + case)
    n = _size(g)
    bits = int(g.integers(1, 33))
    vb = int(g.choice([0, 4, 8]))
    keys = synth.uniform_keys(n, seed=case, bits=bits) if g.random() < 0.7 else synth.random_labels(n, 3, seed=case)
    vals = _payload(g, n, vb)
    in_place = bool(g.random() < 0.3)
    kd, vd = dev(keys), (None if vals is None else dev(vals))
    if in_place:
        ko, vo = bcf.sort(kd, vd, key_bits=bits if keys.max(initial=0) < (1 << bits) else 32, keys_out=kd, vals_out=vd)
    else:
        ko, vo = bcf.sort(kd, vd, key_bits=bits if keys.max(initial=0) < (1 << bits) else 32)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


@pytest.mark.parametrize("case", range(N_CASES))
def test_fuzz_partition(bcf, case):
    g = synth.rng(2000 + case)
    w = int(g.integers(1, 257))
    n = _size(g)
    balanced = bool(g.random() < 0.5)
    if balanced:
        n -= n % w
        keys = synth.partition_keys(n, w, seed=case)
    else:
        keys = synth.random_labels(n, w, seed=case)
    vb = int(g.choice([0, 4, 8]))
    vals = _payload(g, n, vb)
    mode = g.choice(["sweep", "lemma1", "splitters", "direct"])
    if mode == "direct" and w > 32:  # the direct write-out serves at most 32 labels
        mode = "sweep"
    kd, vd = dev(keys), (None if vals is None else dev(vals))
    if mode == "splitters":
        spl = np.arange(1, w, dtype=np.uint32)  # bucket = label
        ko, vo = bcf.partition_splitters(kd, vd, dev(spl) if w > 1 else dev(np.zeros(4, np.uint32))[:0],
                                         balanced=balanced)
    else:
        flags = {"lemma1": bcf.PARTITION_LEMMA1, "direct": bcf.PARTITION_DIRECT}.get(mode, 0)
        ko, vo = bcf.partition(kd, vd, w, balanced=balanced, flags=flags)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=balanced)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


@pytest.mark.parametrize("case", range(N_CASES))
def test_fuzz_permute(bcf, case):
    g = synth.rng(3000 + case)
    n = _size(g)
    vb = int(g.choice([0, 4, 8]))
    keys = synth.uniform_keys(n, seed=case)
    vals = _payload(g, n, vb)
    pi = synth.random_perm(n, seed=case + 1)
    form = g.choice(["scatter", "fused", "bucketed"])
    check = bool(g.random() < 0.5)
    ko, vo = bcf.permute_kv(dev(keys), None if vals is None else dev(vals), dev(pi), check=check,
                            fused=form == "fused", bucketed=form == "bucketed")
    assert bcf.get_status() == bcf.OK
    assert bits_equal(host(ko, np.uint32), oracle.permute(keys, pi))
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), oracle.permute(vals, pi))
