"""GPU parity: Lemma 2's 0-1 partition of 1024 x 32 matrices through the C ABI,
bit-exact against the CPU oracle (labels and payloads, whose order Lemma 2's
steps fix), on several matrices per launch, structured and random labels, the
full 2^24-item workload (sampled matrices against the oracle, every matrix
against the partition's definition) and the error paths."""
import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu

W, M = 1024, 32
ITEMS = W * M


@pytest.fixture(scope="module")
def bcf():
    import paper_1507_01391_b300 as m
    m.lib()
    return m


def _matrix(a, t):
    """Matrix t of a linear array: item k in row k % W, column k // W."""
    return a[t * ITEMS:(t + 1) * ITEMS].reshape(M, W).T


def _expect(keys, vals, tiles=None):
    tiles = range(keys.size // ITEMS) if tiles is None else tiles
    out = {}
    for t in tiles:
        lo, po = oracle.lemma2_partition(_matrix(keys, t), _matrix(vals.view(np.uint32), t))
        out[t] = (lo.ravel(), po.ravel())
    return out


def _run(bcf, keys, vals, in_place=False, pass_vals=True):
    kd = dev(keys)
    vd = dev(vals) if pass_vals else None
    if in_place:
        ko, vo = bcf.partition_lemma2(kd, vd, keys_out=kd, vals_out=vd)
    else:
        ko, vo = bcf.partition_lemma2(kd, vd)
    assert bcf.get_status() == bcf.OK
    return host(ko, np.uint32), host(vo, vals.dtype)


def _check_all(bcf, keys, vals, **kw):
    ko, vo = _run(bcf, keys, vals, **kw)
    for t, (lo, po) in _expect(keys, vals).items():
        assert np.array_equal(ko[t * ITEMS:(t + 1) * ITEMS], lo), t
        assert bits_equal(vo[t * ITEMS:(t + 1) * ITEMS], po), t


@pytest.mark.parametrize("p", [0.0, 0.003, 0.3, 0.5, 0.97, 1.0])
def test_lemma2_random_labels(bcf, p):
    n = 3 * ITEMS
    _check_all(bcf, synth.bernoulli_labels(n, p, seed=int(p * 1000) + 1), synth.index_payload(n))


def _structured(kind, seed):
    r = np.arange(W)[:, None].repeat(M, 1)
    c = np.arange(M)[None, :].repeat(W, 0)
    if kind == "top_half_zero":
        lab = r >= W // 2
    elif kind == "exact_half":
        lab = synth.rng(seed).permutation(np.arange(ITEMS) % 2).reshape(W, M)
    elif kind == "alternating_rows":
        lab = r % 2
    elif kind == "alternating_columns":
        lab = c % 2
    elif kind == "one_zero_per_row":
        lab = c != r % M
    elif kind == "single_one":
        lab = (r == 333) & (c == 7)
    else:
        raise ValueError(kind)
    return lab.astype(np.uint32).T.ravel()  # the matrix laid out column-major


@pytest.mark.parametrize("kind", ["top_half_zero", "exact_half", "alternating_rows", "alternating_columns",
                                  "one_zero_per_row", "single_one"])
def test_lemma2_structured_labels(bcf, kind):
    keys = np.concatenate([_structured(kind, s) for s in (1, 2)])
    _check_all(bcf, keys, synth.index_payload(keys.size))


def test_lemma2_float_payload_bits(bcf):
    n = 2 * ITEMS
    _check_all(bcf, synth.bernoulli_labels(n, 0.4, seed=9), synth.float_bits_payload(n, seed=9))


def test_lemma2_position_payload(bcf):
    """vals NULL: every item carries its input position."""
    n = 2 * ITEMS
    keys = synth.bernoulli_labels(n, 0.6, seed=10)
    _check_all(bcf, keys, synth.index_payload(n), pass_vals=False)


def test_lemma2_in_place(bcf):
    n = 2 * ITEMS
    _check_all(bcf, synth.bernoulli_labels(n, 0.5, seed=11), synth.uniform_keys(n, seed=12), in_place=True)


def test_lemma2_full_size_workload(bcf):
    """2^24 items (512 matrices), the benchmark's launch: six sampled matrices
    bit-exact against the oracle; every matrix partitioned with its pairs kept."""
    n = 1 << 24
    keys = synth.bernoulli_labels(n, 0.5, seed=13)
    vals = synth.index_payload(n)
    ko, vo = _run(bcf, keys, vals)
    tiles = n // ITEMS
    sample = [0, 1, 77, 255, 400, tiles - 1]
    for t, (lo, po) in _expect(keys, vals, sample).items():
        assert np.array_equal(ko[t * ITEMS:(t + 1) * ITEMS], lo)
        assert np.array_equal(vo[t * ITEMS:(t + 1) * ITEMS], po)
    kt = ko.reshape(tiles, ITEMS)
    zeros = (keys.reshape(tiles, M, W) == 0).sum(axis=(1, 2))
    assert np.all(kt == (np.arange(ITEMS)[None, :] >= zeros[:, None]))
    # payloads: a permutation inside each matrix, each carrying its own label
    vt = vo.reshape(tiles, ITEMS).astype(np.int64)
    assert np.array_equal(np.sort(vt, axis=1), np.arange(n).reshape(tiles, ITEMS))
    assert np.array_equal(keys[vo], ko)


def test_lemma2_empty_and_bad_sizes(bcf):
    import torch
    z = torch.empty(0, dtype=torch.int32, device="cuda")
    bcf.partition_lemma2(z, z)
    k = torch.zeros(ITEMS + 4, dtype=torch.int32, device="cuda")
    with pytest.raises(bcf.BcfError) as e:
        bcf.partition_lemma2(k, k.clone())
    assert e.value.code == bcf.E_INVAL


def test_lemma2_bad_label_sets_status(bcf):
    keys = synth.bernoulli_labels(ITEMS, 0.5, seed=14)
    keys[12345] = 2
    kd = dev(keys)
    bcf.partition_lemma2(kd, dev(synth.index_payload(ITEMS)))
    assert bcf.get_status() == bcf.E_BAD_KEY
    assert bcf.get_status() == bcf.OK
