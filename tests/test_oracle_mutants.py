"""The pins must catch plausible oracle mistakes.  Each case copies the oracle's C
source to a temporary directory, plants one mistake there (a flipped comparison,
a swapped index, a dropped phase), compiles the copy and checks that a pin from
test_oracle_pins.py now fails.  The committed oracle is never modified.  CPU only."""
import os

import numpy as np
import pytest

import oracle
import synth

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "bcf_oracle.c")).read()


def _mutant(tmp_path, old, new):
    assert SRC.count(old) >= 1, old
    path = tmp_path / "mutant.c"
    path.write_text(SRC.replace(old, new, 1))
    so = str(tmp_path / "libmutant.so")
    oracle.build(str(path), so, force=True)
    return oracle.load(so)


def _sort_pins(L):
    # stability and order against Python's stable sort on a duplicate-heavy input
    keys = synth.random_labels(500, 4, seed=1)
    ko, vo = oracle.sort_kv(keys, synth.index_payload(500), L=L)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(vo, ref.astype(np.uint32))
    small = synth.random_labels(20, 3, seed=2)
    ko, vo = oracle.sort_kv(small, synth.index_payload(20), L=L)
    assert np.array_equal(vo, np.argsort(small, kind="stable").astype(np.uint32))


def _partition_pins(L):
    keys = synth.partition_keys(64, 4, seed=3)
    ko, vo = oracle.partition_kv(keys, synth.index_payload(64), 4, balanced=True, L=L)
    assert np.array_equal(ko, (np.arange(64) // 16).astype(np.uint32))
    for b in range(4):
        assert np.array_equal(vo[16 * b:16 * b + 16], np.flatnonzero(keys == b).astype(np.uint32))


def _splitter_pins(L):
    keys = np.array([5, 1, 9, 5, 3, 7, 5, 2], dtype=np.uint32)
    ko, vo = oracle.partition_splitters(keys, synth.index_payload(8), np.array([5, 5, 8], dtype=np.uint32), L=L)
    assert ko.tolist() == [1, 3, 2, 5, 5, 7, 5, 9] and vo.tolist() == [1, 4, 7, 0, 3, 5, 6, 2]


def _permute_pins(L):
    pi = synth.random_perm(50, seed=4)
    inv = oracle.permute(synth.index_payload(50), pi, L=L)
    assert np.array_equal(inv, np.argsort(pi).astype(np.uint32))


def _lemma1_pins(L):
    g = synth.rng(5)
    for _ in range(200):
        M = g.integers(0, 2, size=(3, 9), dtype=np.uint32)
        out = oracle.lemma1_sort(M, L=L)
        assert np.all(np.diff(out.reshape(-1).astype(np.int64)) >= 0)


def _bank_pins(L):
    n = 32
    req = np.zeros(n, np.int64)
    lane = np.arange(n, dtype=np.int32)
    for width in (8, 16):
        addr = (np.arange(n) * width).astype(np.uint32)
        assert oracle.bank_count(req, lane, addr, np.full(n, width, np.int32), L=L)[1] == 0
    addr = (np.arange(n) * 4 * 6).astype(np.uint32)  # runs of 6: gcd(6,32) = 2
    assert oracle.bank_count(req, lane, addr, np.full(n, 4, np.int32), L=L)[0] == 2
    same = np.full(n, 128, np.uint32)  # one word read by every lane: a broadcast
    assert oracle.bank_count(req, lane, same, np.full(n, 4, np.int32), L=L)[:2] == (1, 0)


def _lemma2_pins(L):
    g = synth.rng(7)
    w, m = 1024, 32
    pay = np.arange(w * m, dtype=np.uint32).reshape(w, m)
    cases = [(g.random((w, m)) < 0.3).astype(np.uint32), (np.arange(w)[:, None] >= w // 2).repeat(m, 1).astype(np.uint32)]
    for _ in range(6):  # exactly half zeros: the dirty rows sit at row w/2, a square boundary
        cases.append(g.permutation(np.arange(w * m) % 2).reshape(w, m).astype(np.uint32))
    for lab in cases:
        lo, po = oracle.lemma2_partition(lab, pay, L=L)
        assert np.all(np.diff(lo.ravel().astype(np.int64)) >= 0)
        assert sorted(zip(lab.ravel().tolist(), pay.ravel().tolist())) == sorted(zip(lo.ravel().tolist(), po.ravel().tolist()))
        l1, _ = oracle.lemma2_partition(lab, pay, stage=1, L=L)
        zeros = m - l1.sum(axis=1).astype(np.int64)
        w0 = int((lab == 0).sum())
        assert np.all(np.abs(zeros - w0 / w) <= 2)
    cm = np.arange(w * m, dtype=np.uint32).reshape(m, w).T.copy()
    _, po = oracle.lemma2_partition(np.zeros((w, m), np.uint32), cm, L=L)
    assert np.array_equal(po.ravel(), np.arange(w * m, dtype=np.uint32))


MUTANTS = [
    ("merge takes right run on ties", "if (src[j].key < src[i].key)", "if (src[j].key <= src[i].key)", _sort_pins),
    ("insertion sort moves past equal keys", "while (j >= 0 && a[j].key > x.key)", "while (j >= 0 && a[j].key >= x.key)", _sort_pins),
    ("merge copies a wrong right tail", "while (j < hi) dst[k++] = src[j++];", "while (j < hi) { dst[k++] = src[mid - 1]; j++; }", _sort_pins),
    ("partition scans backwards", "for (int64_t i = 0; i < n; ++i) {\n        int64_t p = count[keys[i]]++;",
     "for (int64_t i = n - 1; i >= 0; --i) {\n        int64_t p = count[keys[i]]++;", _partition_pins),
    ("splitter bucket counts splitters below, not at or below", "for (int64_t t = 0; t < nsplit; ++t) b += splitters[t] <= keys[i];",
     "for (int64_t t = 0; t < nsplit; ++t) b += splitters[t] < keys[i];", _splitter_pins),
    ("permute writes gather-style", "memcpy((char*)dst + (int64_t)pi[i] * elem_bytes, (const char*)src + i * elem_bytes,",
     "memcpy((char*)dst + i * elem_bytes, (const char*)src + (int64_t)pi[i] * elem_bytes,", _permute_pins),
    ("row->col conversion transposed", "for (int64_t r = 0; r < w; ++r) M[r * m + c] = seq[c * w + r];",
     "for (int64_t r = 0; r < w; ++r) M[r * m + c] = seq[r * m + c];", _lemma1_pins),
    ("Lemma 1 runs its loop once", "for (int rep = 0; rep < 2; ++rep) {", "for (int rep = 0; rep < 1; ++rep) {", _lemma1_pins),
    ("Lemma 2 balancing squares take contiguous rows", "for (int64_t t = 0; t < m; ++t) rows[t] = g * group + t * sub + j;",
     "for (int64_t t = 0; t < m; ++t) rows[t] = g * group + j * m + t;", _lemma2_pins),
    ("Lemma 2 skips the shifted squares", "for (int64_t r0 = m / 2; r0 + m <= w", "for (int64_t r0 = w; r0 + m <= w", _lemma2_pins),
    ("Lemma 2 step sort puts 1s first", "for (int label = 0; label <= 1; ++label)", "for (int label = 1; label >= 0; --label)", _lemma2_pins),
    ("Lemma 2 converts row to column", "for (int64_t r = 0; r < w; ++r) seq[c * w + r] = a[r * m + c];\n    memcpy(a, seq",
     "for (int64_t r = 0; r < w; ++r) seq[r * m + c] = a[c * w + r];\n    memcpy(a, seq", _lemma2_pins),
    ("bank model ignores phases", "int lanes_per_phase = 32 / words_per_lane;", "int lanes_per_phase = 32;", _bank_pins),
    ("bank model counts lanes not words", "if (words[bank][q] == word) dup = 1;", "if (0) dup = 1;", _bank_pins),
]


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new, pins):
    L = _mutant(tmp_path, old, new)
    with pytest.raises((AssertionError, oracle.OracleError)):
        pins(L)


def test_unmutated_copy_passes_the_same_pins(tmp_path):
    L = _mutant(tmp_path, "#include <stdlib.h>", "#include <stdlib.h>")
    for pins in (_sort_pins, _partition_pins, _splitter_pins, _permute_pins, _lemma1_pins, _lemma2_pins, _bank_pins):
        pins(L)
