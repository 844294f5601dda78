"""Pins for the CPU oracle: each function is checked against something other than
itself -- brute force over every input of tiny sizes, closed forms the paper
states, invariants that determine the answer uniquely, and library routines
(numpy's stable argsort, Python's sorted) for special cases.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import synth


# ----------------------------------------------------------------- sorting ----
def _stable_sorted_order(keys):
    # Python's sort is documented to be stable: an independent reference.
    return sorted(range(len(keys)), key=lambda i: keys[i])


def test_sort_bruteforce_all_sequences_n8(orc):
    """Every key sequence of length 8 over {0,1,2,3} (4^8 = 65536 inputs), with
    payload = original index: keys ascending and equal keys in input order."""
    L = orc.lib()
    idx = np.arange(8, dtype=np.uint32)
    for seq in itertools.product(range(4), repeat=8):
        keys = np.array(seq, dtype=np.uint32)
        ko, vo = orc.sort_kv(keys, idx, L=L)
        order = _stable_sorted_order(seq)
        assert vo.tolist() == order
        assert ko.tolist() == [seq[i] for i in order]


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 63, 64, 65, 1000, 4097, 100_003])
@pytest.mark.parametrize("kind", ["uniform", "few", "zipf"])
def test_sort_matches_numpy_stable(orc, n, kind):
    if kind == "uniform":
        keys = synth.uniform_keys(n, seed=n + 1)
    elif kind == "few":
        keys = synth.random_labels(n, 5, seed=n + 2)
    else:
        keys = synth.zipf_keys(n, seed=n + 3)
    vals = synth.index_payload(n)
    ko, vo = orc.sort_kv(keys, vals)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(vo, ref.astype(np.uint32))
    assert np.array_equal(ko, keys[ref])


def test_sort_special_cases(orc):
    n = 5000
    # all keys equal -> identity
    keys = np.full(n, 7, dtype=np.uint32)
    ko, vo = orc.sort_kv(keys, synth.index_payload(n))
    assert np.array_equal(vo, np.arange(n, dtype=np.uint32))
    # keys form a permutation of [n] -> keys become 0..n-1, payload the inverse
    pi = synth.random_perm(n, seed=11)
    ko, vo = orc.sort_kv(pi, synth.index_payload(n))
    assert np.array_equal(ko, np.arange(n, dtype=np.uint32))
    assert np.array_equal(pi[vo], np.arange(n, dtype=np.uint32))
    # reverse-sorted input with duplicates
    keys = np.repeat(np.arange(100, 0, -1, dtype=np.uint32), 30)
    ko, vo = orc.sort_kv(keys, synth.index_payload(keys.size))
    assert np.all(np.diff(ko.astype(np.int64)) >= 0)


def test_sort_payload_bits_and_widths(orc):
    n = 3000
    keys = synth.random_labels(n, 17, seed=5)
    f = synth.float_bits_payload(n, seed=6)  # NaN / -0.0 patterns included
    ko, vo = orc.sort_kv(keys, f)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(vo.view(np.uint32), f.view(np.uint32)[ref])
    v8 = np.arange(n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    ko, vo = orc.sort_kv(keys, v8)
    assert np.array_equal(vo, v8[ref])
    ko, vo = orc.sort_kv(keys, None)
    assert vo is None and np.array_equal(ko, keys[ref])


def test_stable_rank_is_sorted_position(orc):
    keys = synth.random_labels(777, 9, seed=3)
    ko, vo = orc.sort_kv(keys, synth.index_payload(keys.size))
    for p in range(0, 777, 37):
        assert orc.stable_rank(keys, int(vo[p])) == p


# --------------------------------------------------------------- partition ----
def _check_partition_closed_form(ko, vo, keys, w):
    """Partition problem: exactly m = n/w copies of each label, so label b fills
    positions [b*m, (b+1)*m) -- key_out[p] = floor(p/m); the payload (original
    index) of bucket b lists the positions of label b in increasing order."""
    n = keys.size
    m = n // w
    assert np.array_equal(ko, (np.arange(n) // m).astype(np.uint32))
    for b in range(w):
        assert np.array_equal(vo[b * m:(b + 1) * m], np.flatnonzero(keys == b).astype(np.uint32))


def _multiset_arrangements(counts):
    """Every distinct sequence holding counts[b] copies of label b."""
    total = sum(counts)
    if total == 0:
        yield ()
        return
    for b, c in enumerate(counts):
        if c:
            counts[b] -= 1
            for rest in _multiset_arrangements(counts):
                yield (b,) + rest
            counts[b] += 1


@pytest.mark.parametrize("w,m", [(2, 4), (4, 2), (3, 3), (2, 8)])
def test_partition_bruteforce_all_arrangements(orc, w, m):
    L = orc.lib()
    seen = set()
    for arr in _multiset_arrangements([m] * w):
        seen.add(arr)
        keys = np.array(arr, dtype=np.uint32)
        ko, vo = orc.partition_kv(keys, synth.index_payload(keys.size), w, balanced=True, L=L)
        _check_partition_closed_form(ko, vo, keys, w)
    assert len(seen) == math.factorial(w * m) // math.factorial(m) ** w


@pytest.mark.parametrize("n,w", [(65536, 32), (1 << 16, 256), (4096, 1), (99, 3)])
def test_partition_balanced_closed_form(orc, n, w):
    keys = synth.partition_keys(n, w, seed=n + w)
    ko, vo = orc.partition_kv(keys, synth.index_payload(n), w, balanced=True)
    _check_partition_closed_form(ko, vo, keys, w)


def test_partition_unbalanced_and_errors(orc):
    keys = synth.random_labels(10_000, 37, seed=1)
    ko, vo = orc.partition_kv(keys, synth.index_payload(keys.size), 37)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(vo, ref.astype(np.uint32)) and np.array_equal(ko, keys[ref])
    with pytest.raises(orc.OracleError):
        orc.partition_kv(keys, None, 36)  # a label equals w
    with pytest.raises(orc.OracleError):
        orc.partition_kv(keys[:370], None, 37, balanced=True)  # counts are not n/w
    with pytest.raises(orc.OracleError):
        orc.partition_kv(keys[:100], None, 37, balanced=True)  # n % w != 0


# ------------------------------------------------------ splitter partition ----
def _bisect_order(keys, spl):
    # bucket = number of splitters <= key (bisect_right, a library routine), then
    # Python's stable sort by bucket
    import bisect
    lab = [bisect.bisect_right(list(spl), int(k)) for k in keys]
    return sorted(range(len(keys)), key=lambda i: lab[i]), lab


@pytest.mark.parametrize("nsplit", [0, 1, 5, 255])
def test_partition_splitters_against_bisect(orc, nsplit):
    n = 3000
    g = synth.rng(nsplit + 7)
    keys = g.integers(0, 1 << 12, size=n, dtype=np.uint32)
    spl = np.sort(g.integers(0, 1 << 12, size=nsplit, dtype=np.uint32))
    if nsplit:
        keys[:nsplit] = spl  # keys equal to splitters sit in the upper bucket
    order, lab = _bisect_order(keys, spl)
    ko, vo = orc.partition_splitters(keys, synth.index_payload(n), spl)
    assert np.array_equal(vo, np.asarray(order, dtype=np.uint32))
    assert np.array_equal(ko, keys[order])
    # every key lies in its bucket's range [s[b-1], s[b])
    labs = np.asarray(lab)[order]
    assert np.all(np.diff(labs) >= 0)
    for b in np.unique(labs):
        kb = ko[labs == b].astype(np.int64)
        if b > 0:
            assert kb.min() >= int(spl[b - 1])
        if b < nsplit:
            assert kb.max() < int(spl[b])


def test_partition_splitters_reduces_to_label_partition(orc):
    """Splitters 1..w-1 on keys in [0, w): the bucket is the key itself."""
    w, n = 37, 5000
    keys = synth.random_labels(n, w, seed=9)
    spl = np.arange(1, w, dtype=np.uint32)
    ko, vo = orc.partition_splitters(keys, synth.index_payload(n), spl)
    rk, rv = orc.partition_kv(keys, synth.index_payload(n), w)
    assert np.array_equal(ko, rk) and np.array_equal(vo, rv)


def test_partition_splitters_duplicates_balanced_and_errors(orc):
    keys = np.array([5, 1, 9, 5, 3, 7, 5, 2], dtype=np.uint32)
    ko, vo = orc.partition_splitters(keys, synth.index_payload(8), np.array([5, 5, 8], dtype=np.uint32))
    # buckets: [<5] = 1,3,2 ; [5,5) empty ; [5,8) = 5,5,7,5 ; [>=8] = 9
    assert ko.tolist() == [1, 3, 2, 5, 5, 7, 5, 9] and vo.tolist() == [1, 4, 7, 0, 3, 5, 6, 2]
    bal = np.array([8, 1, 9, 2, 7, 3, 6, 0], dtype=np.uint32)
    ko, _ = orc.partition_splitters(bal, None, np.array([5], dtype=np.uint32), balanced=True)
    assert ko.tolist() == [1, 2, 3, 0, 8, 9, 7, 6]
    with pytest.raises(orc.OracleError):
        orc.partition_splitters(bal, None, np.array([3], dtype=np.uint32), balanced=True)  # 3 vs 5
    with pytest.raises(orc.OracleError):
        orc.partition_splitters(keys, None, np.array([6, 2], dtype=np.uint32))  # descending


# ------------------------------------------------------------- permutation ----
def test_permute_all_permutations_n8(orc):
    """For every pi of [8]: permuting the index array yields pi^-1, which numpy's
    argsort of pi also yields; permuting then gathering by pi is the identity."""
    L = orc.lib()
    x = np.arange(100, 108, dtype=np.uint32)
    iota = np.arange(8, dtype=np.uint32)
    for p in itertools.permutations(range(8)):
        pi = np.array(p, dtype=np.uint32)
        inv = orc.permute(iota, pi, L=L)
        assert np.array_equal(inv, np.argsort(pi).astype(np.uint32))
        y = orc.permute(x, pi, L=L)
        assert np.array_equal(orc.gather(y, pi, L=L), x)


@pytest.mark.parametrize("n", [0, 1, 33, 4096, 1 << 20])
def test_permute_invariants(orc, n):
    pi = synth.random_perm(n, seed=n + 9)
    iota = synth.index_payload(n)
    inv = orc.permute(iota, pi)
    assert np.array_equal(inv, np.argsort(pi, kind="stable").astype(np.uint32))
    f = synth.float_bits_payload(n, seed=4)
    y = orc.permute(f, pi)
    assert np.array_equal(orc.gather(y, pi).view(np.uint32), f.view(np.uint32))
    # composing with the inverse gives the identity permutation
    assert np.array_equal(orc.permute(orc.permute(iota, pi), inv), iota)


def test_permute_rejects_non_bijection(orc):
    pi = np.array([0, 1, 1, 3], dtype=np.uint32)
    with pytest.raises(orc.OracleError):
        orc.permute(np.zeros(4, np.uint32), pi)
    with pytest.raises(orc.OracleError):
        orc.permute(np.zeros(4, np.uint32), np.array([0, 1, 2, 4], dtype=np.uint32))
    with pytest.raises(orc.OracleError):
        orc.gather(np.zeros(4, np.uint32), np.array([0, 9], dtype=np.uint32))


@pytest.mark.parametrize("n,tile", [(4096 * 3, 4096), (4096 * 2 + 1000, 4096), (50, 16), (7, 4096)])
def test_permute_tiles_matches_global_permute(orc, n, tile):
    lpi = synth.tile_local_perms(n, tile, seed=n)
    src = synth.uniform_keys(n, seed=1)
    tiles = np.arange(n, dtype=np.int64) // tile
    gpi = (tiles * tile + lpi.astype(np.int64)).astype(np.uint32)
    assert np.array_equal(orc.permute_tiles(src, lpi, tile), orc.permute(src, gpi))
    ident = (np.arange(n) % tile).astype(np.uint16)
    assert np.array_equal(orc.permute_tiles(src, ident, tile), src)
    bad = lpi.copy()
    bad[0] = bad[1]
    with pytest.raises(orc.OracleError):
        orc.permute_tiles(src, bad, tile)


# ---------------------------------------------------------------- segmented ----
def test_segmented_sort_per_segment(orc):
    sizes = [0, 1, 5, 0, 300, 1024, 33, 0]
    offs = synth.offsets_from_sizes(sizes)
    keys = synth.random_labels(int(offs[-1]), 50, seed=2)
    vals = synth.index_payload(keys.size)
    ko, vo = orc.segmented_sort_kv(keys, vals, offs)
    for s in range(len(sizes)):
        lo, hi = offs[s], offs[s + 1]
        ref = lo + np.argsort(keys[lo:hi], kind="stable")
        assert np.array_equal(vo[lo:hi], ref.astype(np.uint32))


def test_segmented_partition_closed_form(orc):
    keys, offs, w = synth.segmented_partition_input(12, seed=5, hi_log2=11)
    vals = synth.index_payload(keys.size)
    ko, vo = orc.segmented_partition_kv(keys, vals, offs, w, balanced=True)
    for s in range(w.size):
        lo, hi = int(offs[s]), int(offs[s + 1])
        _check_partition_closed_form(ko[lo:hi], vo[lo:hi] - lo, keys[lo:hi], int(w[s]))


# ------------------------------------------------------------ Lemma 1 model ----
def _dirty_rows(M):
    return int(sum(1 for r in M if 0 < r.sum() < r.size))


def _dirty_cols(M):
    return _dirty_rows(M.T)


def _dirty_row_indices(M):
    return [i for i, r in enumerate(M) if 0 < r.sum() < r.size]


def _lemma1_with_dirt(orc, M, L):
    """Run Lemma 1 step by step on a 0-1 matrix and assert the dirty-row and
    dirty-column bounds used in its proof (Sec. 2, proof of Lemma 1)."""
    w, m = M.shape
    oracle = orc
    oracle.l1_sort_rows(M, True, L=L)
    oracle.l1_row_to_col(M, L=L)
    assert _dirty_cols(M) <= w               # at most w dirty columns
    oracle.l1_sort_rows(M, False, L=L)
    oracle.l1_col_to_row(M, L=L)
    d = _dirty_row_indices(M)
    assert len(d) <= 2                        # two dirty rows ...
    if len(d) == 2:
        assert d[1] == d[0] + 1               # ... and they are adjacent
    oracle.l1_sort_rows(M, True, L=L)
    oracle.l1_row_to_col(M, L=L)
    assert _dirty_cols(M) <= 2
    oracle.l1_sort_rows(M, False, L=L)
    assert _dirty_cols(M) <= 1                # one dirty column after step 3
    oracle.l1_col_to_row(M, L=L)
    assert _dirty_rows(M) <= 1                # one dirty row after step 4
    oracle.l1_sort_rows(M, False, L=L)
    flat = M.reshape(-1)
    assert np.all(np.diff(flat.astype(np.int64)) >= 0)


def test_lemma1_zero_one_exhaustive_2x4(orc):
    L = orc.lib()
    for bits in range(1 << 8):
        M = np.array([(bits >> k) & 1 for k in range(8)], dtype=np.uint32).reshape(2, 4)
        _lemma1_with_dirt(orc, M.copy(), L)


@pytest.mark.parametrize("w,m", [(3, 9), (4, 16), (2, 6), (3, 12)])
def test_lemma1_zero_one_sampled(orc, w, m):
    L = orc.lib()
    g = synth.rng(w * 100 + m)
    for _ in range(3000):
        M = g.integers(0, 2, size=(w, m), dtype=np.uint32)
        # bias toward few ones / few zeros, where dirt concentrates
        if _ % 3 == 1:
            M = (g.random((w, m)) < 0.1).astype(np.uint32)
        elif _ % 3 == 2:
            M = (g.random((w, m)) < 0.9).astype(np.uint32)
        _lemma1_with_dirt(orc, np.ascontiguousarray(M), L)


def test_lemma1_all_permutations_2x4(orc):
    L = orc.lib()
    for p in itertools.permutations(range(8)):
        M = np.array(p, dtype=np.uint32).reshape(2, 4)
        out = orc.lemma1_sort(M, L=L)
        assert out.reshape(-1).tolist() == list(range(8))


@pytest.mark.parametrize("w,m", [(4, 16), (8, 64), (16, 256), (32, 1024)])
def test_lemma1_sorts_random_matrices(orc, w, m):
    g = synth.rng(w)
    M = g.integers(0, 1000, size=(w, m), dtype=np.uint32)
    out = orc.lemma1_sort(M)
    assert np.array_equal(out.reshape(-1), np.sort(M.reshape(-1)))


# --------------------------------------------------------------- bank model ----
def _request(addrs, width=4):
    n = len(addrs)
    return (np.zeros(n, np.int64), np.arange(n, dtype=np.int32),
            np.array(addrs, dtype=np.uint32), np.full(n, width, np.int32))


def test_bank_strided_access_is_conflict_free(orc):
    """Strided access A[w*i + t] keeps lane t in bank t (Sec. 1): no conflicts."""
    for i in range(5):
        wf, hw, strict = orc.bank_count(*_request([4 * (32 * i + t) for t in range(32)]))
        assert (wf, hw, strict) == (1, 0, 0)


@pytest.mark.parametrize("s", list(range(1, 70)))
def test_bank_contiguous_runs_gcd(orc, s):
    """Contiguous runs of s words per lane: lane t reads word t*s + i.  The number
    of lanes sharing a bank is gcd(s, 32), so runs are conflict-free exactly when
    s is co-prime to 32 (Sec. 1, the padding remark)."""
    for i in (0, 3):
        wf, hw, strict = orc.bank_count(*_request([4 * (t * s + i) for t in range(32)]))
        g = math.gcd(s, 32)
        assert wf == g and hw == g - 1 and strict == g - 1


def test_bank_broadcast_and_wide_accesses(orc):
    # every lane reads one word: the hardware broadcasts; the strict model does not
    assert orc.bank_count(*_request([64] * 32)) == (1, 0, 31)
    # 8-byte consecutive accesses: two half-warp phases, no conflict
    assert orc.bank_count(*_request([8 * t for t in range(32)], 8)) == (2, 0, 1)
    # 16-byte consecutive accesses: four quarter-warp phases, no conflict
    assert orc.bank_count(*_request([16 * t for t in range(32)], 16)) == (4, 0, 3)
    # 8-byte accesses at a 16-byte stride: each half-warp hits every used bank twice
    wf, hw, _ = orc.bank_count(*_request([16 * t for t in range(32)], 8))
    assert wf == 4 and hw == 2
    # two requests are counted separately
    req, lane, addr, width = _request([4 * 32 * t for t in range(32)])
    req2 = np.concatenate([req, req + 1])
    res = orc.bank_count(req2, np.concatenate([lane, lane]),
                         np.concatenate([addr, addr]), np.concatenate([width, width]))
    assert res == (64, 62, 62)


# ------------------------------------------------------- Theorem 1 (Sec. 2) ----
def _contiguous(rows):
    return len(rows) == 0 or rows[-1] - rows[0] + 1 == len(rows)


def _theorem1_steps_hold(orc, M):
    """Dirty-row bounds of the proof of Theorem 1 on a 0-1 matrix: at most one
    dirty row per super-row after the first step; dirty rows contiguous once the
    columns are sorted; at most two after the alternating super-row sorts; one
    after the next column sort; none at the end."""
    m = M.shape[0]
    r = int(round(m ** 0.5))
    rec = []
    out = orc.theorem1_sort(M, record=rec)
    s1, s2, s3, s4, s5 = rec
    for g in range(r):
        assert _dirty_rows(s1[g * r:(g + 1) * r]) <= 1
    assert _dirty_rows(s1) <= r
    assert _contiguous(_dirty_row_indices(s2))
    assert _dirty_rows(s3) <= 2
    assert _dirty_rows(s4) <= 1
    assert np.all(np.diff(s5.reshape(-1).astype(np.int64)) >= 0)
    return out


def test_theorem1_zero_one_exhaustive_4x4(orc):
    for bits in range(1 << 16):
        M = ((bits >> np.arange(16)) & 1).astype(np.uint32).reshape(4, 4)
        _theorem1_steps_hold(orc, M)


def test_theorem1_zero_one_sampled_9x9(orc):
    g = synth.rng(91)
    for _ in range(3000):
        M = (g.random((9, 9)) < g.random()).astype(np.uint32)
        _theorem1_steps_hold(orc, M)


@pytest.mark.parametrize("m", [4, 9, 16])
def test_theorem1_sorts_random_matrices(orc, m):
    g = synth.rng(m)
    for _ in range(200):
        M = g.integers(0, 1000, size=(m, m), dtype=np.uint32)
        out = orc.theorem1_sort(M)
        assert np.array_equal(out.reshape(-1), np.sort(M.reshape(-1)))


def test_theorem1_rejects_other_shapes(orc):
    with pytest.raises(orc.OracleError):
        orc.theorem1_sort(np.zeros((4, 8), np.uint32))
    with pytest.raises(orc.OracleError):
        orc.theorem1_sort(np.zeros((5, 5), np.uint32))


def test_corollary1_partition_small_alphabets(orc):
    """Corollary 1: with w <= sqrt(m), Lemma 1 partitions a matrix of labels (the
    row sorts then only order labels, the radix-sort case).  Every 2 x 4 matrix
    over labels {0, 1, 2} and sampled 3 x 9 ones end partitioned."""
    for code in range(3 ** 8):
        M = np.array([(code // 3 ** k) % 3 for k in range(8)], dtype=np.uint32).reshape(2, 4)
        out = orc.lemma1_sort(M)
        assert np.array_equal(out.reshape(-1), np.sort(M.reshape(-1)))
    g = synth.rng(39)
    for _ in range(2000):
        M = g.integers(0, 3, size=(3, 9), dtype=np.uint32)
        assert np.array_equal(orc.lemma1_sort(M).reshape(-1), np.sort(M.reshape(-1)))


# ------------------------------------------------------------ race check ----
def _rec(thread, addr, kind, width=4, block=0):
    return [0, thread | (block << 16), addr, width | (kind << 8) | (1 << 16)]


def _bar(thread, block=0):
    return [0, thread | (block << 16), 0, (3 << 8) | (30 << 16)]


def test_race_check_rules(orc):
    """Different threads, one word, no barrier between, a store among them: a race.
    A barrier in every warp between them, one thread, loads only, atomics, or
    different blocks: none."""
    R = lambda rows: orc.race_check(np.array(rows, dtype=np.uint32))[0]
    assert R([_rec(0, 64, 1), _rec(33, 64, 1)]) == 1                     # two writers
    assert R([_rec(0, 64, 1), _rec(5, 64, 0)]) == 1                      # write, other thread reads
    assert R([_rec(0, 64, 1), _rec(0, 64, 0), _rec(0, 64, 1)]) == 0      # one thread
    assert R([_rec(0, 64, 0), _rec(40, 64, 0)]) == 0                     # loads only
    assert R([_rec(0, 64, 2), _rec(40, 64, 2)]) == 0                     # atomics
    assert R([_rec(0, 64, 1, block=0), _rec(40, 64, 1, block=1)]) == 0  # other block
    assert R([_rec(0, 64, 1), _bar(0), _bar(32), _rec(40, 64, 0)]) == 0  # barrier between
    assert R([_rec(0, 64, 1), _bar(0), _rec(40, 64, 0)]) == 1            # warp 1 not past it yet
    assert R([_rec(0, 60, 1, width=8), _rec(3, 64, 0)]) == 1             # wide store covers the word
    assert R([_rec(0, 56, 1, width=8), _rec(3, 64, 0)]) == 0
    races, words = orc.race_check(np.array([_rec(0, 0, 1, width=16), _rec(1, 16, 1)], dtype=np.uint32))
    assert (races, words) == (0, 5)


def _wbar(thread, block=0):
    return [0, thread | (block << 16), 0, (4 << 8) | (30 << 16)]


def test_race_check_warp_barriers(orc):
    """A warp barrier orders the accesses of one warp's lanes, not those of two warps;
    a block barrier still splits everything."""
    R = lambda rows: orc.race_check(np.array(rows, dtype=np.uint32))[0]
    assert R([_rec(0, 64, 1), _wbar(0), _rec(7, 64, 0)]) == 0              # same warp, barrier between
    assert R([_rec(0, 64, 1), _rec(7, 64, 0)]) == 1                        # same warp, none
    assert R([_rec(0, 64, 1), _wbar(0), _wbar(32), _rec(40, 64, 0)]) == 1  # two warps: not ordered
    assert R([_rec(7, 64, 0), _wbar(0), _rec(0, 64, 1)]) == 0              # read, barrier, then write
    assert R([_rec(0, 64, 1), _wbar(0), _rec(7, 64, 1), _rec(9, 64, 0)]) == 1  # 7 and 9 after it, unordered
    # a block barrier between makes the warp epochs irrelevant
    assert R([_rec(0, 64, 1), _wbar(0), _bar(0), _bar(32), _rec(40, 64, 0)]) == 0


# ------------------------------------------------- Lemma 2 (0-1 partition) ----
def _l2_inputs(w, m, seed):
    """Random labels at several densities and structured ones (all 0, all 1, one
    1, alternating rows, alternating columns, one 0 per row, 0s in the top half,
    random with exactly half 0s), payload = cell index."""
    g = np.random.default_rng(seed)
    pay = np.arange(w * m, dtype=np.uint32).reshape(w, m)
    cases = [(g.random((w, m)) < p).astype(np.uint32) for p in (0.003, 0.3, 0.5, 0.7, 0.97)]
    cases.append(np.zeros((w, m), np.uint32))
    cases.append(np.ones((w, m), np.uint32))
    one = np.zeros((w, m), np.uint32)
    one[w // 3, m // 2] = 1
    cases.append(one)
    cases.append(np.tile((np.arange(w) % 2)[:, None], (1, m)).astype(np.uint32))
    cases.append(np.tile((np.arange(m) % 2)[None, :], (w, 1)).astype(np.uint32))
    lone = np.ones((w, m), np.uint32)
    lone[np.arange(w), np.arange(w) % m] = 0
    cases.append(lone)
    cases.append((np.arange(w)[:, None] >= w // 2).repeat(m, 1).astype(np.uint32))  # zeros in the top half
    for _ in range(4):  # exactly half zeros: the dirty rows sit at row w/2, a square boundary
        cases.append(g.permutation(np.arange(w * m) % 2).reshape(w, m).astype(np.uint32))
    return [(lab, pay) for lab in cases]


def _is_partitioned(lab):
    f = lab.ravel().astype(np.int64)
    return bool(np.all(np.diff(f) >= 0))


@pytest.mark.parametrize("w,m", [(1024, 32), (256, 16), (16, 4), (32, 32), (8, 8)])
def test_lemma2_partitions_and_keeps_pairs(orc, w, m):
    """The whole algorithm: read row by row, the labels are all 0s then all 1s
    (the partition problem's definition), and every (label, payload) pair survives."""
    for lab, pay in _l2_inputs(w, m, seed=w + m):
        lo, po = orc.lemma2_partition(lab, pay)
        assert _is_partitioned(lo)
        assert int(lo.sum()) == int(lab.sum())
        assert sorted(zip(lab.ravel().tolist(), pay.ravel().tolist())) == sorted(zip(lo.ravel().tolist(), po.ravel().tolist()))


@pytest.mark.parametrize("w,m", [(1024, 32), (256, 16), (64, 8)])
def test_lemma2_balancing_bounds(orc, w, m):
    """After balancing (k = log_m w = 2 rounds) every row holds between w0/w - k
    and w0/w + k zeros (w0 = all zeros), its 0s left of its 1s, so at most 2k
    columns are dirty (Lemma 2's proof, "Convert and Divide")."""
    k = 2
    for lab, pay in _l2_inputs(w, m, seed=3 * w):
        lo, _ = orc.lemma2_partition(lab, pay, stage=1)
        zeros = m - lo.sum(axis=1).astype(np.int64)
        w0 = int((lab == 0).sum())
        assert np.all(zeros >= w0 / w - k) and np.all(zeros <= w0 / w + k)
        for r in range(w):
            assert np.all(np.diff(lo[r].astype(np.int64)) >= 0)
        dirty_cols = sum(1 for c in range(m) if 0 < lo[:, c].sum() < w)
        assert dirty_cols <= 2 * k


@pytest.mark.parametrize("w,m", [(1024, 32), (256, 16)])
def test_lemma2_leaves_columns_and_dirty_rows(orc, w, m):
    """After convert-and-divide every sub-problem of w/(4m) rows is sorted row by row
    (at most one dirty row each); after the column sorts every column is 0s above 1s,
    and the dirty rows are contiguous and at most m/2 of them, so one of the two
    square decompositions holds them all."""
    chunk = w // (4 * m)
    for lab, pay in _l2_inputs(w, m, seed=5 * w):
        l2, _ = orc.lemma2_partition(lab, pay, stage=2)
        for r0 in range(0, w, chunk):
            assert _is_partitioned(l2[r0:r0 + chunk])
        l3, _ = orc.lemma2_partition(lab, pay, stage=3)
        for c in range(m):
            assert np.all(np.diff(l3[:, c].astype(np.int64)) >= 0)
        dirty = [r for r in range(w) if 0 < l3[r].sum() < m]
        assert len(dirty) <= m // 2
        if dirty:
            assert dirty == list(range(dirty[0], dirty[-1] + 1))
            assert np.all(l3[:dirty[0]] == 0) and np.all(l3[dirty[-1] + 1:] == 1)


@pytest.mark.parametrize("label", [0, 1])
def test_lemma2_uniform_labels_move_nothing(orc, label):
    """With one label every sort is the identity, so the algorithm only converts:
    the output read row by row is the input read column by column (the array's
    column-major layout, Sec. 1)."""
    w, m = 1024, 32
    lab = np.full((w, m), label, np.uint32)
    pay = np.arange(w * m, dtype=np.uint32).reshape(m, w).T.copy()  # A[k] in row k % w, column k // w
    _, po = orc.lemma2_partition(lab, pay)
    assert np.array_equal(po.ravel(), np.arange(w * m, dtype=np.uint32))


def test_lemma2_step_sorts_against_stable_argsort(orc):
    """The two step sorts are stable 0-1 sorts of a cell sequence: compared with
    numpy's stable argsort of the labels gathered in that sequence."""
    g = np.random.default_rng(11)
    w, m = 64, 8
    for _ in range(20):
        lab = g.integers(0, 2, size=(w, m), dtype=np.uint32)
        pay = np.arange(w * m, dtype=np.uint32).reshape(w, m)
        rows = g.permutation(w)[:m]
        seq = [(r, c) for c in range(m) for r in rows]  # column-major order of the square
        l1, p1 = lab.copy(), pay.copy()
        orc.l2_sort_colmajor(l1, p1, rows)
        src = np.array([lab[r, c] for r, c in seq])
        order = np.argsort(src, kind="stable")
        assert [p1[r, c] for r, c in seq] == [pay[seq[i]] for i in order]
        r0, h = int(g.integers(0, w - 8)), 8
        l2, p2 = lab.copy(), pay.copy()
        orc.l2_sort_rowmajor(l2, p2, r0, h)
        flat = lab[r0:r0 + h].ravel()
        order = np.argsort(flat, kind="stable")
        assert np.array_equal(p2[r0:r0 + h].ravel(), pay[r0:r0 + h].ravel()[order])
        assert np.array_equal(np.delete(p2, range(r0, r0 + h), 0), np.delete(pay, range(r0, r0 + h), 0))


def test_lemma2_rejects_other_shapes_and_labels(orc):
    with pytest.raises(orc.OracleError):
        orc.lemma2_partition(np.zeros((512, 32), np.uint32), np.zeros((512, 32), np.uint32))
    with pytest.raises(orc.OracleError):
        orc.lemma2_partition(np.zeros((36, 6), np.uint32), np.zeros((36, 6), np.uint32))
    lab = np.zeros((16, 4), np.uint32)
    lab[3, 1] = 2
    with pytest.raises(orc.OracleError):
        orc.lemma2_partition(lab, np.zeros((16, 4), np.uint32))
