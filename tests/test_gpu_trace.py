"""Bank-model replay of the tile kernels' shared-memory traces.

The trace build (libbcf_trace.so) records every instrumented shared-memory access;
the CPU bank model of the oracle (Sec. 1 "Model of Computation": 32 banks of 4-byte
words, a request conflicts when two of its lanes need different words of one bank)
replays them.  The schedules that follow the paper -- Lemma 1's row sorts and
diagonal conversions, the strided staging reads, and the colour-class sends of
Sec. 3 -- must replay with zero hardware conflicts; the direct scatter of a random
permutation must show the conflicts they avoid.  The traced kernels also still
produce the oracle's results."""
import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    import paper_1507_01391_b300 as bcf
    bcf.lib()
    from paper_1507_01391_b300 import trace
    trace.load()
    return trace


def _replay(tr, rec, site=None):
    req, lane, addr, width, store, s = tr.fields(tr.accesses(rec))
    if site is not None:
        keep = s == tr.SITES[site]
        req, lane, addr, width = req[keep], lane[keep], addr[keep], width[keep]
    if req.size == 0:
        return None
    wf, hw, strict = oracle.bank_count(req, lane, addr, width)
    nreq = int(np.count_nonzero(np.diff(req)) + 1)
    r = {"requests": nreq, "wavefronts": wf, "hw_conflicts": hw, "strict_conflicts": strict}
    print("replay %-14s %s" % (site or "all", r))  # shown with pytest -s
    return r


def test_lemma1_tile_sort_replays_conflict_free(tr):
    import paper_1507_01391_b300 as bcf
    n = 4096
    keys = synth.uniform_keys(n, seed=1)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.sort_tiles(dev(keys), dev(vals))
    rec, total = tr.capture(run)
    assert total == rec.shape[0] > 100_000
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    for site in ("l1_row_ld", "l1_row_st", "l1_convert", "l1_io"):
        r = _replay(tr, rec, site)
        assert r is not None and r["hw_conflicts"] == 0, (site, r)
    assert _replay(tr, rec)["hw_conflicts"] == 0
    _no_races(rec)


def _no_races(rec):
    """No two threads touch one word between the same two barriers with a store
    among them (the trace's barrier records split each warp's accesses)."""
    races, words = oracle.race_check(rec)
    print("race check: %d racing words of %d checked" % (races, words))
    assert words > 0 and races == 0


def test_coloured_sends_meet_the_conflict_avoidance_condition(tr):
    """Every colour-class send touches distinct banks -- even under the strict
    rule, in which two lanes may never share a bank (the paper's CAC)."""
    import paper_1507_01391_b300 as bcf
    tile = 4096
    src = synth.uniform_keys(tile, seed=2)
    lpi = synth.tile_local_perms(tile, tile, seed=3)
    out = {}

    def run():
        out["y"] = bcf.permute_tiles(dev(src), dev(lpi), tile=tile, coloured=True, seed=7)
    rec, _ = tr.capture(run)
    assert bits_equal(host(out["y"], np.uint32), oracle.permute_tiles(src, lpi, tile))
    send = _replay(tr, rec, "col_send")
    assert send["requests"] > 100 and send["hw_conflicts"] == 0 and send["strict_conflicts"] == 0, send
    for site in ("col_table", "col_finish", "writeout_read"):
        r = _replay(tr, rec, site)
        if r is not None:
            assert r["hw_conflicts"] == 0, (site, r)
    assert _replay(tr, rec)["hw_conflicts"] == 0
    _no_races(rec)


@pytest.mark.parametrize("tile", [1024, 4096])
def test_sorted_finish_sends_meet_the_conflict_avoidance_condition(tr, tile):
    """The finishing step of Sec. 3: leftovers sorted by destination and sent in
    three groups.  Every finishing send request touches distinct banks (strict
    rule); only the ordering/packing step may conflict."""
    import paper_1507_01391_b300 as bcf
    lpi = synth.tile_local_perms(4 * tile, tile, seed=5)
    src = synth.uniform_keys(4 * tile, seed=6)
    out = {}

    def run():
        out["y"] = bcf.permute_tiles(dev(src), dev(lpi), tile=tile, coloured=True, seed=11, finish="sorted")
    rec, _ = tr.capture(run)
    assert bits_equal(host(out["y"], np.uint32), oracle.permute_tiles(src, lpi, tile))
    fin = _replay(tr, rec, "col_finish")  # random permutations leave a few items per tile
    assert fin is not None and fin["requests"] > 0, "no leftovers reached the finishing step"
    assert fin["hw_conflicts"] == 0 and fin["strict_conflicts"] == 0, fin
    for site in ("col_send", "col_read"):
        r = _replay(tr, rec, site)
        assert r is None or r["hw_conflicts"] == 0, (site, r)
    assert _replay(tr, rec, "col_pack") is not None
    _no_races(rec)


def test_direct_scatter_shows_the_conflicts(tr):
    """The same permutation scattered directly: random banks within each request,
    so the replay must count conflicts (about 2-4 wavefronts per request)."""
    import paper_1507_01391_b300 as bcf
    tile = 4096
    src = synth.uniform_keys(tile, seed=2)
    lpi = synth.tile_local_perms(tile, tile, seed=3)
    rec, _ = tr.capture(lambda: bcf.permute_tiles(dev(src), dev(lpi), tile=tile, coloured=False))
    sc = _replay(tr, rec, "scatter")
    per_req = sc["wavefronts"] / sc["requests"]
    assert sc["hw_conflicts"] > 0 and 2.0 < per_req < 5.0, sc
    assert _replay(tr, rec, "stage_read")["hw_conflicts"] == 0
    _no_races(rec)


def test_sweep_strided_reads_are_conflict_free(tr):
    """Digit sweep of a w = 32 partition (the staged-tile configuration): the
    strided staging reads (lane l reads word 32i + l) replay conflict-free; the
    scatter into label order does not."""
    import paper_1507_01391_b300 as bcf
    n, w = 4096, 32
    keys = synth.partition_keys(n, w, seed=4)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.partition(dev(keys), dev(vals), w, balanced=True)
    L = tr.load()
    assert L.bcf_tune_config_form(8) == 2  # the staged-tile sweep, 256 x 16
    assert L.bcf_tune_set(bcf.OP_PARTITION, 12, 8) == bcf.OK
    try:
        rec, _ = tr.capture(run)
    finally:
        L.bcf_tune_set(bcf.OP_PARTITION, 12, -1)
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=True)
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    assert _replay(tr, rec, "stage_read")["hw_conflicts"] == 0
    assert _replay(tr, rec, "writeout_read")["hw_conflicts"] == 0
    sc = _replay(tr, rec, "scatter")
    assert sc is not None and sc["requests"] == n // 32
    _no_races(rec)


@pytest.mark.parametrize("n", [3 * 2048 + 5, 3 * 4096])
def test_single_launch_sort_trace(tr, n):
    """The single-launch sort passes: the one-read histogram keeps every lane's
    counters in the lane's own bank, so its counting atomics and the diagonal sums
    replay with zero conflicts even under the strict rule; the per-warp offset rows
    and the ordered write-out read replay conflict-free; the scatter into digit
    order and the leaders' run claims are random-bank accesses and are counted
    (reported, not asserted zero).  No word races between barriers."""
    import paper_1507_01391_b300 as bcf
    keys = synth.uniform_keys(n, seed=n)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.sort(dev(keys), dev(vals))
    L = tr.load()
    lg = (n - 1).bit_length()
    assert L.bcf_tune_config_form(1) == 0  # single launch per pass, 256 x 8
    assert L.bcf_tune_set(bcf.OP_SORT, lg, 1) == bcf.OK
    try:
        rec, _ = tr.capture(run)
    finally:
        L.bcf_tune_set(bcf.OP_SORT, lg, -1)
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    for site in ("hist_atom", "hist_sum"):
        r = _replay(tr, rec, site)
        assert r is not None and r["hw_conflicts"] == 0 and r["strict_conflicts"] == 0, (site, r)
    for site in ("warp_offsets", "writeout_read"):
        r = _replay(tr, rec, site)
        assert r is not None and r["hw_conflicts"] == 0, (site, r)
    sc = _replay(tr, rec, "scatter")
    assert sc is not None and sc["requests"] >= 4 * n // 32  # keys and payloads, four passes
    assert _replay(tr, rec, "claim_atom") is not None
    _no_races(rec)


@pytest.mark.parametrize("n", [8 * 4096, 8 * 4096 + 3 * 1024 + 7])
def test_tile_count_sort_trace(tr, n):
    """The reduce-then-scan sort passes (counts, scan, pass body): the per-tile
    count kernel keeps every lane's byte counters in the lane's own bank, so its
    counting atomics replay with zero conflicts under both rules (full groups of
    four tiles; a ragged remainder takes the shared-histogram path), and the
    diagonal 16-byte sums of the lane words with zero under the hardware rule (the
    strict rule counts the four words of one lane's 16-byte access as four lanes on
    a bank).  No word races between barriers."""
    import paper_1507_01391_b300 as bcf
    keys = synth.uniform_keys(n, seed=n + 1)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.sort(dev(keys), dev(vals))
    L = tr.load()
    lg = (n - 1).bit_length()
    assert L.bcf_tune_config_form(4) == 1  # counts + scan + pass body, 256 x 16
    assert L.bcf_tune_set(bcf.OP_SORT, lg, 4) == bcf.OK
    try:
        rec, _ = tr.capture(run)
    finally:
        L.bcf_tune_set(bcf.OP_SORT, lg, -1)
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    r = _replay(tr, rec, "tile_count_atom")
    assert r is not None and r["hw_conflicts"] == 0 and r["strict_conflicts"] == 0, r
    r = _replay(tr, rec, "tile_count_sum")
    assert r is not None and r["hw_conflicts"] == 0 and r["wavefronts"] == 4 * r["requests"], r
    assert _replay(tr, rec, "tile_count_atom")["requests"] == 4 * (8 * 4096 // 32)  # four passes, full tiles
    _no_races(rec)


def test_lemma1_partition_replays_conflict_free(tr):
    """The Lemma 1 tile partition: every shared access of its schedule replays
    with zero hardware conflicts (the label counts are the only atomics)."""
    import paper_1507_01391_b300 as bcf
    n, w = 4096, 32
    keys = synth.partition_keys(n, w, seed=9)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.partition(dev(keys), dev(vals), w, balanced=True, flags=bcf.PARTITION_LEMMA1)
    rec, _ = tr.capture(run)
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=True)
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    for site in ("l1_row_ld", "l1_row_st", "l1_convert", "l1_io"):
        r = _replay(tr, rec, site)
        assert r is not None and r["hw_conflicts"] == 0, (site, r)
    _no_races(rec)


@pytest.mark.parametrize("n", [65536, 3 * 2048 + 5])
def test_direct_partition_replays_conflict_free(tr, n):
    """The partition by 32 labels with the direct write-out: label = bank, so the
    run claims, the warps' starts and the offset lookups touch one word per label,
    the staging reads are strided, and no key is scattered in shared memory --
    every shared access of the pass replays with zero hardware conflicts, and no
    word races between barriers."""
    import paper_1507_01391_b300 as bcf
    w = 32
    keys = synth.partition_keys(n - n % w, w, seed=n) if n % w == 0 else synth.random_labels(n, w, seed=n)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.partition(dev(keys), dev(vals), w, balanced=(n % w == 0),
                                           flags=bcf.PARTITION_DIRECT)
    rec, _ = tr.capture(run)
    rk, rv = oracle.partition_kv(keys, vals, w, balanced=(n % w == 0))
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    whole = _replay(tr, rec)
    assert whole is not None and whole["requests"] > n // 32 and whole["hw_conflicts"] == 0, whole
    assert _replay(tr, rec, "scatter") is None  # nothing scattered in shared memory
    for site in ("claim_atom", "warp_offsets", "offset_read", "stage_read"):
        r = _replay(tr, rec, site)
        assert r is not None and r["hw_conflicts"] == 0, (site, r)
    _no_races(rec)


def test_segmented_small_path_has_no_races(tr):
    """The batched sort's small-segment path (one tile per segment and packed bins
    of tiny segments) keeps every shared word private between barriers."""
    import torch

    import paper_1507_01391_b300 as bcf
    sizes = [3000, 17, 1, 2048, 900, 5, 4000]
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    keys = synth.uniform_keys(n, seed=12)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.segmented_sort(dev(keys), dev(vals), torch.from_numpy(offs).cuda())
    rec, _ = tr.capture(run)
    rk, rv = oracle.segmented_sort_kv(keys, vals, offs)
    assert bits_equal(host(out["k"], np.uint32), rk) and bits_equal(host(out["v"], np.uint32), rv)
    _no_races(rec)


L2_SITES = ("l2_square", "l2_convert", "l2_divide", "l2_column", "l2_rows", "l2_shifted", "l2_io")


@pytest.mark.parametrize("p", [0.5, 0.03])
def test_lemma2_partition_trace(tr, p):
    """Lemma 2's 0-1 partition (two 1024 x 32 matrices): the result is the oracle's,
    no two threads race on a word (warp barriers order each step sort's reads
    before its writes), and every step's accesses replay through the bank model;
    the per-step counts under both rules are printed (pytest -s)."""
    import paper_1507_01391_b300 as bcf
    n = 2 * 32768
    keys = synth.bernoulli_labels(n, p, seed=31)
    vals = synth.index_payload(n)
    out = {}

    def run():
        out["k"], out["v"] = bcf.partition_lemma2(dev(keys), dev(vals))
    rec, total = tr.capture(run)
    assert total == rec.shape[0]
    ko, vo = host(out["k"], np.uint32), host(out["v"], np.uint32)
    for t in range(2):
        a = slice(t * 32768, (t + 1) * 32768)
        lo, po = oracle.lemma2_partition(keys[a].reshape(32, 1024).T, vals[a].reshape(32, 1024).T)
        assert np.array_equal(ko[a], lo.ravel()) and bits_equal(vo[a], po.ravel())
    _, _, _, _, store, _ = tr.fields(rec)
    assert np.count_nonzero(store == 4) > 0  # the step sorts' warp barriers were recorded
    seen = {site: _replay(tr, rec, site) for site in L2_SITES}
    for site in ("l2_square", "l2_convert", "l2_column", "l2_io"):
        assert seen[site] is not None, site
    # The step sorts scatter a run of 0-items and a run of 1-items, each to
    # consecutive positions: a square's column step is at most 2-way, and so is
    # every access of the shifted squares (the row rotation maps lanes 0 and 31 of
    # a window to one bank).  The padded row-major write-out is conflict-free.
    for site in ("l2_square", "l2_convert", "l2_shifted"):
        if seen[site] is not None:
            assert seen[site]["wavefronts"] <= 2 * seen[site]["requests"], (site, seen[site])
    assert seen["l2_io"]["hw_conflicts"] == 0
    _no_races(rec)


PROBE_BLOCKS, PROBE_REPS = 3 * 148, 32


@pytest.mark.parametrize("pattern", range(9))
def test_bank_probe_patterns(tr, pattern):
    """The probe kernels (one shared-memory access pattern of the Lemma 1 tile sort
    each): the traced copy replays with zero hardware conflicts in the bank model
    and no races; the untraced copies run with every kind of global traffic
    beside them, and the traffic that does not feed the checksum (none / store,
    and L1 / L2-only gathers of the same words) leaves it unchanged."""
    import ctypes

    import torch

    L = tr.load()
    OK = 0
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    blocks = PROBE_BLOCKS
    gin = torch.arange(blocks * 4096, dtype=torch.int32, device="cuda")
    outs = []

    def run():
        gout = torch.zeros(blocks * (4096 + 256), dtype=torch.int32, device="cuda")
        assert L.bcf_trace_bank_probe(pattern, 0, 1, ptr(gin), ptr(gout), 2, 2, None) == OK
    rec, total = tr.capture(run)
    assert total == rec.shape[0]
    r = _replay(tr, rec, "probe")
    assert r is not None and r["hw_conflicts"] == 0, r
    _no_races(rec)
    for traffic in range(4):
        gout = torch.zeros(blocks * (4096 + 256), dtype=torch.int32, device="cuda")
        assert L.bcf_trace_bank_probe(pattern, traffic, 0, ptr(gin), ptr(gout), blocks, PROBE_REPS, None) == OK
        torch.cuda.synchronize()
        outs.append(gout[blocks * 4096:].cpu())
    assert torch.equal(outs[0], outs[3]) and torch.equal(outs[1], outs[2])
    assert not torch.equal(outs[0], outs[1])
