"""GPU parity: Lemma 1 tile sort, segmented sort and segmented partition through
the C ABI, bit-exact against the CPU oracle, including empty and one-key
segments, the small/long boundary (4096 keys), misaligned segment starts, the
batched workload at full size, CUDA-graph capture and bad offsets."""
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


# ---------------------------------------------------------------- tile sort
@pytest.mark.parametrize("n", [1, 5, 4095, 4096, 4097, 3 * 4096 + 1234])
@pytest.mark.parametrize("vb", [0, 4, 8])
def test_sort_tiles(bcf, n, vb):
    keys = synth.random_labels(n, 1000, seed=n) if n % 2 else synth.uniform_keys(n, seed=n)
    vals = None if vb == 0 else (synth.float_bits_payload(n, seed=2) if vb == 4
                                 else synth.uniform_keys(2 * n, seed=3).view(np.uint64))
    ko, vo = bcf.sort_tiles(dev(keys), None if vals is None else dev(vals))
    offs = synth.offsets_from_sizes([min(4096, n - s) for s in range(0, n, 4096)])
    rk, rv = oracle.segmented_sort_kv(keys, vals, offs)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


@pytest.mark.parametrize("kind", ["equal", "sorted", "reverse", "max"])
def test_sort_tiles_structured(bcf, kind):
    n = 2 * 4096
    keys = {"equal": np.full(n, 7, np.uint32),
            "sorted": np.arange(n, dtype=np.uint32),
            "reverse": np.arange(n, 0, -1, dtype=np.uint32),
            "max": np.full(n, 0xFFFFFFFF, np.uint32)}[kind]
    ko, vo = bcf.sort_tiles(dev(keys), dev(synth.index_payload(n)))
    rk, rv = oracle.segmented_sort_kv(keys, synth.index_payload(n), np.array([0, 4096, n]))
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv)


# ------------------------------------------------------------ segmented sort
def _seg_sort_case(bcf, keys, vals, offs, key_bits=32):
    import torch
    ko, vo = bcf.segmented_sort(dev(keys), None if vals is None else dev(vals),
                                torch.from_numpy(offs).cuda(), key_bits=key_bits)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.segmented_sort_kv(keys, vals, offs)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


@pytest.mark.parametrize("sizes", [
    [0, 1, 2, 3, 0, 4095, 4096, 4097, 0],          # small/long boundary, empty segments
    [1, 10_000, 3, 8193, 5, 70_001],               # misaligned long segments
    [4096 * 3],                                     # one long segment
    [17] * 50,                                      # many small ones
    # tiny segments (<= 2048 keys) share tiles: bins cut at running offsets 2048,
    # 4096, ...; 2048/2049 and 4096/4097 are the tiny/one-tile/long boundaries
    [2048, 1, 2047, 2, 2048, 0, 2049, 1, 1, 4096, 30, 5000, 7, 2048, 2048, 1],
    [1] * 3000 + [2048] + [3] * 700,                # thousands of one-key segments in a bin
    [1000, 9000, 1000, 1500, 0, 600, 4097, 2000, 47],  # tiny ones separated by long ones
])
@pytest.mark.parametrize("vb", [0, 4, 8])
def test_segmented_sort_sizes(bcf, sizes, vb):
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    keys = synth.uniform_keys(n, seed=len(sizes) + vb)
    vals = None if vb == 0 else (synth.index_payload(n) if vb == 4 else synth.uniform_keys(2 * n, seed=1).view(np.uint64))
    _seg_sort_case(bcf, keys, vals, offs)


@pytest.mark.parametrize("key_bits", [8, 20, 32])
def test_segmented_sort_log_uniform(bcf, key_bits):
    sizes = synth.log_uniform_sizes(300, seed=key_bits, hi_log2=15)
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    _seg_sort_case(bcf, synth.uniform_keys(n, seed=7, bits=key_bits), synth.index_payload(n), offs, key_bits)


def test_segmented_sort_index_payload(bcf):
    import torch
    sizes = [100, 5000, 3, 20000]
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    keys = synth.random_labels(n, 50, seed=3)
    ko, perm = bcf.segmented_sort(dev(keys), None, torch.from_numpy(offs).cuda(), index_payload=True)
    rk, rv = oracle.segmented_sort_kv(keys, synth.index_payload(n), offs)
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(perm, np.uint32), rv)


@pytest.mark.parametrize("config", [4, 8])
@pytest.mark.parametrize("vb", [0, 4, 8])
def test_segmented_sort_pass_forms(bcf, config, vb):
    """Both pass forms the tuning table can name for a batch -- the pass body fed
    scanned offsets (configuration 4) and the staged sweep (8) -- give the
    oracle's result: segment starts off the 16-byte grid (payload copies that
    begin mid-vector), ragged last pieces, empty and small segments between long
    ones, and (4-byte payloads) the index-payload mode."""
    import torch
    L = bcf.lib()
    sizes = [1, 10_000, 3, 8193, 5, 70_001, 0, 4097, 12_288, 2, 4099]
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    lg = (n - 1).bit_length()
    assert L.bcf_tune_config_form(config) == (1 if config == 4 else 2)
    assert L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, lg, config) == bcf.OK
    try:
        keys = synth.uniform_keys(n, seed=40 + vb)
        vals = None if vb == 0 else (synth.float_bits_payload(n, seed=41) if vb == 4
                                     else synth.uniform_keys(2 * n, seed=42).view(np.uint64))
        _seg_sort_case(bcf, keys, vals, offs)
        _seg_sort_case(bcf, synth.random_labels(n, 7, seed=43), vals, offs, key_bits=20)
        if vb == 4:
            ko, perm = bcf.segmented_sort(dev(keys), None, torch.from_numpy(offs).cuda(), index_payload=True)
            rk, rv = oracle.segmented_sort_kv(keys, synth.index_payload(n), offs)
            assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(perm, np.uint32), rv)
    finally:
        L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, lg, -1)


@pytest.mark.slow
def test_segmented_sort_batched_full_size(bcf):
    """The batched workload: 10,000 segments, sizes log-uniform in [32, 2^18]."""
    sizes = synth.log_uniform_sizes(10_000, seed=0x4A)
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    _seg_sort_case(bcf, synth.uniform_keys(n, seed=0x4B), synth.index_payload(n), offs)


def test_segmented_sort_graph_capture(bcf):
    """The whole call is capturable: replaying the graph on new keys in the same
    buffers gives the oracle's answer for the new keys."""
    import torch
    sizes = [100, 5000, 0, 9000, 4096]
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    kd = dev(synth.uniform_keys(n, seed=1))
    vd = dev(synth.index_payload(n))
    od = torch.from_numpy(offs).cuda()
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    ws = bcf.workspace(bcf.segmented_sort_workspace_size(n, len(sizes), 4, 32))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bcf.segmented_sort(kd, vd, od, keys_out=ko, vals_out=vo, ws=ws)  # warm-up outside capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bcf.segmented_sort(kd, vd, od, keys_out=ko, vals_out=vo, ws=ws)
    new = synth.uniform_keys(n, seed=99)
    kd.copy_(dev(new))
    g.replay()
    torch.cuda.synchronize()
    rk, rv = oracle.segmented_sort_kv(new, synth.index_payload(n), offs)
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv)
    assert bcf.get_status() == bcf.OK


@pytest.mark.slow
def test_segmented_sort_batched_full_size_graph_replay(bcf):
    """The batched workload as the benchmark times it: one call captured in a CUDA
    graph, replayed on new keys copied into the captured buffers; the replay's
    output is compared in full with the oracle."""
    import torch
    sizes = synth.log_uniform_sizes(10_000, seed=0x4A)
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    kd = dev(synth.uniform_keys(n, seed=0x4B))
    vd = dev(synth.index_payload(n))
    od = torch.from_numpy(offs).cuda()
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    ws = bcf.workspace(bcf.segmented_sort_workspace_size(n, sizes.size, 4, 32))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bcf.segmented_sort(kd, vd, od, keys_out=ko, vals_out=vo, ws=ws)  # warm-up outside capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bcf.segmented_sort(kd, vd, od, keys_out=ko, vals_out=vo, ws=ws)
    new = synth.uniform_keys(n, seed=0x4D)
    kd.copy_(dev(new))
    torch.cuda.synchronize()
    g.replay()
    g.replay()  # a second replay over its own output's inputs: the same answer
    torch.cuda.synchronize()
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.segmented_sort_kv(new, synth.index_payload(n), offs)
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv)


def test_segmented_reports_bad_offsets(bcf):
    import torch
    offs = np.array([0, 10, 5, 20], dtype=np.int64)  # decreasing
    keys = synth.uniform_keys(20, seed=1)
    bcf.segmented_sort(dev(keys), None, torch.from_numpy(offs).cuda())
    assert bcf.get_status() == bcf.E_INVAL


# ------------------------------------------------------ segmented partition
def _seg_part_case(bcf, keys, vals, offs, w, balanced):
    import torch
    ko, vo = bcf.segmented_partition(dev(keys), None if vals is None else dev(vals),
                                     torch.from_numpy(offs).cuda(), dev(w.astype(np.int32)),
                                     balanced=balanced)
    assert bcf.get_status() == bcf.OK
    rk, rv = oracle.segmented_partition_kv(keys, vals, offs, w, balanced=balanced)
    assert bits_equal(host(ko, np.uint32), rk)
    if vals is not None:
        assert bits_equal(host(vo, vals.dtype), rv)


@pytest.mark.parametrize("balanced", [True, False])
def test_segmented_partition(bcf, balanced):
    keys, offs, w = synth.segmented_partition_input(60, seed=3, hi_log2=14)
    if not balanced:
        keys = np.concatenate([synth.random_labels(int(offs[s + 1] - offs[s]), int(w[s]), seed=s)
                               for s in range(w.size)]).astype(np.uint32)
    _seg_part_case(bcf, keys, synth.index_payload(keys.size), offs, w, balanced)


@pytest.mark.parametrize("config", [4, 8])
@pytest.mark.parametrize("vb", [0, 4, 8])
@pytest.mark.parametrize("balanced", [True, False])
def test_segmented_partition_pass_forms(bcf, config, vb, balanced):
    """Both pass forms the batched tuning entry can name -- the pass body fed
    scanned offsets (4) and the staged sweep (8) -- partition every segment as the
    oracle does: segments of every width, empty ones, starts off the 16-byte grid,
    ragged last pieces."""
    L = bcf.lib()
    w = np.array([32, 256, 7, 64, 1, 128, 200, 3], dtype=np.int32)
    sizes = [32 * 300, 256 * 40, 7 * 3, 0, 5, 128 * 70, 200 * 21, 3 * 1001]
    offs = synth.offsets_from_sizes(sizes)
    n = int(offs[-1])
    g = synth.rng(11 + vb)
    keys = np.concatenate([(g.permutation(np.arange(sizes[s]) % w[s]) if balanced
                            else g.integers(0, w[s], sizes[s])) for s in range(w.size)]).astype(np.uint32)
    vals = None if vb == 0 else (synth.float_bits_payload(n, seed=12) if vb == 4
                                 else synth.uniform_keys(2 * n, seed=13).view(np.uint64))
    lg = (n - 1).bit_length()
    assert L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, lg, config) == bcf.OK
    try:
        _seg_part_case(bcf, keys, vals, offs, w, balanced)
    finally:
        L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, lg, -1)


@pytest.mark.slow
def test_segmented_partition_batched_full_size(bcf):
    keys, offs, w = synth.segmented_partition_input(10_000, seed=0x4C)
    _seg_part_case(bcf, keys, synth.index_payload(keys.size), offs, w, True)


@pytest.mark.parametrize("balanced", [True, False])
def test_segmented_partition_graph_capture(bcf, balanced):
    """The segmented partition is capturable: a graph of one call, replayed on new
    labels in the same buffers, gives the oracle's answer for the new labels."""
    import torch
    keys, offs, w = synth.segmented_partition_input(40, seed=5, hi_log2=14)
    n = keys.size

    def labels(seed):
        if balanced:  # the same label multiset per segment, reshuffled
            g = synth.rng(seed)
            out = keys.copy()
            for s in range(w.size):
                g.shuffle(out[offs[s]:offs[s + 1]])
            return out
        return np.concatenate([synth.random_labels(int(offs[s + 1] - offs[s]), int(w[s]), seed=seed + s)
                               for s in range(w.size)]).astype(np.uint32)
    kd = dev(labels(1))
    vd = dev(synth.index_payload(n))
    od = torch.from_numpy(offs).cuda()
    wd = dev(w.astype(np.int32))
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    ws = bcf.workspace(bcf.segmented_partition_workspace_size(n, w.size, 4))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bcf.segmented_partition(kd, vd, od, wd, balanced=balanced, keys_out=ko, vals_out=vo, ws=ws)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bcf.segmented_partition(kd, vd, od, wd, balanced=balanced, keys_out=ko, vals_out=vo, ws=ws)
    for seed in (2, 3):
        new = labels(seed)
        kd.copy_(dev(new))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert bcf.get_status() == bcf.OK
        rk, rv = oracle.segmented_partition_kv(new, synth.index_payload(n), offs, w, balanced=balanced)
        assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv)


@pytest.mark.parametrize("balanced", [True, False])
def test_segmented_partition_reports_bad_label_and_unbalanced_counts(bcf, balanced):
    """A label at its segment's width is flagged (E_BAD_KEY; with balanced=True the
    counts it upsets are reported first, E_NOT_BALANCED), and with balanced=True a
    segment whose labels are not equally frequent is flagged (E_NOT_BALANCED)."""
    import torch
    offs = np.array([0, 4096 * 2 + 64, 4096 * 2 + 128, 4096 * 3 + 128], dtype=np.int64)
    w = np.array([32, 64, 128], dtype=np.int32)
    keys = np.concatenate([np.tile(np.arange(int(w[s]), dtype=np.uint32), int(offs[s + 1] - offs[s]) // int(w[s]))
                           for s in range(3)])
    keys = np.concatenate([synth.rng(s).permutation(keys[offs[s]:offs[s + 1]]) for s in range(3)]).astype(np.uint32)
    od, wd = torch.from_numpy(offs).cuda(), dev(w)
    _seg_part_case(bcf, keys, None, offs, w, balanced)  # well-formed: OK
    bad = keys.copy()
    bad[int(offs[1]) + 7] = 64  # segment 1 has width 64 (and, balanced, one label fewer)
    bcf.segmented_partition(dev(bad), None, od, wd, balanced=balanced)
    assert bcf.get_status() == (bcf.E_NOT_BALANCED if balanced else bcf.E_BAD_KEY)  # both flagged when balanced
    if balanced:
        skew = keys.copy()
        skew[int(offs[2]) + 3] = (int(skew[int(offs[2]) + 3]) + 1) % 128  # one label one more, another one fewer
        bcf.segmented_partition(dev(skew), None, od, wd, balanced=True)
        assert bcf.get_status() == bcf.E_NOT_BALANCED


def test_segmented_partition_reports_bad_width(bcf):
    import torch
    offs = np.array([0, 64, 128], dtype=np.int64)
    w = np.array([32, 300], dtype=np.int32)
    bcf.segmented_partition(dev(synth.random_labels(128, 32, seed=1)), None,
                            torch.from_numpy(offs).cuda(), dev(w))
    assert bcf.get_status() == bcf.E_INVAL


# ------------------------------------------------------- row-local permute
def test_permute_rows_and_gather_rows(bcf):
    B, n = 5, 1003
    v = synth.float_bits_payload(B * n, seed=1)
    pi = np.concatenate([synth.random_perm(n, seed=10 + b) for b in range(B)])
    y = bcf.permute(dev(v), dev(pi), row_len=n)
    gpi = (np.repeat(np.arange(B), n) * n + pi).astype(np.uint32)
    assert bits_equal(host(y, np.float32), oracle.permute(v, gpi))
    z = bcf.gather(y, dev(pi), row_len=n)
    assert bits_equal(host(z, np.float32), oracle.gather(oracle.permute(v, gpi), gpi))
    assert bcf.get_status() == bcf.OK
    bad = pi.copy()
    bad[7] = n  # outside its row
    bcf.permute(dev(v), dev(bad), row_len=n)
    assert bcf.get_status() == bcf.E_BAD_PERM


def test_sort_index_payload(bcf):
    n = 3 * 4096 + 11
    keys = synth.zipf_keys(n, seed=5)
    ko, perm = bcf.sort(dev(keys), None, index_payload=True)
    rk, rv = oracle.sort_kv(keys, synth.index_payload(n))
    assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(perm, np.uint32), rv)
