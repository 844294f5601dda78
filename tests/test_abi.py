"""The C ABI library loads and exports every function include/bcf.h declares, and
its host-side argument checks reject bad calls before touching the GPU.  CPU only:
no call here launches a kernel."""
import ctypes
import os
import subprocess

import pytest

import paper_1507_01391_b300 as bcf


def test_library_exports_every_header_function():
    L = bcf.lib()
    names = bcf.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(names) == set(bcf._SIGS)


def test_exports_listed_by_nm():
    out = subprocess.run(["nm", "-D", "--defined-only", bcf._LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(bcf.header_functions()) <= exported


def test_status_strings_and_version():
    L = bcf.lib()
    for code in range(9):
        assert L.bcf_status_string(code)
    assert L.bcf_status_string(99) == b"unknown status"
    assert L.bcf_version() >= 10000


def test_workspace_queries():
    L = bcf.lib()
    sz = ctypes.c_size_t(0)
    assert L.bcf_sort_workspace_size(1 << 20, 4, 32, ctypes.byref(sz)) == bcf.OK
    assert sz.value >= (1 << 20) * 8  # ping-pong buffers for keys and values
    assert L.bcf_sort_workspace_size(-1, 4, 32, ctypes.byref(sz)) == bcf.E_INVAL
    assert L.bcf_sort_workspace_size(10, 3, 32, ctypes.byref(sz)) == bcf.E_INVAL
    assert L.bcf_sort_workspace_size(10, 4, 33, ctypes.byref(sz)) == bcf.E_INVAL
    assert L.bcf_sort_workspace_size(1 << 30, 4, 32, ctypes.byref(sz)) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_workspace_size(4096, 257, 4, 0, ctypes.byref(sz)) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_workspace_size(4096, 0, 4, 0, ctypes.byref(sz)) == bcf.E_INVAL
    assert L.bcf_permute_workspace_size(100, 0, 0, ctypes.byref(sz)) == bcf.OK and sz.value == 0
    assert L.bcf_permute_workspace_size(100, 0, bcf.CHECK_PERM, ctypes.byref(sz)) == bcf.OK and sz.value >= 16
    # bucketed form: pi's low bits (2 B), keys (4 B) and payloads (vb) per element
    assert L.bcf_permute_workspace_size(1 << 20, 4, bcf.PERMUTE_BUCKETED, ctypes.byref(sz)) == bcf.OK
    assert sz.value >= 10 << 20
    assert L.bcf_permute_workspace_size(1 << 20, 0, bcf.PERMUTE_BUCKETED, ctypes.byref(sz)) == bcf.OK
    assert (6 << 20) <= sz.value < (10 << 20)
    # beyond 2^26 elements, or with 8-byte payloads, the one-pass scatter runs: no bucketed region
    assert L.bcf_permute_workspace_size((1 << 26) + 1, 4, bcf.PERMUTE_BUCKETED, ctypes.byref(sz)) == bcf.OK
    assert sz.value == 0
    assert L.bcf_permute_workspace_size(1 << 20, 8, bcf.PERMUTE_BUCKETED, ctypes.byref(sz)) == bcf.OK
    assert sz.value == 0
    assert L.bcf_permute_workspace_size(100, 3, 0, ctypes.byref(sz)) == bcf.E_INVAL
    assert L.bcf_partition_splitters_workspace_size(1 << 20, 255, 4, 0, ctypes.byref(sz)) == bcf.OK
    assert sz.value >= 8 << 20  # room for an in-place copy of keys and payloads
    assert L.bcf_partition_splitters_workspace_size(100, 256, 4, 0, ctypes.byref(sz)) == bcf.E_UNSUPPORTED


def test_argument_checks_reject_without_launching():
    """Null, misaligned or overlapping pointers fail on the host: fake addresses
    are safe here because nothing is launched for a rejected call."""
    L = bcf.lib()
    P = ctypes.c_void_p
    a, b, ws = P(0x10000), P(0x20000), P(0x40000)
    mis = P(0x10004)
    assert L.bcf_sort(None, None, b, None, 10, 0, 32, ws, 1 << 20, None) == bcf.E_INVAL
    assert L.bcf_sort(mis, None, b, None, 10, 0, 32, ws, 1 << 20, None) == bcf.E_INVAL
    assert L.bcf_sort(a, None, b, None, 10, 0, 32, ws, 8, None) == bcf.E_WORKSPACE
    assert L.bcf_sort(a, None, P(0x10008), None, 10, 0, 32, ws, 1 << 20, None) == bcf.E_INVAL
    assert L.bcf_sort(a, None, b, None, 10, 4, 32, ws, 1 << 20, None) == bcf.E_INVAL  # vals missing
    assert L.bcf_partition(a, None, b, None, 10, 3, 0, bcf.ASSUME_BALANCED, ws, 1 << 20, None) == bcf.E_INVAL
    assert L.bcf_partition(a, None, b, None, 10, 300, 0, 0, ws, 1 << 20, None) == bcf.E_UNSUPPORTED
    # the direct write-out serves at most 32 labels, and not with the Lemma 1 schedule
    assert L.bcf_partition(a, None, b, None, 64, 33, 0, bcf.PARTITION_DIRECT, ws, 1 << 20, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition(a, None, b, None, 64, 32, 0, bcf.PARTITION_DIRECT | bcf.PARTITION_LEMMA1, ws, 1 << 20,
                           None) == bcf.E_UNSUPPORTED
    assert L.bcf_permute(a, P(0x10010), b, 64, 0, 4, 0, None, 0, None) == bcf.E_INVAL  # overlap
    assert L.bcf_permute(a, b, None, 64, 0, 4, 0, None, 0, None) == bcf.E_INVAL
    assert L.bcf_permute(a, b, ws, 64, 0, 3, 0, None, 0, None) == bcf.E_INVAL
    assert L.bcf_permute(a, b, ws, 64, -1, 4, 0, None, 0, None) == bcf.E_INVAL
    assert L.bcf_permute(a, b, ws, 64, 0, 4, bcf.CHECK_PERM, None, 0, None) == bcf.E_INVAL
    assert L.bcf_permute_tiles(a, b, ws, 64, 1000, 0, 0, None) == bcf.E_INVAL
    assert L.bcf_gather(a, b, ws, 64, 64, 0, 2, None) == bcf.E_INVAL
    # empty inputs are valid no-ops
    assert L.bcf_sort(None, None, None, None, 0, 0, 32, None, 0, None) == bcf.OK
    assert L.bcf_permute(None, None, None, 0, 0, 4, 0, None, 0, None) == bcf.OK
    # segmented forms: out-of-place only, offsets required
    assert L.bcf_segmented_sort(a, None, a, None, 10, ws, 1, 0, 32, ws, 1 << 30, None) == bcf.E_INVAL
    assert L.bcf_segmented_sort(a, None, b, None, 10, None, 1, 0, 32, ws, 1 << 30, None) == bcf.E_INVAL
    assert L.bcf_segmented_sort(a, None, b, None, 10, ws, 1, 0, 32, ws, 8, None) == bcf.E_WORKSPACE
    assert L.bcf_sort_tiles(a, None, b, None, 10, 1024, 0, None) == bcf.E_INVAL
    assert L.bcf_sort_tiles(a, None, a, None, 10, 4096, 0, None) == bcf.E_INVAL
    # Lemma 2 partition: whole 32768-item matrices, 16-byte aligned, below 2^32 items
    c, d = P(0x1000000), P(0x2000000)
    assert L.bcf_partition_lemma2(a, None, b, c, 32768 + 4, None) == bcf.E_INVAL
    assert L.bcf_partition_lemma2(mis, None, b, c, 32768, None) == bcf.E_INVAL
    assert L.bcf_partition_lemma2(a, None, b, None, 32768, None) == bcf.E_INVAL  # no payload output
    assert L.bcf_partition_lemma2(a, c, b, c, 32768, None) == bcf.E_INVAL  # keys out of place, payloads in place
    assert L.bcf_partition_lemma2(a, c, b, d, 1 << 32, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_lemma2(None, None, None, None, 0, None) == bcf.OK


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib.util
    spec = importlib.util.spec_from_file_location("bcf_copy", os.path.join(os.path.dirname(bcf.__file__), "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    monkeypatch.setattr(mod, "_LIB_PATH", str(tmp_path / "missing.so"))
    mod._lib = None
    with pytest.raises(ImportError):
        mod.lib()


def test_trace_build_exports_both_headers():
    """libbcf_trace.so (the same kernels compiled with -DBCF_TRACE) exports the
    library functions and the trace functions; libbcf.so has no trace code."""
    import re
    hdr = os.path.join(os.path.dirname(bcf.HEADER), "bcf_trace.h")
    text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
    trace_names = set(re.findall(r"\b(bcf_[a-z0-9_]+)\s*\(", text))
    assert trace_names == {"bcf_trace_begin", "bcf_trace_end", "bcf_trace_bank_probe"}
    nm = lambda p: {l.split()[-1] for l in subprocess.run(["nm", "-D", "--defined-only", p], capture_output=True,
                                                          text=True).stdout.splitlines() if " T " in l}
    tlib = os.path.join(os.path.dirname(bcf._LIB_PATH), "libbcf_trace.so")
    assert set(bcf.header_functions()) | trace_names <= nm(tlib)
    assert not (trace_names & nm(bcf._LIB_PATH))


def test_tuning_table_on_the_host():
    """The tuning table is host state: set/get need no GPU."""
    L = bcf.lib()
    nconf = L.bcf_tune_num_configs()
    assert nconf >= 2
    t, k = ctypes.c_int(0), ctypes.c_int(0)
    tiles = set()
    for c in range(nconf):
        assert L.bcf_tune_config_info(c, ctypes.byref(t), ctypes.byref(k)) == bcf.OK
        assert t.value % 32 == 0 and t.value >= 256 and k.value >= 1
        form = L.bcf_tune_config_form(c)
        assert form in (0, 1, 2)
        tiles.add((t.value, k.value, form))
    assert min(a * b for a, b, _ in tiles) >= 1024 and len(tiles) == nconf
    assert L.bcf_tune_config_form(0) == 0 and L.bcf_tune_config_form(nconf - 1) == 2
    assert L.bcf_tune_config_form(nconf) == bcf.E_INVAL
    assert L.bcf_tune_config_info(nconf, ctypes.byref(t), ctypes.byref(k)) == bcf.E_INVAL
    got = ctypes.c_int(-5)
    assert L.bcf_tune_get(bcf.OP_SORT, 1 << 26, ctypes.byref(got)) == bcf.OK and got.value == 4
    assert L.bcf_tune_get(bcf.OP_PARTITION, 1 << 26, ctypes.byref(got)) == bcf.OK and got.value == 4
    assert L.bcf_tune_get(bcf.OP_PARTITION, 1 << 16, ctypes.byref(got)) == bcf.OK and got.value == 1
    assert L.bcf_tune_get(bcf.OP_SORT, 1 << 12, ctypes.byref(got)) == bcf.OK and got.value == 11
    assert L.bcf_tune_set(bcf.OP_SORT, 26, nconf - 1) == bcf.OK
    assert L.bcf_tune_get(bcf.OP_SORT, (1 << 25) + 1, ctypes.byref(got)) == bcf.OK and got.value == nconf - 1
    assert L.bcf_tune_set(bcf.OP_SORT, 26, -1) == bcf.OK  # back to the size rule
    assert L.bcf_tune_get(bcf.OP_SORT, 1 << 26, ctypes.byref(got)) == bcf.OK and got.value == 4
    assert L.bcf_tune_set(bcf.OP_SORT, 64, 0) == bcf.E_INVAL
    assert L.bcf_tune_set(bcf.OP_SORT, 3, nconf) == bcf.E_INVAL
    assert L.bcf_tune_set(7, 3, 0) == bcf.E_INVAL
    # the cache file needs the device's name, so only the argument checks run here
    applied = ctypes.c_int(-1)
    assert L.bcf_tune_save(None) == bcf.E_INVAL
    assert L.bcf_tune_load(None, ctypes.byref(applied)) == bcf.E_INVAL


def test_lookback_testing_aid_arguments():
    """bcf_debug_lookback is host state: a silent tile needs a poll limit."""
    L = bcf.lib()
    assert L.bcf_debug_lookback(3, 0) == bcf.E_INVAL
    assert L.bcf_debug_lookback(-1, 0) == bcf.OK


def test_batched_sort_tuning_entries():
    """The batched sort's table takes only the 256 x 16 counts + scan forms and
    defaults to the pass body fed scanned offsets (host only)."""
    L = bcf.lib()
    c = ctypes.c_int(-5)
    assert L.bcf_tune_get(bcf.OP_SEGMENTED_SORT, 1 << 28, ctypes.byref(c)) == bcf.OK and c.value == 4
    assert L.bcf_tune_get(bcf.OP_SEGMENTED_SORT, 100, ctypes.byref(c)) == bcf.OK and c.value == 4
    for cfg, ok in [(4, True), (8, True), (0, False), (1, False), (5, False), (9, False), (10, False)]:
        assert (L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, 20, cfg) == bcf.OK) == ok, cfg
    assert L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, 20, 8) == bcf.OK
    assert L.bcf_tune_get(bcf.OP_SEGMENTED_SORT, 1 << 20, ctypes.byref(c)) == bcf.OK and c.value == 8
    assert L.bcf_tune_set(bcf.OP_SEGMENTED_SORT, 20, -1) == bcf.OK
    assert L.bcf_tune_get(bcf.OP_SEGMENTED_SORT, 1 << 20, ctypes.byref(c)) == bcf.OK and c.value == 4
    assert L.bcf_tune_set(3, 20, 4) == bcf.E_INVAL
    assert L.bcf_tune_get(3, 1 << 20, ctypes.byref(c)) == bcf.E_INVAL


def test_bank_probe_argument_checks():
    """The probe entry point rejects bad arguments before launching (CPU)."""
    from paper_1507_01391_b300 import trace
    L = trace.load()
    P = ctypes.c_void_p
    a, b = P(0x10000), P(0x20000)
    assert L.bcf_trace_bank_probe(9, 0, 0, a, b, 1, 1, None) == bcf.E_INVAL
    assert L.bcf_trace_bank_probe(0, 4, 0, a, b, 1, 1, None) == bcf.E_INVAL
    assert L.bcf_trace_bank_probe(-1, 0, 0, a, b, 1, 1, None) == bcf.E_INVAL
    assert L.bcf_trace_bank_probe(0, 0, 0, None, b, 1, 1, None) == bcf.E_INVAL
    assert L.bcf_trace_bank_probe(0, 0, 0, a, b, 0, 1, None) == bcf.E_INVAL
    assert L.bcf_trace_bank_probe(0, 0, 0, a, b, 1, 0, None) == bcf.E_INVAL
