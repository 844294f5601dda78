"""GPU parity: the radix sort skips the digit passes whose digit is the same in
every key, on the device.  Keys built so that 0 to 4 of the four 8-bit digits
vary, out of place (where, with no digit varying, the last pass still runs and
copies the keys over) and in place (where an odd number of passes run ends in the
temporary and is copied home), with float payloads, position payloads and none,
on both sides of the small/large path boundary.  The result is compared bit by
bit with the oracle's stable sort and the number of passes run with the count of
varying digits."""
import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host

pytestmark = pytest.mark.gpu

# key = (random bits) & mask | fixed, so that digit d varies iff mask has bits in it
KINDS = {
    "uniform": (0xFFFFFFFF, 0, 4),
    "top_byte_constant": (0x00FFFFFF, 0x5A000000, 3),
    "second_byte_only": (0x0000FF00, 0x12000034, 1),
    "middle_bytes": (0x00FFFF00, 0x80000001, 2),
    "one_bit_in_top": (0x01000000, 0x00ABCDEF, 1),
    "all_equal": (0, 0xCAFEF00D, 0),
}


@pytest.fixture(scope="module")
def bcf():
    import paper_1507_01391_b300 as m
    m.lib()
    return m


def _expected_passes(kind, in_place):
    """Passes whose digit varies; out of place, with none, the last pass still runs
    (a stable pass over equal digits copies the input to the output)."""
    k = KINDS[kind][2]
    return k if (k or in_place) else 1


def _keys(n, kind, seed):
    mask, fixed, _ = KINDS[kind]
    return ((synth.uniform_keys(n, seed=seed) & np.uint32(mask)) | np.uint32(fixed)).astype(np.uint32)


@pytest.mark.parametrize("n", [1000, 3 * 4096 + 5, (1 << 18) + 1, 700_001])
@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("payload", ["float", "index", "none"])
def test_sort_skips_constant_digits(bcf, n, kind, in_place, payload):
    keys = _keys(n, kind, seed=n + len(kind))
    vals = synth.float_bits_payload(n, seed=n) if payload == "float" else None
    kd = dev(keys)
    vd = None if vals is None else dev(vals)
    vb = 0 if payload == "none" else 4
    ws = bcf.workspace(bcf.sort_workspace_size(n, vb, 32))
    if in_place:
        vo_in = vd if payload == "float" else (dev(np.zeros(n, np.uint32)) if payload == "index" else None)
        ko, vo = bcf.sort(kd, vd, keys_out=kd, vals_out=vo_in, ws=ws, index_payload=payload == "index")
    else:
        ko, vo = bcf.sort(kd, vd, ws=ws, index_payload=payload == "index")
    assert bcf.get_status() == bcf.OK
    assert bcf.sort_passes_run(ws, n, vb, 32) == _expected_passes(kind, in_place)
    ref_vals = vals if payload == "float" else (synth.index_payload(n) if payload == "index" else None)
    rk, rv = oracle.sort_kv(keys, ref_vals)
    assert bits_equal(host(ko, np.uint32), rk)
    if payload == "float":
        assert bits_equal(host(vo, np.float32), rv)
    elif payload == "index":
        assert bits_equal(host(vo, np.uint32), rv)


@pytest.mark.parametrize("key_bits", [20, 24])
def test_sort_skips_with_fewer_key_bits(bcf, key_bits):
    """key_bits < 32 plans fewer passes (key bytes 0..2 for 20 and 24 bits); keys
    below 2^16 leave the pass of byte 2 without a varying digit."""
    n = 300_001
    keys = synth.uniform_keys(n, seed=3, bits=16)
    vals = synth.index_payload(n)
    ws = bcf.workspace(bcf.sort_workspace_size(n, 4, key_bits))
    ko, vo = bcf.sort(dev(keys), dev(vals), key_bits=key_bits, ws=ws)
    assert bcf.get_status() == bcf.OK
    # 20 and 24 bits: digits at shifts 0, 8, 16 (bits 16-23 never vary)
    assert bcf.sort_passes_run(ws, n, 4, key_bits) == 2
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(ko, np.uint32), rk)
    assert bits_equal(host(vo, np.uint32), rv)


def test_sort_skip_in_a_cuda_graph(bcf):
    """The skip is decided on the device: a captured sort replayed on new keys with
    other constant digits still sorts them."""
    import torch
    n = 300_001
    kd = dev(_keys(n, "uniform", 1))
    vd = dev(synth.index_payload(n))
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    ws = bcf.workspace(bcf.sort_workspace_size(n, 4, 32))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bcf.sort(kd, vd, keys_out=ko, vals_out=vo, ws=ws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bcf.sort(kd, vd, keys_out=ko, vals_out=vo, ws=ws, stream=s)
    for kind in ("second_byte_only", "middle_bytes", "uniform", "all_equal"):
        keys = _keys(n, kind, 7)
        kd.copy_(dev(keys))
        g.replay()
        torch.cuda.synchronize()
        assert bcf.get_status() == bcf.OK
        assert bcf.sort_passes_run(ws, n, 4, 32) == _expected_passes(kind, False)
        rk, rv = oracle.sort_kv(keys, synth.index_payload(n))
        assert bits_equal(host(ko, np.uint32), rk)
        assert bits_equal(host(vo, np.uint32), rv)


@pytest.mark.parametrize("n", [5000, 300_001])
@pytest.mark.parametrize("kind", ["top_byte_constant", "second_byte_only", "all_equal"])
def test_sort_skip_in_place_8_byte_payloads(bcf, n, kind):
    """In place with 8-byte payloads: 3 or 1 passes run (odd), so the result is
    copied home from the temporary, payload words included; with none, nothing
    moves."""
    keys = _keys(n, kind, seed=n + 3)
    vals = synth.uniform_keys(2 * n, seed=n + 4).view(np.uint64)
    kd, vd = dev(keys), dev(vals)
    ws = bcf.workspace(bcf.sort_workspace_size(n, 8, 32))
    ko, vo = bcf.sort(kd, vd, keys_out=kd, vals_out=vd, ws=ws)
    assert bcf.get_status() == bcf.OK
    assert bcf.sort_passes_run(ws, n, 8, 32) == _expected_passes(kind, True)
    rk, rv = oracle.sort_kv(keys, vals)
    assert bits_equal(host(ko, np.uint32), rk)
    assert bits_equal(host(vo, np.uint64), rv)


@pytest.mark.parametrize("config", [4, 5, 6, 7])
@pytest.mark.parametrize("kind", ["uniform", "middle_bytes", "top_byte_constant", "one_bit_in_top"])
def test_counts_pass_forms_skip_passes(bcf, config, kind):
    """Every counts + scan + pass body configuration (tile shapes 256x16, 256x8,
    512x12, 384x16) with passes skipped on the device: whole groups of four count
    tiles and a ragged tail, bit-exact against the oracle."""
    L = bcf.lib()
    n = 5 * 16384 + 1234
    lg = (n - 1).bit_length()
    assert L.bcf_tune_config_form(config) == 1
    assert L.bcf_tune_set(bcf.OP_SORT, lg, config) == bcf.OK
    try:
        keys = _keys(n, kind, seed=config * 7 + len(kind))
        vals = synth.float_bits_payload(n, seed=config)
        ws = bcf.workspace(bcf.sort_workspace_size(n, 4, 32))
        ko, vo = bcf.sort(dev(keys), dev(vals), ws=ws)
        assert bcf.get_status() == bcf.OK
        assert bcf.sort_passes_run(ws, n, 4, 32) == _expected_passes(kind, False)
        rk, rv = oracle.sort_kv(keys, vals)
        assert bits_equal(host(ko, np.uint32), rk) and bits_equal(host(vo, np.uint32), rv)
    finally:
        L.bcf_tune_set(bcf.OP_SORT, lg, -1)
