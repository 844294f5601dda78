"""bcf_partition_noalloc: the partition for callers that cannot allocate device
memory when they call the library (inside stream capture, under a host
framework's memory pool, in allocation-free loops).  Its scratch is a fixed
array inside libbcf.so, so this file checks, through the C ABI, that two calls
in a row give exactly what the CPU oracle and the workspace-based bcf_partition
give (the array keeps the previous call's contents, so the second call also
checks that everything that must start at zero is cleared), and that the call
can be captured in a CUDA graph and replayed with new inputs.  Collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import bits_equal, dev, host


def _raw(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_rejects_on_the_host():
    """Size, flag and overlap errors come back before anything is launched (CPU)."""
    import paper_1507_01391_b300 as bcf
    L = bcf.lib()
    P = ctypes.c_void_p
    a, b = P(0x10000), P(0x20000)
    assert L.bcf_partition_noalloc(a, None, b, None, bcf.NOALLOC_MAX_N + 1, 32, 0, 0, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_noalloc(a, None, a, None, 1000, 32, 0, 0, None) == bcf.E_INVAL  # in place
    assert L.bcf_partition_noalloc(a, None, b, None, 1000, 300, 0, 0, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_noalloc(a, None, b, None, 1001, 32, 0, bcf.ASSUME_BALANCED, None) == bcf.E_INVAL
    # only BCF_ASSUME_BALANCED is honoured: the Lemma 1 schedule is refused, not ignored
    assert L.bcf_partition_noalloc(a, None, b, None, 1024, 32, 0, bcf.PARTITION_LEMMA1, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_noalloc(None, None, None, None, 0, 32, 0, 0, None) == bcf.OK


@pytest.mark.gpu
@pytest.mark.parametrize("w,balanced,n", [(32, True, 65536), (256, False, 3 * 4096 + 77), (7, False, 1 << 22)])
def test_noalloc_matches_oracle_and_workspace_partition_twice(w, balanced, n):
    import torch

    import paper_1507_01391_b300 as bcf
    L = bcf.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):  # two calls in a row share the library's scratch array
        keys = synth.partition_keys(n, w, seed=10 * call + w) if balanced else synth.random_labels(n, w, seed=call + n)
        vals = synth.index_payload(n)
        k = dev(keys)
        v = dev(vals)
        ko_a, vo_a = torch.empty_like(k), torch.empty_like(v)
        flags = bcf.ASSUME_BALANCED if balanced else 0
        rc = L.bcf_partition_noalloc(_raw(k), _raw(v), _raw(ko_a), _raw(vo_a), n, w, 4, flags, stream)
        assert rc == bcf.OK
        assert bcf.get_status() == bcf.OK
        rk, rv = oracle.partition_kv(keys, vals, w, balanced=balanced)
        assert bits_equal(host(ko_a, np.uint32), rk) and bits_equal(host(vo_a, np.uint32), rv)
        ko_b, vo_b = bcf.partition(k, v, w, balanced=balanced)
        assert bcf.get_status() == bcf.OK
        assert bits_equal(host(ko_a, np.uint32), host(ko_b, np.uint32))
        assert bits_equal(host(vo_a, np.uint32), host(vo_b, np.uint32))


@pytest.mark.gpu
@pytest.mark.parametrize("vb,n", [(4, 5000), (8, 300_001)])
def test_noalloc_captured_in_a_graph(vb, n):
    """One warm-up call (it looks the scratch address up), then the call captured on
    a non-default stream and replayed twice with new inputs copied into the
    captured buffers; every replay's output matches the oracle.  vb = 4 runs with
    vals NULL (the payload is the input position), vb = 8 with 8-byte payloads."""
    import torch

    import paper_1507_01391_b300 as bcf
    L = bcf.lib()
    w = 64
    k = torch.empty(n, dtype=torch.int32, device="cuda")
    v = None if vb == 4 else torch.empty(n, dtype=torch.int64, device="cuda")
    ko = torch.empty_like(k)
    vo = torch.empty(n, dtype=torch.int32 if vb == 4 else torch.int64, device="cuda")

    def inputs(seed):
        keys = synth.random_labels(n, w, seed=seed)
        vals = synth.index_payload(n) if vb == 4 else synth.uniform_keys(2 * n, seed=seed + 1).view(np.uint64)
        return keys, vals

    def call(s):
        return L.bcf_partition_noalloc(_raw(k), _raw(v), _raw(ko), _raw(vo), n, w, vb, 0,
                                       ctypes.c_void_p(s.cuda_stream))

    keys, vals = inputs(1)
    k.copy_(dev(keys))
    if v is not None:
        v.copy_(dev(vals))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        assert call(s) == bcf.OK  # warm-up, outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert call(s) == bcf.OK
    for seed in (2, 3):
        keys, vals = inputs(seed)
        k.copy_(dev(keys))
        if v is not None:
            v.copy_(dev(vals))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert bcf.get_status() == bcf.OK
        rk, rv = oracle.partition_kv(keys, vals if vb == 8 else synth.index_payload(n), w)
        assert bits_equal(host(ko, np.uint32), rk)
        assert bits_equal(host(vo, np.uint32 if vb == 4 else np.uint64), rv)
