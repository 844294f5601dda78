"""bcf_partition_noalloc: the partition for callers that cannot allocate device
memory when they call the library (inside stream capture, under a host
framework's memory pool, in allocation-free loops).  Its scratch is a fixed
array inside libbcf.so, so this file checks, through the C ABI, that two calls
in a row give exactly what the workspace-based bcf_partition gives (the array
keeps the previous call's contents, so the second call also checks that
everything that must start at zero is cleared).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from helpers import bits_equal, dev, host


def _raw(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_rejects_on_the_host():
    """Size and overlap errors come back before anything is launched (CPU)."""
    import paper_1507_01391_b300 as bcf
    L = bcf.lib()
    P = ctypes.c_void_p
    a, b = P(0x10000), P(0x20000)
    assert L.bcf_partition_noalloc(a, None, b, None, bcf.NOALLOC_MAX_N + 1, 32, 0, 0, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_noalloc(a, None, a, None, 1000, 32, 0, 0, None) == bcf.E_INVAL  # in place
    assert L.bcf_partition_noalloc(a, None, b, None, 1000, 300, 0, 0, None) == bcf.E_UNSUPPORTED
    assert L.bcf_partition_noalloc(a, None, b, None, 1001, 32, 0, bcf.ASSUME_BALANCED, None) == bcf.E_INVAL
    assert L.bcf_partition_noalloc(None, None, None, None, 0, 32, 0, 0, None) == bcf.OK


@pytest.mark.gpu
@pytest.mark.parametrize("w,balanced,n", [(32, True, 65536), (256, False, 3 * 4096 + 77), (7, False, 1 << 22)])
def test_noalloc_matches_workspace_partition_twice(w, balanced, n):
    import torch

    import paper_1507_01391_b300 as bcf
    L = bcf.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):  # two calls in a row share the library's scratch array
        keys = synth.partition_keys(n, w, seed=10 * call + w) if balanced else synth.random_labels(n, w, seed=call + n)
        k = dev(keys)
        v = dev(synth.index_payload(n))
        ko_a, vo_a = torch.empty_like(k), torch.empty_like(v)
        flags = bcf.ASSUME_BALANCED if balanced else 0
        rc = L.bcf_partition_noalloc(_raw(k), _raw(v), _raw(ko_a), _raw(vo_a), n, w, 4, flags, stream)
        assert rc == bcf.OK
        ko_b, vo_b = bcf.partition(k, v, w, balanced=balanced)
        assert bcf.get_status() == bcf.OK
        assert bits_equal(host(ko_a, np.uint32), host(ko_b, np.uint32))
        assert bits_equal(host(vo_a, np.uint32), host(vo_b, np.uint32))
