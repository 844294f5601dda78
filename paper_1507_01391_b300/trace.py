"""Shared-memory access traces from the trace build (libbcf_trace.so).

``capture(fn)`` runs ``fn()`` with the binding switched to libbcf_trace.so (the
same kernels compiled with -DBCF_TRACE) and returns the recorded accesses as a
numpy array of shape (N, 4): request id, lane, shared byte address, and
width | store << 8 | site << 16 (see include/bcf_trace.h).  Replaying the records
through a bank model counts the bank conflicts of each traced kernel.
"""
from __future__ import annotations

import contextlib
import ctypes
import os

import numpy as np

from . import _SIGS, _PKG, BcfError, OK

TRACE_LIB_PATH = os.path.join(_PKG, "libbcf_trace.so")

# access sites (mirrors csrc/trace.cuh)
SITES = {
    "stage_read": 1, "count_atom": 2, "claim_atom": 3, "scatter": 4, "writeout_read": 5,
    "offset_read": 6, "hist_atom": 7, "hist_sum": 8, "warp_offsets": 9, "l1_row_ld": 10, "l1_row_st": 11, "l1_convert": 12, "l1_io": 13,
    "tile_count_atom": 14, "tile_count_sum": 15,
    "col_table": 20, "col_send": 21, "col_read": 22, "col_finish": 23, "col_pack": 24,
    "barrier": 30,
    "l2_square": 40, "l2_convert": 41, "l2_divide": 42, "l2_column": 43, "l2_rows": 44, "l2_shifted": 45,
    "l2_io": 47, "probe": 50,
}

_trace_lib = None


def load() -> ctypes.CDLL:
    global _trace_lib
    if _trace_lib is None:
        if not os.path.exists(TRACE_LIB_PATH):
            raise ImportError("libbcf_trace.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(TRACE_LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        L.bcf_trace_begin.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
        L.bcf_trace_begin.restype = ctypes.c_int
        L.bcf_trace_end.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.bcf_trace_end.restype = ctypes.c_int
        L.bcf_trace_bank_probe.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [
            ctypes.c_void_p]
        L.bcf_trace_bank_probe.restype = ctypes.c_int
        _trace_lib = L
    return _trace_lib


@contextlib.contextmanager
def _using(lib):
    import paper_1507_01391_b300 as bcf
    saved = bcf._lib
    bcf._lib = lib
    try:
        yield
    finally:
        bcf._lib = saved


def capture(fn, max_records: int = 1 << 22):
    """Run fn() on the trace build and return (records, total_recorded)."""
    import torch
    L = load()
    buf = torch.zeros(16 + 16 * max_records, dtype=torch.uint8, device="cuda")
    rc = L.bcf_trace_begin(ctypes.c_void_p(buf.data_ptr()), buf.numel())
    if rc != OK:
        raise BcfError(rc, "bcf_trace_begin")
    try:
        with _using(L):
            fn()
    finally:
        n = ctypes.c_uint64(0)
        rc = L.bcf_trace_end(ctypes.byref(n))
    if rc != OK:
        raise BcfError(rc, "bcf_trace_end")
    total = int(n.value)
    kept = min(total, max_records)
    rec = buf[16:16 + 16 * kept].cpu().numpy().view(np.uint32).reshape(kept, 4)
    return rec, total


def fields(rec):
    """Split records into (request, lane, address, width, store, site) arrays
    (barrier records have store 3, or 4 for a warp barrier, and width 0)."""
    return (rec[:, 0].astype(np.int64), (rec[:, 1] & 31).astype(np.int32), rec[:, 2].astype(np.uint32),
            (rec[:, 3] & 0xFF).astype(np.int32), ((rec[:, 3] >> 8) & 0xFF).astype(np.int32),
            (rec[:, 3] >> 16).astype(np.int32))


def accesses(rec):
    """The records without the barrier ones."""
    return rec[((rec[:, 3] >> 8) & 0xFF) < 3]
