"""CPU oracle -- TEST INFRASTRUCTURE ONLY, never part of the library's product path.

Plain, slow and obviously correct definitions of what the bank-conflict-free
library computes (Afshani & Sitchinava, "Sorting and Permuting without Bank
Conflicts on GPUs"): stable sort, stable counting partition, permutation scatter,
tile-local permutation and gather, their segmented forms, models of the Lemma 1
schedule and of Lemma 2's 0-1 partition (Sec. 2) and of the bank model (Sec. 1, "Model of Computation").

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
this package.  It is written in plain C (``bcf_oracle.c``) and shares no code with
the CUDA library; this module only compiles it with gcc and marshals numpy arrays.

Pins: every function here is checked against something other than itself in
``tests/test_oracle_pins.py`` (brute force, closed forms, invariants, library
routines).  The strict bank rule has no paper-printed example; it is pinned by the
closed forms the paper states for strided and contiguous access.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcf_oracle.c")
_HDR = os.path.join(_HERE, "bcf_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, E_KEY, E_BALANCE, E_PERM, E_ARG, E_NOMEM = 0, -1, -2, -3, -4, -5


class OracleError(RuntimeError):
    pass


def build(src: str = _SRC, out: str = _LIB, force: bool = False) -> str:
    """Compile the oracle's C source into a shared object with gcc."""
    stale = (not os.path.exists(out)) or any(
        os.path.getmtime(p) > os.path.getmtime(out) for p in (src, _HDR))
    if force or stale:
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-I", _HERE, "-o", tmp, src])
        os.replace(tmp, out)
    return out


def load(path: str | None = None) -> ctypes.CDLL:
    lib = ctypes.CDLL(path or build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    sig = {
        "oracle_sort_kv": [P, P, P, P, I64, I],
        "oracle_stable_rank": [P, I64, I64],
        "oracle_partition_kv": [P, P, P, P, I64, I64, I, I],
        "oracle_partition_splitters": [P, P, P, P, I64, P, I64, I, I],
        "oracle_permute": [P, P, P, I64, I],
        "oracle_permute_tiles": [P, P, P, I64, I64],
        "oracle_gather": [P, P, P, I64, I64, I],
        "oracle_segmented_sort_kv": [P, P, P, P, P, I64, I],
        "oracle_segmented_partition_kv": [P, P, P, P, P, P, I64, I, I],
        "oracle_l1_sort_rows": [P, I64, I64, I],
        "oracle_l1_row_to_col": [P, I64, I64],
        "oracle_l1_col_to_row": [P, I64, I64],
        "oracle_lemma1_sort": [P, I64, I64],
        "oracle_lemma2_partition": [P, P, I64, I64, I],
        "oracle_l2_sort_colmajor": [P, P, I64, P, I64],
        "oracle_l2_sort_rowmajor": [P, P, I64, I64, I64],
        "oracle_race_check": [P, I64, P, P],
        "oracle_bank_count": [P, P, P, P, I64, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int64 if name == "oracle_stable_rank" else ctypes.c_int
        if name.startswith("oracle_l1_") and name != "oracle_lemma1_sort":
            f.restype = None
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != OK:
        raise OracleError("oracle rejected its input (code %d)" % rc)


def _vb(vals):
    return 0 if vals is None else vals.dtype.itemsize


def sort_kv(keys, vals=None, L=None):
    """Stable ascending sort of (key, payload) pairs; returns (keys, vals)."""
    L = L or lib()
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    vals = None if vals is None else np.ascontiguousarray(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    _check(L.oracle_sort_kv(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.size, _vb(vals)))
    return ko, vo


def stable_rank(keys, i, L=None):
    L = L or lib()
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    return int(L.oracle_stable_rank(_ptr(keys), keys.size, int(i)))


def partition_kv(keys, vals, w, balanced=False, L=None):
    L = L or lib()
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    vals = None if vals is None else np.ascontiguousarray(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    _check(L.oracle_partition_kv(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.size,
                                 int(w), int(bool(balanced)), _vb(vals)))
    return ko, vo


def partition_splitters(keys, vals, splitters, balanced=False, L=None):
    """Stable partition of the keys (and payloads) into len(splitters) + 1 buckets,
    bucket = number of splitters <= key."""
    L = L or lib()
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    spl = np.ascontiguousarray(splitters, dtype=np.uint32)
    vals = None if vals is None else np.ascontiguousarray(vals)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    _check(L.oracle_partition_splitters(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.size,
                                        _ptr(spl), spl.size, int(bool(balanced)), _vb(vals)))
    return ko, vo


def permute(src, pi, L=None):
    """out[pi[i]] = src[i] for any fixed-width element type."""
    L = L or lib()
    src = np.ascontiguousarray(src)
    pi = np.ascontiguousarray(pi, dtype=np.uint32)
    if pi.size != src.size:
        raise OracleError("pi and src differ in length")
    dst = np.empty_like(src)
    _check(L.oracle_permute(_ptr(src), _ptr(dst), _ptr(pi), src.size, src.dtype.itemsize))
    return dst


def permute_tiles(src, lpi, tile, L=None):
    L = L or lib()
    src = np.ascontiguousarray(src, dtype=np.uint32)
    lpi = np.ascontiguousarray(lpi, dtype=np.uint16)
    dst = np.empty_like(src)
    _check(L.oracle_permute_tiles(_ptr(src), _ptr(dst), _ptr(lpi), src.size, int(tile)))
    return dst


def gather(src, idx, L=None):
    L = L or lib()
    src = np.ascontiguousarray(src)
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    dst = np.empty(idx.size, dtype=src.dtype)
    _check(L.oracle_gather(_ptr(src), _ptr(dst), _ptr(idx), idx.size, src.size,
                           src.dtype.itemsize))
    return dst


def segmented_sort_kv(keys, vals, offs, L=None):
    L = L or lib()
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    vals = None if vals is None else np.ascontiguousarray(vals)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    _check(L.oracle_segmented_sort_kv(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), _ptr(offs),
                                      offs.size - 1, _vb(vals)))
    return ko, vo


def segmented_partition_kv(keys, vals, offs, w_per_seg, balanced=False, L=None):
    L = L or lib()
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    vals = None if vals is None else np.ascontiguousarray(vals)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    wps = np.ascontiguousarray(w_per_seg, dtype=np.int32)
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    _check(L.oracle_segmented_partition_kv(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo),
                                           _ptr(offs), _ptr(wps), offs.size - 1,
                                           int(bool(balanced)), _vb(vals)))
    return ko, vo


def l1_sort_rows(M, alternating, L=None):
    L = L or lib()
    assert M.dtype == np.uint32 and M.flags.c_contiguous
    L.oracle_l1_sort_rows(_ptr(M), M.shape[0], M.shape[1], int(bool(alternating)))


def l1_row_to_col(M, L=None):
    L = L or lib()
    L.oracle_l1_row_to_col(_ptr(M), M.shape[0], M.shape[1])


def l1_col_to_row(M, L=None):
    L = L or lib()
    L.oracle_l1_col_to_row(_ptr(M), M.shape[0], M.shape[1])


def lemma2_partition(lab, pay, stage=4, L=None):
    """Lemma 2's 0-1 partition of a w x m matrix (labels and payloads as (w, m)
    arrays); returns new (labels, payloads) after the given stage (4: all)."""
    L = L or lib()
    lab = np.array(lab, dtype=np.uint32, order="C", copy=True)
    pay = np.array(pay, dtype=np.uint32, order="C", copy=True)
    assert lab.shape == pay.shape and lab.ndim == 2
    _check(L.oracle_lemma2_partition(_ptr(lab), _ptr(pay), lab.shape[0], lab.shape[1], stage))
    return lab, pay


def l2_sort_colmajor(lab, pay, rows, L=None):
    """One step of Lemma 2: the rows listed, as a matrix, sorted in column-major order (in place)."""
    L = L or lib()
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    _check(L.oracle_l2_sort_colmajor(_ptr(lab), _ptr(pay), lab.shape[1], _ptr(rows), rows.size))


def l2_sort_rowmajor(lab, pay, r0, h, L=None):
    """One step of Lemma 2: rows [r0, r0 + h) sorted in row-major order (in place)."""
    L = L or lib()
    _check(L.oracle_l2_sort_rowmajor(_ptr(lab), _ptr(pay), lab.shape[1], r0, h))


def lemma1_sort(M, L=None):
    """Lemma 1 on a w x m matrix (returns a sorted copy, read row by row)."""
    L = L or lib()
    M = np.array(M, dtype=np.uint32, order="C", copy=True)
    _check(L.oracle_lemma1_sort(_ptr(M), M.shape[0], M.shape[1]))
    return M


def theorem1_sort(M, record=None, L=None):
    """Theorem 1 (Sec. 2) on an m x m matrix, m a perfect square: super-rows of
    sqrt(m) adjacent rows each sorted by Lemma 1; columns sorted ascending; super-
    rows sorted again in alternating order (super-row 0 ascending); columns sorted;
    rows sorted.  Returns the matrix, sorted in row-major order.  `record`, if
    given, receives a copy of the matrix after each of the five steps."""
    L = L or lib()
    M = np.array(M, dtype=np.uint32, order="C", copy=True)
    m = M.shape[0]
    r = int(round(m ** 0.5))
    if M.shape != (m, m) or r * r != m:
        raise OracleError("Theorem 1 needs a square matrix whose side is a perfect square")

    def sort_super_rows(alternating):
        for g in range(r):
            blk = np.ascontiguousarray(M[g * r:(g + 1) * r])
            _check(L.oracle_lemma1_sort(_ptr(blk), r, m))  # ascending, row-major
            if alternating and g % 2 == 1:
                blk = blk.reshape(-1)[::-1].reshape(r, m)  # descending order
            M[g * r:(g + 1) * r] = blk

    def note():
        if record is not None:
            record.append(M.copy())

    sort_super_rows(False)
    note()
    M[:] = np.sort(M, axis=0)  # columns ascending (top to bottom)
    note()
    sort_super_rows(True)
    note()
    M[:] = np.sort(M, axis=0)
    note()
    M[:] = np.sort(M, axis=1)  # rows ascending
    note()
    return M


def race_check(rec, L=None):
    """(racing words, words checked) of a shared-memory trace: records (N, 4) of
    uint32 as the trace build writes them (request, thread | block << 16, address,
    width | kind << 8 | site << 16)."""
    L = L or lib()
    rec = np.ascontiguousarray(rec, dtype=np.uint32)
    races, words = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(L.oracle_race_check(_ptr(rec), rec.shape[0], ctypes.byref(races), ctypes.byref(words)))
    return races.value, words.value


def bank_count(req, lane, addr, width, L=None):
    """Return (hw_wavefronts, hw_conflicts, strict_conflicts) for a trace."""
    L = L or lib()
    req = np.ascontiguousarray(req, dtype=np.int64)
    lane = np.ascontiguousarray(lane, dtype=np.int32)
    addr = np.ascontiguousarray(addr, dtype=np.uint32)
    width = np.ascontiguousarray(width, dtype=np.int32)
    out = [ctypes.c_int64(0) for _ in range(3)]
    _check(L.oracle_bank_count(_ptr(req), _ptr(lane), _ptr(addr), _ptr(width), req.size,
                               *[ctypes.byref(o) for o in out]))
    return tuple(int(o.value) for o in out)
