"""bcf: bank-conflict-free sort, permute and w-way partition on B300 (sm_103a).

Thin Python binding over ``libbcf.so`` (C ABI in ``include/bcf.h``).  This module
only marshals arguments: it turns torch tensors into device pointers, sizes
workspaces and passes the current CUDA stream.  Every data operation runs in the
library's CUDA kernels; there is no CPU or PyTorch fallback, and importing this
module raises if the library is missing or CUDA is unavailable when a call is
made.

The functions named ``bcf_*`` are the raw C entry points (ctypes); the snake-case
helpers (``sort``, ``partition``, ``permute`` ...) allocate outputs with torch and
call them.  Autograd forms live in ``paper_1507_01391_b300.autograd``.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libbcf.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "bcf.h")

# status codes and flags (mirrors include/bcf.h)
OK, E_INVAL, E_WORKSPACE, E_UNSUPPORTED, E_CUDA, E_TIMEOUT, E_NOT_BALANCED, E_BAD_PERM, E_BAD_KEY = range(9)
ASSUME_BALANCED = 0x1
CHECK_PERM = 0x2
TILES_COLOURED = 0x10
PARTITION_LEMMA1 = 0x20
PERMUTE_FUSED = 0x40
PERMUTE_BUCKETED = 0x80
TILES_SORTED_FINISH = 0x100
PARTITION_DIRECT = 0x200
# Sizes from which permute()/permute_kv() pick the bucketed form by default.
BUCKETED_MIN_N = 1 << 20
BUCKETED_MAX_N = 1 << 26


class BcfError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().bcf_status_string(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (status %d)" % (what or "bcf", msg, code))


_lib = None

_P, _I, _I64, _SZ, _U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_uint64
_SIGS = {
    "bcf_status_string": ([_I], ctypes.c_char_p),
    "bcf_version": ([], _I),
    "bcf_get_status": ([_P, ctypes.POINTER(_I)], _I),
    "bcf_sort_workspace_size": ([_I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "bcf_sort": ([_P, _P, _P, _P, _I64, _I, _I, _P, _SZ, _P], _I),
    "bcf_partition_workspace_size": ([_I64, _I, _I, _I, ctypes.POINTER(_SZ)], _I),
    "bcf_partition": ([_P, _P, _P, _P, _I64, _I, _I, _I, _P, _SZ, _P], _I),
    "bcf_partition_splitters_workspace_size": ([_I64, _I, _I, _I, ctypes.POINTER(_SZ)], _I),
    "bcf_partition_splitters": ([_P, _P, _P, _P, _I64, _P, _I, _I, _I, _P, _SZ, _P], _I),
    "bcf_permute_workspace_size": ([_I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "bcf_permute": ([_P, _P, _P, _I64, _I64, _I, _I, _P, _SZ, _P], _I),
    "bcf_permute_kv": ([_P, _P, _P, _P, _P, _I64, _I64, _I, _I, _P, _SZ, _P], _I),
    "bcf_permute_tiles": ([_P, _P, _P, _I64, _I, _I, _U64, _P], _I),
    "bcf_gather": ([_P, _P, _P, _I64, _I64, _I64, _I, _P], _I),
    "bcf_sort_passes_run": ([_P, _I64, _I, _I, ctypes.POINTER(_I), _P], _I),
    "bcf_sort_tiles": ([_P, _P, _P, _P, _I64, _I, _I, _P], _I),
    "bcf_partition_lemma2": ([_P, _P, _P, _P, _I64, _P], _I),
    "bcf_segmented_sort_workspace_size": ([_I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "bcf_segmented_sort": ([_P, _P, _P, _P, _I64, _P, _I64, _I, _I, _P, _SZ, _P], _I),
    "bcf_segmented_partition_workspace_size": ([_I64, _I64, _I, ctypes.POINTER(_SZ)], _I),
    "bcf_segmented_partition": ([_P, _P, _P, _P, _I64, _P, _P, _I64, _I, _I, _P, _SZ, _P], _I),
    "bcf_partition_noalloc": ([_P, _P, _P, _P, _I64, _I, _I, _I, _P], _I),
    "bcf_tune_num_configs": ([], _I),
    "bcf_tune_config_info": ([_I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "bcf_tune_config_form": ([_I], _I),
    "bcf_tune_set": ([_I, _I, _I], _I),
    "bcf_tune_get": ([_I, _I64, ctypes.POINTER(_I)], _I),
    "bcf_debug_lookback": ([_I, ctypes.c_uint], _I),
    "bcf_tune_save": ([ctypes.c_char_p], _I),
    "bcf_tune_load": ([ctypes.c_char_p, ctypes.POINTER(_I)], _I),
}
OP_SORT, OP_PARTITION, OP_SEGMENTED_SORT = 0, 1, 2
NOALLOC_MAX_N = 1 << 22


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions include/bcf.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bcf_[a-z0-9_]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libbcf.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libbcf.so is not built (run __graft_entry__.build()); "
                              "there is no fallback implementation")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def __getattr__(name):  # raw entry points: bcf_sort, bcf_permute, ...; the autograd forms
    if name.startswith("bcf_") and name in _SIGS:
        return getattr(lib(), name)
    if name in ("SortByKey", "PermuteFn", "sort_by_key", "permute_rows"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)


# ------------------------------------------------------------------ helpers
_cuda_ok = False


def _torch():
    global _cuda_ok
    import torch
    if not _cuda_ok:  # checked once per process
        if not torch.cuda.is_available():
            raise RuntimeError("bcf needs a CUDA device; there is no CPU path")
        _cuda_ok = True
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc, what):
    if rc != OK:
        raise BcfError(rc, what)


def _vb(vals):
    return 0 if vals is None else vals.element_size()


def _dev_u32(t, what):
    torch = _torch()
    if t.device.type != "cuda" or t.dtype not in (torch.int32, torch.uint32) or not t.is_contiguous():
        raise ValueError("%s must be a contiguous 32-bit CUDA tensor" % what)
    return t


def get_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device error status."""
    out = ctypes.c_int(0)
    _check(lib().bcf_get_status(_stream(stream), ctypes.byref(out)), "bcf_get_status")
    return out.value


def raise_on_device_error(stream=None):
    st = get_status(stream)
    if st != OK:
        raise BcfError(st, "device")


def sort_workspace_size(n, val_bytes=4, key_bits=32) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().bcf_sort_workspace_size(n, val_bytes, key_bits, ctypes.byref(out)), "workspace")
    return out.value


def partition_workspace_size(n, w, val_bytes=4, flags=0) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().bcf_partition_workspace_size(n, w, val_bytes, flags, ctypes.byref(out)), "workspace")
    return out.value


def workspace(nbytes, device=None):
    torch = _torch()
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device or "cuda")


def sort(keys, vals=None, key_bits=32, keys_out=None, vals_out=None, ws=None, stream=None,
         index_payload=False):
    """Stable ascending sort by uint32 key (bcf_sort).  Returns (keys, vals).
    index_payload=True (vals None): vals_out receives the sorting permutation."""
    torch = _torch()
    _dev_u32(keys, "keys")
    n = keys.numel()
    vb = 4 if index_payload else _vb(vals)
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals_out is None and (vals is not None or index_payload):
        vals_out = torch.empty_like(keys) if index_payload else torch.empty_like(vals)
    need = sort_workspace_size(n, vb, key_bits)
    ws = workspace(need, keys.device) if ws is None else ws
    _check(lib().bcf_sort(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n, vb, key_bits,
                          _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "bcf_sort")
    return keys_out, vals_out


sort_kv = sort  # the key-value sort under its other name


def sort_passes_run(ws, n, val_bytes=4, key_bits=32, stream=None) -> int:
    """Digit passes the last sort that used workspace ws ran; the others were
    skipped because their digit is the same in every key (syncs the stream)."""
    out = ctypes.c_int(0)
    _check(lib().bcf_sort_passes_run(_ptr(ws), int(n), int(val_bytes), int(key_bits), ctypes.byref(out),
                                     _stream(stream)), "bcf_sort_passes_run")
    return out.value


def partition(keys, vals, w, balanced=False, keys_out=None, vals_out=None, ws=None, stream=None,
              flags=0):
    """Stable w-way partition by label in [0, w) (bcf_partition)."""
    torch = _torch()
    _dev_u32(keys, "keys")
    n = keys.numel()
    vb = _vb(vals)
    flags = flags | (ASSUME_BALANCED if balanced else 0)
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    if ws is None:  # a caller's workspace is checked against the size by the library
        ws = workspace(partition_workspace_size(n, w, vb, flags), keys.device)
    _check(lib().bcf_partition(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n, w, vb,
                               flags, _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "bcf_partition")
    return keys_out, vals_out


def partition_splitters_workspace_size(n, nsplit, val_bytes=4, flags=0) -> int:
    sz = ctypes.c_size_t(0)
    _check(lib().bcf_partition_splitters_workspace_size(int(n), int(nsplit), int(val_bytes), int(flags),
                                                        ctypes.byref(sz)), "bcf_partition_splitters_workspace_size")
    return sz.value


def partition_splitters(keys, vals, splitters, balanced=False, keys_out=None, vals_out=None, ws=None,
                        stream=None):
    """Stable partition of keys (and payloads) into len(splitters) + 1 buckets, bucket =
    number of splitters <= key (bcf_partition_splitters); splitters: ascending uint32
    values in a 32-bit CUDA tensor."""
    torch = _torch()
    _dev_u32(splitters, "splitters")
    n = keys.numel()
    nsplit = splitters.numel()
    vb = _vb(vals)
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    flags = ASSUME_BALANCED if balanced else 0
    if ws is None:
        ws = workspace(partition_splitters_workspace_size(n, nsplit, vb, flags), keys.device)
    _check(lib().bcf_partition_splitters(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n,
                                         _ptr(splitters), nsplit, vb, flags, _ptr(ws), ws.numel(),
                                         _stream(stream)), "bcf_partition_splitters")
    return keys_out, vals_out


def _permute_flags(n, elem_bytes, val_bytes, check, fused, bucketed):
    if bucketed is None:  # default: the bucketed form where it applies and pays (keys with payloads;
        # a single array of 2^24 keys measures the same either way, and one scatter pass needs no workspace)
        bucketed = (elem_bytes == 4 and val_bytes == 4 and BUCKETED_MIN_N <= n <= BUCKETED_MAX_N)
    return (CHECK_PERM if check else 0) | (PERMUTE_FUSED if fused else 0) | (PERMUTE_BUCKETED if bucketed else 0)


def permute_workspace_size(n, val_bytes=0, flags=0):
    sz = ctypes.c_size_t(0)
    _check(lib().bcf_permute_workspace_size(int(n), int(val_bytes), int(flags), ctypes.byref(sz)),
           "bcf_permute_workspace_size")
    return sz.value


def permute(src, pi, dst=None, check=False, row_len=0, stream=None, bucketed=None, ws=None):
    """dst[pi[i]] = src[i] for 4- or 8-byte elements (bcf_permute); with row_len,
    pi is local to rows of row_len items.  bucketed: True (two coalesced passes;
    4-byte elements, n <= 2^26), False (one scatter pass), or None: the library's
    choice, which for a single array is one scatter pass (with payloads,
    permute_kv picks the bucketed form for 2^20 <= n <= 2^26); ws: optional
    preallocated workspace (uint8 tensor)."""
    torch = _torch()
    _dev_u32(pi, "pi")
    n = src.numel()
    dst = torch.empty_like(src) if dst is None else dst
    flags = _permute_flags(n, src.element_size(), 0, check, False, bucketed)
    need = permute_workspace_size(n, 0, flags)
    if need and (ws is None or ws.numel() < need):
        ws = workspace(need, src.device)
    _check(lib().bcf_permute(_ptr(src), _ptr(dst), _ptr(pi), n, row_len, src.element_size(), flags, _ptr(ws),
                             0 if ws is None else ws.numel(), _stream(stream)), "bcf_permute")
    return dst


def permute_kv(keys, vals, pi, keys_out=None, vals_out=None, check=False, row_len=0, stream=None,
               fused=False, bucketed=None, ws=None):
    """Keys and payloads moved by one permutation (bcf_permute_kv).  Forms: two
    scatter passes (default below 2^20 keys), one fused scatter (fused=True) or
    two coalesced bucketed passes (bucketed; default from 2^20 to 2^26 keys)."""
    torch = _torch()
    n = keys.numel()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    vb = _vb(vals)
    flags = _permute_flags(n, 4, vb, check, fused, bucketed)
    need = permute_workspace_size(n, vb, flags)
    if need and (ws is None or ws.numel() < need):
        ws = workspace(need, keys.device)
    _check(lib().bcf_permute_kv(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), _ptr(pi), n,
                                row_len, vb, flags, _ptr(ws), 0 if ws is None else ws.numel(),
                                _stream(stream)), "bcf_permute_kv")
    return keys_out, vals_out


def permute_tiles(src, lpi, tile=4096, coloured=False, seed=0x150701391, dst=None, stream=None,
                  finish="greedy"):
    """Tile-local permutation by uint16 local labels (bcf_permute_tiles).  With
    coloured=True, finish="sorted" sends the leftovers by the three-group
    finishing step instead of greedily."""
    torch = _torch()
    dst = torch.empty_like(src) if dst is None else dst
    if finish not in ("greedy", "sorted"):
        raise ValueError("finish must be 'greedy' or 'sorted'")
    flags = (TILES_COLOURED if coloured else 0) | (TILES_SORTED_FINISH if finish == "sorted" else 0)
    _check(lib().bcf_permute_tiles(_ptr(src), _ptr(dst), _ptr(lpi), src.numel(), tile, flags,
                                   seed & 0xFFFFFFFFFFFFFFFF, _stream(stream)), "bcf_permute_tiles")
    return dst


def gather(src, idx, dst=None, row_len=0, stream=None):
    """dst[i] = src[idx[i]] (bcf_gather); with row_len, idx is local to rows."""
    torch = _torch()
    n = idx.numel()
    dst = torch.empty(n, dtype=src.dtype, device=src.device) if dst is None else dst
    _check(lib().bcf_gather(_ptr(src), _ptr(dst), _ptr(idx), n, src.numel(), row_len,
                            src.element_size(), _stream(stream)), "bcf_gather")
    return dst


LEMMA2_ITEMS = 32768  # items of one 1024 x 32 matrix


def partition_lemma2(keys, vals=None, keys_out=None, vals_out=None, stream=None):
    """Lemma 2's 0-1 partition of every 1024 x 32 matrix (32768 items, column-major
    in, row-major out).  vals None: each item carries its input position."""
    torch = _torch()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals_out is None:
        vals_out = torch.empty_like(keys) if vals is None else torch.empty_like(vals)
    _check(lib().bcf_partition_lemma2(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), keys.numel(),
                                      _stream(stream)), "bcf_partition_lemma2")
    return keys_out, vals_out


def sort_tiles(keys, vals=None, tile=4096, keys_out=None, vals_out=None, stream=None):
    """Sort every tile of `tile` keys on its own with the Lemma 1 schedule."""
    torch = _torch()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    _check(lib().bcf_sort_tiles(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), keys.numel(),
                                tile, _vb(vals), _stream(stream)), "bcf_sort_tiles")
    return keys_out, vals_out


def segmented_sort_workspace_size(n_total, nseg, val_bytes=4, key_bits=32) -> int:
    sz = ctypes.c_size_t(0)
    _check(lib().bcf_segmented_sort_workspace_size(n_total, nseg, val_bytes, key_bits, ctypes.byref(sz)),
           "workspace")
    return sz.value


def segmented_partition_workspace_size(n_total, nseg, val_bytes=4) -> int:
    sz = ctypes.c_size_t(0)
    _check(lib().bcf_segmented_partition_workspace_size(n_total, nseg, val_bytes, ctypes.byref(sz)),
           "workspace")
    return sz.value


def segmented_sort(keys, vals, offs, key_bits=32, keys_out=None, vals_out=None, ws=None, stream=None,
                   index_payload=False):
    """Sort each CSR segment on its own (bcf_segmented_sort); offs is an int64 CUDA tensor.
    index_payload=True (vals None): vals_out receives global input positions."""
    torch = _torch()
    n = keys.numel()
    nseg = offs.numel() - 1
    vb = 4 if index_payload else _vb(vals)
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals_out is None and (vals is not None or index_payload):
        vals_out = torch.empty_like(keys) if index_payload else torch.empty_like(vals)
    if ws is None:
        ws = workspace(segmented_sort_workspace_size(n, nseg, vb, key_bits), keys.device)
    _check(lib().bcf_segmented_sort(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n,
                                    _ptr(offs), nseg, vb, key_bits, _ptr(ws), ws.numel(),
                                    _stream(stream)), "bcf_segmented_sort")
    return keys_out, vals_out


def segmented_partition(keys, vals, offs, w_per_seg, balanced=False, keys_out=None, vals_out=None,
                        ws=None, stream=None):
    """Partition each CSR segment by its own w (bcf_segmented_partition)."""
    torch = _torch()
    n = keys.numel()
    nseg = offs.numel() - 1
    vb = _vb(vals)
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    if ws is None:
        ws = workspace(segmented_partition_workspace_size(n, nseg, vb), keys.device)
    flags = ASSUME_BALANCED if balanced else 0
    _check(lib().bcf_segmented_partition(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n,
                                         _ptr(offs), _ptr(w_per_seg), nseg, vb, flags, _ptr(ws),
                                         ws.numel(), _stream(stream)), "bcf_segmented_partition")
    return keys_out, vals_out


def partition_noalloc(keys, vals, w, balanced=False, keys_out=None, vals_out=None, stream=None):
    """Stable w-way partition whose scratch is a fixed array inside the library
    (bcf_partition_noalloc): for callers that cannot allocate device memory at
    call time.  n <= NOALLOC_MAX_N, out of place only.  The outputs are
    allocated here only when not given."""
    torch = _torch()
    _dev_u32(keys, "keys")
    n = keys.numel()
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    if vals is not None and vals_out is None:
        vals_out = torch.empty_like(vals)
    flags = ASSUME_BALANCED if balanced else 0
    _check(lib().bcf_partition_noalloc(_ptr(keys), _ptr(vals), _ptr(keys_out), _ptr(vals_out), n, w,
                                       _vb(vals), flags, _stream(stream)), "bcf_partition_noalloc")
    return keys_out, vals_out
