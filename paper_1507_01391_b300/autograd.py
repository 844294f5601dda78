"""Differentiable sort-by-key and permutation of float payloads.

Both functions only move payloads, so their Jacobians are permutation matrices and
the backward pass is the inverse permutation applied to the upstream gradient:

* SortByKey: y[b, r] = v[b, perm[b, r]] where perm[b] is the stable ascending order
  of keys[b].  Forward = one segmented key sort whose payload is the global input
  position (the library's index-payload mode), then a gather of the values.
  Backward = grad_v[b, perm[b, r]] = g[b, r], a scatter by perm (bcf_permute).
* PermuteFn: y[b, pi[b, i]] = v[b, i] (pi local to each row).  Forward = bcf_permute
  with row_len = n; backward = grad_v[b, i] = g[b, pi[b, i]] (bcf_gather).

Keys and pi are 32-bit integer tensors (uint32 bit patterns in int32); values are
float32 or float64.  Every step runs in libbcf's kernels on the current stream.
"""
from __future__ import annotations

import torch

from . import gather, permute, segmented_sort, segmented_sort_workspace_size, workspace


_OFFS = {}


def _row_offsets(B: int, n: int, device) -> torch.Tensor:
    """CSR offsets of B rows of n items (B + 1 int64 values), built on the host
    once per shape and device and kept resident."""
    key = (B, n, str(device))
    t = _OFFS.get(key)
    if t is None:
        t = torch.tensor([b * n for b in range(B + 1)], dtype=torch.int64).to(device)
        _OFFS[key] = t
    return t


_WS = {}


def _workspace(nbytes: int, device) -> torch.Tensor:
    """Workspace reused across calls of the same size on the same stream and
    device (the library only needs it for the duration of a call)."""
    key = (int(nbytes), str(device), torch.cuda.current_stream(device).cuda_stream)
    t = _WS.get(key)
    if t is None:
        t = workspace(nbytes, device)
        _WS[key] = t
    return t


class SortByKey(torch.autograd.Function):
    """(keys [B, n] int32, values [B, n] float) -> (sorted keys, values in key order)."""

    @staticmethod
    def forward(ctx, keys, values, key_bits=32):
        if keys.dim() == 1:
            keys, values = keys.unsqueeze(0), values.unsqueeze(0)
        B, n = keys.shape
        k = keys.contiguous().view(-1)
        v = values.contiguous().view(-1)
        offs = _row_offsets(B, n, keys.device)
        ws = _workspace(segmented_sort_workspace_size(B * n, B, 4, key_bits), keys.device)
        ko, perm = segmented_sort(k, None, offs, key_bits=key_bits, ws=ws, index_payload=True)
        y = gather(v, perm)  # perm holds global positions
        ctx.save_for_backward(perm)
        ctx.shape = (B, n)
        ctx.mark_non_differentiable(ko)
        return ko.view(B, n), y.view(B, n)

    @staticmethod
    def backward(ctx, g_keys, g_y):
        (perm,) = ctx.saved_tensors
        B, n = ctx.shape
        grad_v = None
        if ctx.needs_input_grad[1]:
            grad_v = permute(g_y.contiguous().view(-1), perm).view(B, n)  # grad_v[perm[r]] = g[r]
        return None, grad_v, None


class PermuteFn(torch.autograd.Function):
    """(values [B, n] float, pi [B, n] int32 local to each row) -> y, y[b, pi[b,i]] = v[b,i]."""

    @staticmethod
    def forward(ctx, values, pi):
        if values.dim() == 1:
            values, pi = values.unsqueeze(0), pi.unsqueeze(0)
        B, n = values.shape
        p = pi.contiguous().view(-1)
        y = permute(values.contiguous().view(-1), p, row_len=n)
        ctx.save_for_backward(p)
        ctx.shape = (B, n)
        ctx.mark_non_differentiable(pi)
        return y.view(B, n)

    @staticmethod
    def backward(ctx, g):
        (p,) = ctx.saved_tensors
        B, n = ctx.shape
        grad_v = None
        if ctx.needs_input_grad[0]:
            grad_v = gather(g.contiguous().view(-1), p, row_len=n).view(B, n)  # g[pi[i]]
        return grad_v, None


def sort_by_key(keys, values, key_bits=32):
    return SortByKey.apply(keys, values, key_bits)


def permute_rows(values, pi):
    return PermuteFn.apply(values, pi)
