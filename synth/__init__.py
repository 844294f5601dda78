"""Seeded synthetic input generators shared by the tests and the benchmark.

This module draws inputs only: it holds none of the sort / partition / permute
arithmetic, so both the CPU oracle and the CUDA path can be fed from it without
sharing any computation.  All randomness comes from numpy's PCG64 generator seeded
with the value passed in, so every input is reproducible.

Workload shapes follow the paper's three problems (Sec. 1, "Problems of
interest") at the sizes the library is measured on:

* partition inputs hold exactly n/w copies of every label in [0, w), shuffled;
* permutation inputs carry a uniform random bijection pi;
* sort inputs are uniform 32-bit keys or Zipf(1.1) keys over 2^16 distinct values;
* batched inputs use log-uniform segment sizes.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x150701391  # arXiv 1507.01391


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def index_payload(n: int) -> np.ndarray:
    """uint32 payload = original position, which makes a stable result unique."""
    return np.arange(n, dtype=np.uint32)


def partition_keys(n: int, w: int, seed: int) -> np.ndarray:
    """Exactly n/w copies of every label 0..w-1 in a seeded shuffled order."""
    if n % w:
        raise ValueError("n must be a multiple of w")
    keys = (np.arange(n, dtype=np.int64) % w).astype(np.uint32)
    rng(seed).shuffle(keys)
    return keys


def random_labels(n: int, w: int, seed: int) -> np.ndarray:
    """Labels drawn independently and uniformly from [0, w) (unbalanced counts)."""
    return rng(seed).integers(0, w, size=n, dtype=np.uint32)


def bernoulli_labels(n: int, p: float, seed: int) -> np.ndarray:
    """0/1 labels, each 1 with probability p (uint32)."""
    return (rng(seed).random(n) < p).astype(np.uint32)


def uniform_keys(n: int, seed: int, bits: int = 32) -> np.ndarray:
    """Keys uniform on [0, 2^bits)."""
    return rng(seed).integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)


def zipf_keys(n: int, seed: int, s: float = 1.1, distinct: int = 1 << 16) -> np.ndarray:
    """Zipf(s) over `distinct` values: rank r in [1, distinct] is drawn with
    probability proportional to r^-s (inverse CDF by binary search); the key is
    (r - 1) * 2654435761 mod 2^32, an odd-multiplier bijection that spreads the
    ranks over all four key bytes."""
    r = np.arange(1, distinct + 1, dtype=np.float64)
    cdf = np.cumsum(r ** (-s))
    cdf /= cdf[-1]
    u = rng(seed).random(n)
    rank = np.searchsorted(cdf, u, side="right")  # 0-based rank
    rank = np.minimum(rank, distinct - 1).astype(np.uint64)
    return ((rank * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def random_perm(n: int, seed: int) -> np.ndarray:
    """A uniform random permutation of [0, n) (Fisher-Yates via numpy)."""
    return rng(seed).permutation(n).astype(np.uint32)


def float_bits_payload(n: int, seed: int) -> np.ndarray:
    """Random 32-bit patterns viewed as float32: includes NaN, Inf, -0.0 and
    denormal encodings, so any arithmetic on payloads would show up."""
    return rng(seed).integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32).view(np.float32)


def tile_local_perms(n: int, tile: int, seed: int) -> np.ndarray:
    """uint16 local permutation per tile of `tile` items (the last tile may be
    shorter); tile t is an independent uniform permutation of its length."""
    if tile > 65536:
        raise ValueError("tile-local indices are 16-bit")
    g = rng(seed)
    out = np.empty(n, dtype=np.uint16)
    full = n // tile
    if full:
        # one independent permutation per row of a (full, tile) matrix
        out[: full * tile] = g.permuted(
            np.tile(np.arange(tile, dtype=np.uint16), (full, 1)), axis=1).reshape(-1)
    rest = n - full * tile
    if rest:
        out[full * tile:] = g.permutation(rest).astype(np.uint16)
    return out


def normal_f32(shape, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(shape, dtype=np.float64).astype(np.float32)


def log_uniform_sizes(nseg: int, seed: int, lo_log2: int = 5, hi_log2: int = 18) -> np.ndarray:
    """Segment sizes floor(2^U) with U uniform on [lo_log2, hi_log2], clamped."""
    u = rng(seed).uniform(lo_log2, hi_log2, size=nseg)
    sizes = np.floor(np.exp2(u)).astype(np.int64)
    return np.clip(sizes, 1 << lo_log2, 1 << hi_log2)


def offsets_from_sizes(sizes) -> np.ndarray:
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(np.asarray(sizes, dtype=np.int64), out=offs[1:])
    return offs


def segmented_partition_input(nseg: int, seed: int, widths=(32, 64, 128, 256),
                              lo_log2: int = 5, hi_log2: int = 18):
    """Per segment: w drawn from `widths`, size rounded down to a multiple of w
    (at least w), exactly size/w copies of every label, shuffled.  Returns
    (keys, offsets, w_per_segment)."""
    g = rng(seed)
    sizes = log_uniform_sizes(nseg, seed + 1, lo_log2, hi_log2)
    w = g.choice(np.asarray(widths, dtype=np.int32), size=nseg)
    sizes = np.maximum(w.astype(np.int64), (sizes // w) * w)
    offs = offsets_from_sizes(sizes)
    keys = np.empty(int(offs[-1]), dtype=np.uint32)
    for s in range(nseg):
        lo, hi = int(offs[s]), int(offs[s + 1])
        seg = (np.arange(hi - lo, dtype=np.int64) % int(w[s])).astype(np.uint32)
        g.shuffle(seg)
        keys[lo:hi] = seg
    return keys, offs, w.astype(np.int32)
