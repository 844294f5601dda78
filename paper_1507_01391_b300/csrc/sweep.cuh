// sweep.cuh -- one stable digit sweep over tiles (shared by radix.cu and
// segmented.cu).
//
// One sweep moves every key to the block of its digit (or partition label).  It
// is the paper's partition problem (Sec. 1) at GPU scale: each block of threads
// ranks one tile of keys in shared memory -- the per-row "radix sort" of
// Corollary 1 done per warp -- and finds the tile's global offsets with a
// decoupled look-back over earlier tiles.  Keys and payloads are staged into
// shared memory by bulk copies (TMA engine), read back with the conflict-free
// strided pattern of Sec. 1 (lane t reads word 32i + t), and written out in
// digit order so that global stores form contiguous runs.
//
// Segment mode: tiles belong to CSR segments; a segment's first tile starts the
// look-back chain, digit bases are per segment, and segment starts need not be
// 16-byte aligned (the bulk copy starts at the aligned-down address and the tile
// is read at an offset).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "trace.cuh"

namespace bcf {

constexpr uint32_t LB_AGG = 1u << 30;   // tile aggregate published
constexpr uint32_t LB_INC = 2u << 30;   // inclusive prefix published
constexpr uint32_t LB_MASK = (1u << 30) - 1;

// Pass skipping of the LSD radix sort.  A digit pass in which every key has the
// same digit moves nothing, so it is left out; which passes run is decided on the
// device (no host round trip, so a sort stays capturable in a CUDA graph).  The
// first pass's count kernel (or the histogram of small inputs) ORs every key into
// vary[0] and every complement into vary[1]: key bit b varies iff it is set in
// both.  Each kernel of pass q then finds from vary whether pass q runs and which
// buffers it reads and writes: the runs alternate between the output and a
// temporary so that the last one lands in the output (in place with an odd count:
// in the temporary, and k_pass_copy brings it home).  One thread per block reads
// the choice and hands it to the others.
struct PassSel {
  uint32_t* vary;        // [2], zero before the first pass; nullptr: no skipping
  uint32_t* ran;         // zero before the first pass; bit q set when pass q ran
  int q = 0, passes = 0, in_place = 0;
  int shift[4] = {0, 0, 0, 0};
  const uint32_t* k_in = nullptr;
  const void* v_in = nullptr;  // nullptr with 4-byte payloads: payload = input position
  uint32_t* k_out = nullptr;
  void* v_out = nullptr;
  uint32_t* k_tmp = nullptr;
  void* v_tmp = nullptr;
};

// The varying key bits: AND of the two OR words.  The words are final before the
// kernel that reads them starts, so the read may go through the SM's read-only
// cache: of the many blocks an SM runs, only the first waits on L2.
__device__ __forceinline__ uint32_t vary_bits(const PassSel& s) {
  return __ldg(s.vary) & __ldg(s.vary + 1);
}

// Passes that run (bit q) given the varying bits.  Out of place, when no digit
// varies the last pass still runs (a stable pass over equal digits is a copy),
// so that the result reaches the output.
__device__ __forceinline__ unsigned passes_run_mask(const PassSel& s, uint32_t v) {
  unsigned m = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)  // constant indices: the shifts stay in parameter space
    if (q < s.passes && ((v >> s.shift[q]) & 0xFFu)) m |= 1u << q;
  if (!m && !s.in_place) m = 1u << (s.passes - 1);
  return m;
}

// Route of pass s.q given the varying bits: -1 when the pass is skipped, else
// 3 * src + dst, where src is 0 (the input), 1 (the output) or 2 (the temporary)
// and dst is 1 (the output) or 2 (the temporary).
__device__ __forceinline__ int pass_route(const PassSel& s, uint32_t v) {
  const unsigned m = passes_run_mask(s, v);
  if (!((m >> s.q) & 1u)) return -1;
  const int i = __popc(m & ((1u << s.q) - 1u)), k = __popc(m);
  auto to_out = [&](int j) { return (s.in_place && (k & 1)) ? (j & 1) == 1 : ((k - 1 - j) & 1) == 0; };
  const int src = i == 0 ? 0 : (to_out(i - 1) ? 1 : 2);
  const int dst = to_out(i) ? 1 : 2;
  return 3 * src + dst;
}

// The buffers a route names.
__device__ __forceinline__ void route_buffers(const PassSel& s, int route, const uint32_t*& sk, const void*& sv,
                                              uint32_t*& dk, void*& dv) {
  const int src = route / 3, dst = route % 3;
  sk = src == 0 ? s.k_in : (src == 1 ? s.k_out : s.k_tmp);
  sv = src == 0 ? s.v_in : (src == 1 ? s.v_out : s.v_tmp);
  dk = dst == 1 ? s.k_out : s.k_tmp;
  dv = dst == 1 ? s.v_out : s.v_tmp;
}

// Buffers of pass s.q given the varying bits; false when the pass is skipped.
__device__ __forceinline__ bool pass_buffers(const PassSel& s, uint32_t v, const uint32_t*& sk,
                                             const void*& sv, uint32_t*& dk, void*& dv) {
  const int route = pass_route(s, v);
  if (route < 0) return false;
  route_buffers(s, route, sk, sv, dk, dv);
  return true;
}

struct SweepParams {
  const uint32_t* keys_in;
  const void* vals_in;         // nullptr with 4-byte payloads: payload = input position
  uint32_t* keys_out;
  void* vals_out;
  int64_t n;
  int shift, nbits;            // radix digit = (key >> shift) & (2^nbits - 1)
  int w;                       // > 0: partition by label, labels must be < w
  int balanced;                // partition: block b starts at b * len / w
  const uint32_t* digit_base;  // exclusive global start of every digit
  uint32_t* lookback;          // RADIX x lb_stride status words (digit-major), zero on entry
  int64_t lb_stride;           // tiles rounded up to a multiple of the look-back window
  uint32_t* ticket;            // tile counter, zero on entry
  unsigned* status;
  // reduce-then-scan mode (tile_offsets != nullptr): absolute start of every
  // (digit, tile) run, digit-major with stride lb_stride; no look-back
  const uint32_t* tile_offsets;
  // segment mode (seg_offs != nullptr)
  const int64_t* seg_offs;     // CSR offsets (nseg + 1)
  const int32_t* tile_seg;     // tile -> segment
  const int32_t* seg_tile0;    // segment -> its first tile
  const int32_t* seg_slot;     // segment -> row of seg_base
  const uint32_t* seg_base;    // slot x RADIX absolute digit starts
  const int32_t* seg_w;        // partition: labels of segment s are < seg_w[s]
  const uint32_t* num_tiles;   // tiles of this launch (device count)
  // look-back mode only: polls before a wait gives up (0: kSpinLimit), and 1 + the
  // index of a tile that never publishes its status (0: none) -- a testing aid that
  // makes a later tile's bounded wait run out
  unsigned spin_limit;
  int silent_tile1;
  // splitter mode (k_sweep<..., SPLIT = true>): digit = number of splitters <= key,
  // each key's bucket as the tile counts kept it
  const uint8_t* labels;
  PassSel sel;                 // sel.vary != nullptr: buffers (or a skip) decided on the device
};

template <int BITS>
__device__ __forceinline__ uint32_t digit_of(uint32_t key, int label_mode, int shift, int nbits) {
  if (label_mode) return key & ((1u << BITS) - 1u);
  return (key >> shift) & ((1u << nbits) - 1u);
}

// Exclusive scan of one value per thread over the block; *total gets the sum.
template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* scratch,
                                                    uint32_t* total) {
  constexpr int WARPS = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  BCF_SYNC();
  if (warp == 0) {
    uint32_t s = lane < WARPS ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < WARPS) scratch[lane] = s;
  }
  BCF_SYNC();
  const uint32_t before = warp ? scratch[warp - 1] : 0u;
  *total = scratch[WARPS - 1];
  BCF_SYNC();
  return before + x - v;
}

// Exclusive scans of N independent values per thread over the block, in one set
// of barriers; total[k] gets the sum of sequence k.  scratch holds N * 32 words.
template <int THREADS, int N>
__device__ __forceinline__ void block_excl_scan_n(const uint32_t (&v)[N], uint32_t (&out)[N], uint32_t* scratch,
                                                  uint32_t (&total)[N]) {
  constexpr int WARPS = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x[N];
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = v[k];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x[k], o);
      if (lane >= o) x[k] += y;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int k = 0; k < N; ++k) scratch[k * 32 + warp] = x[k];
  BCF_SYNC();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      uint32_t t = lane < WARPS ? scratch[k * 32 + lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < WARPS) scratch[k * 32 + lane] = t;
    }
  }
  BCF_SYNC();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    out[k] = (warp ? scratch[k * 32 + warp - 1] : 0u) + x[k] - v[k];
    total[k] = scratch[k * 32 + WARPS - 1];
  }
  BCF_SYNC();
}

// ------------------------------------------------------------- histogram
struct HistParams {
  const uint32_t* keys;
  int64_t n;
  int passes;
  int shift[4];
  int nbits[4];
  int label_bits;        // > 0: partition, one "pass" with digit = key & mask
  uint32_t* hist;        // passes x 256, zero on entry
  uint32_t* digit_base;  // passes x 256, written by the last block
  uint32_t* done;        // zero on entry
  uint32_t* vary;        // nullptr, or [2] zero on entry: OR of the keys, OR of their complements
};

// Block-wide OR of (o1, o0) into vary[0], vary[1] (every thread of the block
// takes part; ends with a barrier).
__device__ __forceinline__ void or_into_vary(uint32_t o1, uint32_t o0, uint32_t* vary, uint32_t* scratch2) {
  o1 = __reduce_or_sync(0xffffffffu, o1);
  o0 = __reduce_or_sync(0xffffffffu, o0);
  if (threadIdx.x == 0) scratch2[0] = scratch2[1] = 0u;
  BCF_SYNC();
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&scratch2[0], o1);
    atomicOr(&scratch2[1], o0);
  }
  BCF_SYNC();
  if (threadIdx.x == 0) {
    if (scratch2[0]) atomicOr(&vary[0], scratch2[0]);
    if (scratch2[1]) atomicOr(&vary[1], scratch2[1]);
  }
  BCF_SYNC();
}

// Counts every digit of every pass in one read of the keys; the last block to
// finish turns the counts into exclusive starts.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_histogram(HistParams p) {
  __shared__ uint32_t h[4 * 256];
  __shared__ uint32_t scratch[32];
  __shared__ int is_last;
  const int tid = threadIdx.x;
  for (int i = tid; i < 4 * 256; i += THREADS) h[i] = 0;
  BCF_SYNC();
  uint32_t mask[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    mask[q] = p.label_bits ? ((1u << p.label_bits) - 1u) : ((1u << p.nbits[q]) - 1u);
  const int64_t nvec = p.n >> 2;
  const uint4* kv = reinterpret_cast<const uint4*>(p.keys);
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  uint32_t o1 = 0, o0 = 0;  // OR of the keys and of their complements
  for (int64_t i = (int64_t)blockIdx.x * THREADS + tid; i < nvec; i += stride) {
    uint4 k4 = __ldcs(kv + i);
    uint32_t k[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      o1 |= k[c];
      o0 |= ~k[c];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < p.passes) atomicAdd(&h[q * 256 + ((k[c] >> p.shift[q]) & mask[q])], 1u);
    }
  }
  for (int64_t i = nvec * 4 + (int64_t)blockIdx.x * THREADS + tid; i < p.n; i += stride) {
    uint32_t k = p.keys[i];
    o1 |= k;
    o0 |= ~k;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < p.passes) atomicAdd(&h[q * 256 + ((k >> p.shift[q]) & mask[q])], 1u);
  }
  if (p.vary) or_into_vary(o1, o0, p.vary, scratch);
  BCF_SYNC();
  for (int i = tid; i < p.passes * 256; i += THREADS)
    if (h[i]) atomicAdd(&p.hist[i], h[i]);
  __threadfence();
  BCF_SYNC();
  if (tid == 0) is_last = (atomicAdd(p.done, 1u) == gridDim.x - 1);
  BCF_SYNC();
  if (!is_last) return;
  __threadfence();
  for (int q = 0; q < p.passes; ++q) {
    uint32_t c = tid < 256 ? ld_relaxed(&p.hist[q * 256 + tid]) : 0u;
    uint32_t total;
    uint32_t e = block_excl_scan<THREADS>(c, scratch, &total);
    if (tid < 256) p.digit_base[q * 256 + tid] = e;
  }
}

// Bucket of key k among nsplit ascending splitters: the number of splitters <= k.
// A prefix table narrows the search.  The splitters span [base, base + range];
// prefix P of a key k >= base is (k - base) >> sh, sh the smallest shift that
// leaves every splitter's prefix below kSplitPrefixes (keys below base take prefix
// 0, keys past the last prefix the last).  Entry P is lo | hi << 8: lo counts the
// splitters below the prefix's first value and [lo, hi) are the splitters with
// prefix P.  The bucket is lo plus the number of those <= k, found by a binary
// search over powers of two -- no step at all for the prefixes that hold no
// splitter, most of them when 255 splitters share 4096 prefixes.
__device__ __forceinline__ uint32_t split_bucket(const uint32_t* spl, const uint16_t* spt, uint32_t base,
                                                 uint32_t sh, uint32_t k) {
  const uint32_t e = spt[min((max(k, base) - base) >> sh, (uint32_t)(kSplitPrefixes - 1))];
  uint32_t b = e & 0xFFu, len = (e >> 8) - b;  // the prefix's splitters: spl[b, b + len)
  while (len > 0) {
    const uint32_t half = len >> 1;
    const bool right = spl[b + half] <= k;
    b = right ? b + half + 1 : b;
    len = right ? len - half - 1 : half;
  }
  return b;
}

// ------------------------------------------------------------- reduce-then-scan
// Per-tile digit counts of one pass (digit-major), plus the pass's digit totals.
struct CountParams {
  const uint32_t* keys;
  int64_t n;
  int shift, nbits, label_bits;  // label_bits > 0: digit = key & (2^label_bits - 1)
  uint32_t* counts;              // RADIX x stride
  int64_t stride;
  uint32_t* totals;              // RADIX, zero on entry (nullptr: not needed)
  // segment mode (seg_offs != nullptr): tile ranges come from the segment plan
  const int64_t* seg_offs;
  const int32_t* tile_seg;
  const int32_t* seg_tile0;
  const uint32_t* num_tiles;
  const int32_t* seg_w;          // segment mode, partition: labels of segment s must be < seg_w[s]
  unsigned* status;              //   (a larger one is recorded as DEV_BAD_KEY here)
  const uint32_t* splitters;     // splitter mode: digit = number of splitters <= key,
  int nsplit;                    //   found through the prefix table k_split_table builds
  const uint16_t* split_table;
  uint8_t* labels;               // splitter mode, unsegmented: bucket of key i stored at labels[i]
  PassSel sel;                   // sel.vary != nullptr: pass 0 fills vary, later passes may skip
};

#ifndef BCF_COUNT_TILES_PER_BLOCK
#define BCF_COUNT_TILES_PER_BLOCK 4
#endif
constexpr int kCountTilesPerBlock = BCF_COUNT_TILES_PER_BLOCK;

// FAST: the four-tiles-at-once path for unsegmented inputs (its 16 vector loads in
// flight take registers; the segment-mode instance leaves it out and keeps its
// occupancy for the scalar loads of unaligned segments).
template <int BITS, int T, bool SPLIT = false, bool FAST = true>
__global__ void __launch_bounds__(256, 3) k_tile_counts(CountParams p, int64_t tiles) {
  constexpr int RADIX = 1 << BITS;
  constexpr int NV = T / 1024;  // 16-byte loads per thread per tile
  static_assert(kCountTilesPerBlock == 4, "fast path counts four tiles at once");
  __shared__ uint32_t h[RADIX];
  __shared__ uint32_t tot[RADIX];
  __shared__ __align__(16) uint32_t h4[FAST ? 4 : 1][RADIX];
  // fast path: lane-private byte counters, counter (tile t, digit d) of lane l is
  // byte d mod 4 of lc[t][d / 4][l]
  __shared__ __align__(16) uint32_t lc[FAST ? 4 : 1][FAST ? RADIX / 4 : 1][32];
  const int tid = threadIdx.x;
  for (int i = tid; i < RADIX; i += 256) tot[i] = 0;
  const uint32_t mask = p.label_bits ? ((1u << p.label_bits) - 1u) : (uint32_t)(RADIX - 1);
  const int shift = p.label_bits ? 0 : p.shift;
  __shared__ uint32_t spl[SPLIT ? 256 : 1];
  __shared__ __align__(16) uint16_t spt[SPLIT ? kSplitPrefixes : 1];
  if constexpr (SPLIT) {  // read after a barrier below
    for (int i = tid; i < p.nsplit; i += 256) spl[i] = p.splitters[i];
    for (int i = tid; i < kSplitPrefixes / 8; i += 256)
      reinterpret_cast<uint4*>(spt)[i] = reinterpret_cast<const uint4*>(p.split_table)[i];
  }
  // the table's window: its first splitter and the prefix shift, after the entries
  const uint32_t sbase = SPLIT ? reinterpret_cast<const uint32_t*>(p.split_table + kSplitPrefixes)[0] : 0u;
  const uint32_t ssh = SPLIT ? reinterpret_cast<const uint32_t*>(p.split_table + kSplitPrefixes)[1] : 0u;
  auto dig = [&](uint32_t x) -> uint32_t {
    if constexpr (SPLIT) return split_bucket(spl, spt, sbase, ssh, x);
    else return (x >> shift) & mask;
  };
  // splitter mode: the buckets of keys i..i+3 (i a multiple of 4) kept for the sweep
  auto put4 = [&](int64_t i, uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3) {
    if constexpr (SPLIT)
      if (p.labels) *reinterpret_cast<uint32_t*>(p.labels + i) = d0 | (d1 << 8) | (d2 << 16) | (d3 << 24);
  };
  const int64_t t0 = (int64_t)blockIdx.x * kCountTilesPerBlock;
  const bool segmented = p.seg_offs != nullptr;
  if (segmented) tiles = min(tiles, (int64_t)ld_relaxed(p.num_tiles));
  // Sort passes: pass 0 ORs the keys into sel.vary; a later pass reads the buffer
  // the previous run wrote, or returns if its digit never varies.
  const bool fill_vary = p.sel.vary && p.sel.q == 0;
  const bool sel_later = p.sel.vary && p.sel.q > 0;
  __shared__ const uint32_t* s_keys;  // the device's choice of input, or nullptr: pass skipped
  auto resolve = [&]() -> bool {      // false: this pass is skipped; ends with a barrier
    if (!sel_later) return true;
    if (tid == 0) {
      const uint32_t* sk;
      const void* sv;
      uint32_t* dk;
      void* dv;
      s_keys = pass_buffers(p.sel, vary_bits(p.sel), sk, sv, dk, dv) ? sk : nullptr;
    }
    BCF_SYNC();
    if (!s_keys) return false;
    p.keys = s_keys;
    return true;
  };
  if (!resolve()) return;
  __shared__ uint32_t orw[2];
  uint32_t o1 = 0, o0 = 0;
  auto or4 = [&](const uint4& x) {
    o1 |= x.x | x.y | x.z | x.w;
    o0 |= ~x.x | ~x.y | ~x.z | ~x.w;
  };
  if constexpr (FAST && NV <= 4) {
    // Four full tiles: every load in flight before any count, and the four counts
    // of a digit stored together (the count rows' stride is a multiple of 4 words
    // and t0 a multiple of 4).  The counters are private to a lane -- lane l only
    // ever adds to words in bank l -- so the 32 lanes of a counting atomic touch
    // 32 different banks whatever the digits (the conflict avoidance condition of
    // Sec. 1).  A byte suffices: a lane's counter of one tile sees at most T / 32
    // keys.  Thread (t, g) then sums the 32 lane words of digit group g of tile t,
    // reading them along a diagonal so that the 8 threads of one 16-byte access
    // phase read 8 different bank quads.
    static_assert(T / 32 <= 255 && RADIX % 32 == 0, "byte counters, whole 16-byte phases");
    if (!segmented && (t0 + 4) * T <= p.n) {
      const int lane = tid & 31;
      uint4* lz = reinterpret_cast<uint4*>(&lc[0][0][0]);
      for (int i = tid; i < RADIX * 8; i += 256) lz[i] = make_uint4(0u, 0u, 0u, 0u);
      uint4 x[4][NV];
      const uint4* k4 = reinterpret_cast<const uint4*>(p.keys + t0 * T);
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < NV; ++q) x[t][q] = __ldcs(k4 + t * (T / 4) + tid + 256 * q);
      BCF_SYNC();
      auto count = [&](int t, uint32_t k) -> uint32_t {
        const uint32_t d = dig(k);
        BCF_TR(&lc[t][d >> 2][lane], 4, 2, TS_TILE_COUNT_ATOM);
        atomicAdd(&lc[t][d >> 2][lane], 1u << (8 * (d & 3u)));
        return d;
      };
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const uint32_t d0 = count(t, x[t][q].x), d1 = count(t, x[t][q].y);
          const uint32_t d2 = count(t, x[t][q].z), d3 = count(t, x[t][q].w);
          put4((t0 + t) * T + 4 * (tid + 256 * q), d0, d1, d2, d3);
          if (fill_vary) or4(x[t][q]);
        }
      BCF_SYNC();
      if (tid < RADIX) {  // RADIX pairs (tile, group of four digits)
        const int t = tid / (RADIX / 4), g = tid % (RADIX / 4);
        const uint4* row = reinterpret_cast<const uint4*>(&lc[t][g][0]);
        uint32_t ev = 0, od = 0;  // bytes 0 and 2, bytes 1 and 3: 16-bit sums
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          BCF_TR(&row[(m + g) & 7], 16, 0, TS_TILE_COUNT_SUM);
          const uint4 w = row[(m + g) & 7];
          ev += (w.x & 0x00FF00FFu) + (w.y & 0x00FF00FFu) + (w.z & 0x00FF00FFu) + (w.w & 0x00FF00FFu);
          od += ((w.x >> 8) & 0x00FF00FFu) + ((w.y >> 8) & 0x00FF00FFu) + ((w.z >> 8) & 0x00FF00FFu) +
                ((w.w >> 8) & 0x00FF00FFu);
        }
        BCF_TR(&h4[t][4 * g], 16, 1, TS_TILE_COUNT_SUM);
        *reinterpret_cast<uint4*>(&h4[t][4 * g]) = make_uint4(ev & 0xFFFFu, od & 0xFFFFu, ev >> 16, od >> 16);
      }
      BCF_SYNC();
      for (int d = tid; d < RADIX; d += 256) {
        const uint4 c = make_uint4(h4[0][d], h4[1][d], h4[2][d], h4[3][d]);
        *reinterpret_cast<uint4*>(p.counts + (size_t)d * p.stride + t0) = c;
        if (p.totals && (c.x | c.y | c.z | c.w)) atomicAdd(&p.totals[d], c.x + c.y + c.z + c.w);
      }
      if (fill_vary) or_into_vary(o1, o0, p.sel.vary, orw);
      return;
    }
  }
  for (int64_t tile = t0; tile < min(t0 + kCountTilesPerBlock, tiles); ++tile) {
    int64_t start = tile * T, hi = p.n;
    uint32_t wseg = 0;  // segment mode with seg_w: the segment's label bound
    if (segmented) {
      const int seg = p.tile_seg[tile];
      start = p.seg_offs[seg] + (tile - p.seg_tile0[seg]) * (int64_t)T;
      hi = p.seg_offs[seg + 1];
      if constexpr (!FAST)  // the segment-mode instance
        if (p.seg_w) wseg = (uint32_t)p.seg_w[seg];
    }
    const int cnt = (int)min((int64_t)T, hi - start);
    for (int i = tid; i < RADIX; i += 256) h[i] = 0;
    BCF_SYNC();
    const uint32_t* k = p.keys + start;
    // four keys i..i+3 of an unsegmented tile counted (and, splitter mode, their buckets kept)
    auto count4 = [&](const uint4& xv, int64_t i) {
      const uint32_t d0 = dig(xv.x), d1 = dig(xv.y), d2 = dig(xv.z), d3 = dig(xv.w);
      atomicAdd(&h[d0], 1u);
      atomicAdd(&h[d1], 1u);
      atomicAdd(&h[d2], 1u);
      atomicAdd(&h[d3], 1u);
      put4(i, d0, d1, d2, d3);
      if (fill_vary) or4(xv);
    };
    if (segmented) {
      // Segment starts need not be 16-byte aligned: 16-byte loads of the aligned
      // window around the tile (at most T/1024 + 1 per thread, all in flight
      // before any count), counting only the tile's own elements; a vector that
      // would pass the array's end is read element by element.
      const int mis = (int)((reinterpret_cast<uintptr_t>(k) & 15u) >> 2);
      const int64_t a0 = start - mis;  // element index of the window's first word
      const uint4* k4 = reinterpret_cast<const uint4*>(p.keys + a0);
      const int nv = (cnt + mis + 3) >> 2;
      constexpr int NVS = T / 1024 + 1;
      uint4 xv[NVS];
#pragma unroll
      for (int j = 0; j < NVS; ++j) {
        const int v = tid + 256 * j;
        const int e0 = v * 4 - mis;  // tile-relative index of the vector's first element
        if (v < nv && a0 + (int64_t)v * 4 + 4 <= p.n) {
          xv[j] = __ldcs(k4 + v);
        } else if (v < nv) {
          uint32_t x[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) x[c] = (e0 + c >= 0 && e0 + c < cnt) ? k[e0 + c] : 0u;
          xv[j] = make_uint4(x[0], x[1], x[2], x[3]);
        }
      }
      bool bad = false;
#pragma unroll
      for (int j = 0; j < NVS; ++j) {
        const int v = tid + 256 * j;
        if (v >= nv) continue;
        const int e0 = v * 4 - mis;
        const uint32_t x[4] = {xv[j].x, xv[j].y, xv[j].z, xv[j].w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (e0 + c >= 0 && e0 + c < cnt) {
            atomicAdd(&h[dig(x[c])], 1u);
            if constexpr (!FAST) bad |= p.seg_w && x[c] >= wseg;
          }
      }
      if (!FAST && bad) set_status(p.status, DEV_BAD_KEY);
    } else if (cnt == T) {  // full tile: all T/1024 vector loads in flight before counting
      constexpr int NV = T / 1024;
      uint4 x[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) x[q] = __ldcs(reinterpret_cast<const uint4*>(k) + tid + 256 * q);
#pragma unroll
      for (int q = 0; q < NV; ++q) count4(x[q], start + 4 * (tid + 256 * q));
    } else {
      const int nv = cnt >> 2;
      for (int v = tid; v < nv; v += 256) count4(__ldcs(reinterpret_cast<const uint4*>(k) + v), start + 4 * v);
      for (int i = nv * 4 + tid; i < cnt; i += 256) {
        const uint32_t d = dig(k[i]);
        atomicAdd(&h[d], 1u);
        if (SPLIT && p.labels) p.labels[start + i] = (uint8_t)d;
        if (fill_vary) {
          o1 |= k[i];
          o0 |= ~k[i];
        }
      }
    }
    BCF_SYNC();
    for (int d = tid; d < RADIX; d += 256) {
      const uint32_t c = h[d];
      p.counts[(size_t)d * p.stride + tile] = c;
      tot[d] += c;
    }
    BCF_SYNC();
  }
  if (p.totals)
    for (int d = tid; d < RADIX; d += 256)
      if (tot[d]) atomicAdd(&p.totals[d], tot[d]);
  if (fill_vary) or_into_vary(o1, o0, p.sel.vary, orw);
}

// One block per digit: exclusive scan of the digit's tile counts, offset by the
// digit's global start (sum of smaller digits' totals, or b*n/w for a balanced
// partition, whose counts are checked here).  Entry `tiles` receives the digit's
// total run end, so stride must exceed tiles.
constexpr int kScanPerThread = 16;

template <int kScanThreads>
__global__ void __launch_bounds__(kScanThreads) k_scan_offsets_t(uint32_t* counts, int64_t tiles,
                                                                 int64_t stride, const uint32_t* totals,
                                                                 int balanced, int64_t n, int w,
                                                                 unsigned* status, PassSel sel) {
  constexpr int R = kScanPerThread / 4;
  __shared__ uint32_t scratch[R * 32];
  __shared__ uint32_t s_base;
  const int d = blockIdx.x;
  const int tid = threadIdx.x;
  uint32_t* row = counts + (size_t)d * stride;
  // A chunk is kScanPerThread / 4 rounds; in round r thread t holds the four
  // counts at r * 4 * kScanThreads + 4t, so every warp-wide load and store covers
  // 512 contiguous bytes (rows start 16-byte aligned: every caller's stride is a
  // multiple of the look-back window, 4 or 8 words).  The rounds' sums are
  // scanned together, one set of barriers per chunk.  The first chunk's counts
  // are loaded before the digit start is summed, so that the two global reads
  // overlap.
  constexpr int64_t CH = (int64_t)kScanThreads * kScanPerThread;
  uint4 v[R];
  auto at = [&](int64_t c0, int r) { return c0 + (int64_t)r * 4 * kScanThreads + 4 * tid; };
  auto load = [&](int64_t c0) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i0 = at(c0, r);
      if (i0 + 4 <= tiles) {
        v[r] = *reinterpret_cast<const uint4*>(row + i0);
      } else {
        v[r].x = i0 < tiles ? row[i0] : 0u;
        v[r].y = i0 + 1 < tiles ? row[i0 + 1] : 0u;
        v[r].z = i0 + 2 < tiles ? row[i0 + 2] : 0u;
        v[r].w = i0 + 3 < tiles ? row[i0 + 3] : 0u;
      }
    }
  };
  load(0);
  __shared__ int s_skip;
  if (tid < 32) {  // digit start: warp-wide sum of the smaller digits' totals
    uint32_t b = 0;
    if (totals && !balanced)
      for (int e = tid; e < d; e += 32) b += totals[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (tid == 0) {
      if (balanced) {
        b = (uint32_t)min((int64_t)d * (n / w), n);
        const uint32_t expect = d < w ? (uint32_t)(n / w) : 0u;
        if (totals && totals[d] != expect) set_status(status, DEV_NOT_BALANCED);
      }
      s_base = b;  // segment mode (no totals): plain running sums from 0
      // a skipped sort pass: nothing to scan (its counts were never written)
      s_skip = sel.vary && !((passes_run_mask(sel, vary_bits(sel)) >> sel.q) & 1u);
    }
  }
  BCF_SYNC();
  if (s_skip) return;
  uint32_t carry = s_base;
  for (int64_t c0 = 0; c0 < tiles; c0 += CH) {
    if (c0 > 0) load(c0);
    uint32_t sum[R], ex[R], total[R];
#pragma unroll
    for (int r = 0; r < R; ++r) sum[r] = v[r].x + v[r].y + v[r].z + v[r].w;
    block_excl_scan_n<kScanThreads, R>(sum, ex, scratch, total);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t run = carry + ex[r];
      uint4 o;
      o.x = run;
      run += v[r].x;
      o.y = run;
      run += v[r].y;
      o.z = run;
      run += v[r].z;
      o.w = run;
      const int64_t i0 = at(c0, r);
      if (i0 + 4 <= tiles) {
        *reinterpret_cast<uint4*>(row + i0) = o;
      } else {
        if (i0 < tiles) row[i0] = o.x;
        if (i0 + 1 < tiles) row[i0 + 1] = o.y;
        if (i0 + 2 < tiles) row[i0 + 2] = o.z;
      }
      carry += total[r];
    }
  }
  if (tid == 0 && tiles < stride) row[tiles] = carry;  // end of the digit's runs
}

// One block per digit; a block of 256 threads covers 4096 tiles in one step, so
// only larger tile counts take 1024 (fewer idle threads at every barrier).
// sel.vary != nullptr: a sort pass that may be skipped.
static inline cudaError_t launch_scan_offsets(int radix, uint32_t* counts, int64_t tiles, int64_t stride,
                                              const uint32_t* totals, int balanced, int64_t n, int w,
                                              unsigned* status, cudaStream_t s, const PassSel& sel = PassSel{}) {
  if (tiles <= 256 * kScanPerThread)
    k_scan_offsets_t<256><<<radix, 256, 0, s>>>(counts, tiles, stride, totals, balanced, n, w, status, sel);
  else
    k_scan_offsets_t<1024><<<radix, 1024, 0, s>>>(counts, tiles, stride, totals, balanced, n, w, status, sel);
  return cudaGetLastError();
}

// ------------------------------------------------------------- one sweep
template <int THREADS, int IPT, int BITS, int VB, bool SPLIT = false>
struct SweepSmem {
  static constexpr int T = THREADS * IPT;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int RADIX = 1 << BITS;
  static constexpr size_t keys = 0;                        // T + 4 slots (staging offset)
  static constexpr size_t vals = keys + (size_t)(T + 4) * 4;
  static constexpr size_t whist = vals + (size_t)(T + 4) * VB;
  static constexpr size_t tstart = whist + (size_t)WARPS * RADIX * 4;
  static constexpr size_t gofs = tstart + (size_t)RADIX * 4;
  static constexpr size_t scratch = gofs + (size_t)RADIX * 4;
  static constexpr size_t mbar = scratch + 32 * 4;
  static constexpr size_t info = mbar + 8;                 // tile, seg
  static constexpr size_t sdig = info + 16;                // splitter mode: digit of each ordered key
  static constexpr size_t mbins = (sdig + (SPLIT ? (size_t)T : 0) + 15) / 16 * 16;  // peer masks
  static constexpr size_t bytes = mbins + (BCF_PEERS_MATCH == 2 ? (size_t)WARPS * RADIX * 4 : 0);
  static_assert(scratch % 8 == 0, "scratch also carries pointers; mbar needs 8-byte alignment");
};

template <int THREADS, int IPT, int BITS, int VB, bool SPLIT = false>
__global__ void __launch_bounds__(THREADS, (VB == 8 ? 2 : BCF_SWEEP_MINBLOCKS) * 256 / THREADS > 0
                                               ? (VB == 8 ? 2 : BCF_SWEEP_MINBLOCKS) * 256 / THREADS
                                               : 1) k_sweep(SweepParams p) {
  using VT = typename ValT<VB>::type;
  using S = SweepSmem<THREADS, IPT, BITS, VB, SPLIT>;
  constexpr int T = S::T, RADIX = S::RADIX;
  constexpr uint32_t DMASK = RADIX - 1;
  static_assert(RADIX <= THREADS, "one thread per digit");
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* keys_s = reinterpret_cast<uint32_t*>(smem + S::keys);
  VT* vals_s = reinterpret_cast<VT*>(smem + S::vals);
  unsigned long long* kv_s = reinterpret_cast<unsigned long long*>(smem + S::keys);
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + S::whist);
  uint32_t* tstart = reinterpret_cast<uint32_t*>(smem + S::tstart);
  uint32_t* gofs = reinterpret_cast<uint32_t*>(smem + S::gofs);
  uint32_t* scratch = reinterpret_cast<uint32_t*>(smem + S::scratch);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::mbar);
  int* s_info = reinterpret_cast<int*>(smem + S::info);
  uint8_t* sdig = reinterpret_cast<uint8_t*>(smem + S::sdig);
  uint32_t* mbins = reinterpret_cast<uint32_t*>(smem + S::mbins);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool segmented = p.seg_offs != nullptr;

  // Sort pass with device-side skipping: one thread finds whether the pass runs
  // and which buffers it reads and writes, and hands that to the block.
  struct Choice {
    const uint32_t* sk;
    const void* sv;
    uint32_t* dk;
    void* dv;
    int runs;
  };
  Choice* ch = reinterpret_cast<Choice*>(scratch);
  // Look-back mode takes tiles in launch order (atomic ticket) so that every tile
  // a look-back waits on belongs to a block that is already running.
  if (tid == 0) {
    if (p.sel.vary) {
      Choice c;
      c.runs = pass_buffers(p.sel, vary_bits(p.sel), c.sk, c.sv, c.dk, c.dv);
      *ch = c;
      if (c.runs && blockIdx.x == 0) atomicOr(p.sel.ran, 1u << p.sel.q);
    }
    const int tile = p.tile_offsets ? (int)blockIdx.x : (int)atomicAdd(p.ticket, 1u);
    s_info[0] = tile;
    s_info[1] = (segmented && (uint32_t)tile < ld_relaxed(p.num_tiles)) ? p.tile_seg[tile] : -1;
  }
  BCF_SYNC();
  if (p.sel.vary) {
    const Choice c = *ch;
    if (!c.runs) return;  // skipped pass: nothing to move
    p.keys_in = c.sk;
    p.vals_in = c.sv;
    p.keys_out = c.dk;
    p.vals_out = c.dv;
  }
  const int tile = s_info[0];
  if (segmented && s_info[1] < 0) return;  // more blocks than tiles this time
  const int seg = s_info[1];
  int64_t lo = 0, hi = p.n;  // bounds of the problem this tile belongs to
  int t_in = tile, w = p.w;
  if (segmented) {
    lo = p.seg_offs[seg];
    hi = p.seg_offs[seg + 1];
    t_in = tile - p.seg_tile0[seg];
    if (p.seg_w) w = p.seg_w[seg];
  }
  const int64_t start = lo + (int64_t)t_in * T;
  const int cnt = (int)min((int64_t)T, hi - start);
  const bool last_tile = start + cnt >= hi;
  const int shift = p.shift;  // digit = (key >> shift) & (RADIX - 1); labels use shift 0
  const bool label_mode = w > 0;

  // Stage the tile: bulk copy of the 16-byte-aligned window, plain loads for the
  // ragged end.  Element i of the tile is keys_s[ksh + i].  vals_in == nullptr
  // with 4-byte payloads: the payload is the input position.
  int ksh = 0, vsh = 0, kfull = 0, vfull = 0;
  bool iota = false;
  auto stage = [&]() {
    ksh = (int)((reinterpret_cast<uintptr_t>(p.keys_in + start) & 15u) >> 2);
    iota = VB == 4 && p.vals_in == nullptr;
    vsh = (VB && !iota) ? (int)((reinterpret_cast<uintptr_t>(reinterpret_cast<const VT*>(p.vals_in) + start) & 15u) / VB) : 0;
    kfull = ((ksh + cnt) * 4 & ~15) / 4;  // elements covered by the bulk copy
    vfull = (VB && !iota) ? (((vsh + cnt) * VB) & ~15) / VB : 0;
    if (tid == 0) {
      mbar_init(mbar, 1);
      mbar_arrive_expect_tx(mbar, (unsigned)(kfull * 4 + vfull * VB));
      if (kfull) bulk_g2s(keys_s, p.keys_in + start - ksh, (unsigned)kfull * 4, mbar);
      if (VB && vfull)
        bulk_g2s(vals_s, reinterpret_cast<const VT*>(p.vals_in) + start - vsh, (unsigned)(vfull * VB), mbar);
    }
  };
  stage();
  for (int i = tid; i < S::WARPS * RADIX; i += THREADS) whist[i] = 0;
#if BCF_PEERS_MATCH == 2
  for (int i = tid; i < S::WARPS * RADIX; i += THREADS) mbins[i] = 0;
#endif
  for (int i = max(kfull - ksh, 0) + tid; i < cnt; i += THREADS) keys_s[ksh + i] = p.keys_in[start + i];
  if (VB && !iota) {
    for (int i = max(vfull - vsh, 0) + tid; i < cnt; i += THREADS)
      vals_s[vsh + i] = reinterpret_cast<const VT*>(p.vals_in)[start + i];
  }
  // Splitter mode: the buckets the tile counts kept, four per register, loaded
  // while the tile is staged (lane l of warp q takes items q*32*IPT + 32j + l).
  uint32_t dl[SPLIT ? (IPT + 3) / 4 : 1] = {};
  if constexpr (SPLIT) {
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const int idx = warp * 32 * IPT + j * 32 + lane;
      if (idx < cnt) dl[j >> 2] |= (uint32_t)__ldcs(p.labels + start + idx) << (8 * (j & 3));
    }
  }
  BCF_SYNC();  // mbarrier initialised before anyone waits on it
  mbar_wait(mbar, 0, p.status);
  BCF_SYNC();

  // The rest is written once for full tiles (no per-key bounds tests) and once
  // for the ragged last tile.
  auto body = [&](auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    auto in_tile = [&](int idx) { return FULL || idx < cnt; };

    // Registers, warp-striped: lane l of warp q holds tile items q*32*IPT + 32j + l.
    // Reading them is the strided pattern: lane l always in bank (l + shift).
    uint32_t key[IPT];
    VT val[IPT];
    const int wbase = warp * 32 * IPT;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const int idx = wbase + j * 32 + lane;
      const bool valid = in_tile(idx);
      if (valid) BCF_TR(&keys_s[ksh + idx], 4, 0, TS_STAGE_READ);
      key[j] = valid ? keys_s[ksh + idx] : 0u;
      if (VB && valid && !iota) BCF_TR(&vals_s[vsh + idx], VB, 0, TS_STAGE_READ);
      if (VB) val[j] = !valid ? VT(0) : (iota ? VT(start + idx) : vals_s[vsh + idx]);
      if (label_mode && valid && key[j] >= (uint32_t)w) set_status(p.status, DEV_BAD_KEY);
    }
    // Splitter mode: the keys' buckets, four 8-bit digits per register.
    auto digit = [&](int j) -> uint32_t {
      if constexpr (SPLIT) return (dl[j >> 2] >> (8 * (j & 3))) & 0xFFu;
      else return (key[j] >> shift) & DMASK;
    };

    // Phase A -- counts: every warp histograms its own keys (the row "radix sort"
    // count of Corollary 1, one histogram per warp).
    uint32_t* wh = whist + warp * RADIX;
#pragma unroll
    for (int j = 0; j < IPT; ++j)
      if (in_tile(wbase + j * 32 + lane)) {
        BCF_TR(&wh[digit(j)], 4, 2, TS_COUNT_ATOM);
        atomicAdd(&wh[digit(j)], 1u);
      }
    BCF_SYNC();

    // Phase B -- per digit: tile count, tile-exclusive start, and each warp's base
    // (tile start + counts of earlier warps).  In look-back mode the tile count is
    // published at once so that later tiles can look past this one while it ranks.
    uint32_t count = 0;
    if (tid < RADIX) {
#pragma unroll 4
      for (int q = 0; q < S::WARPS; ++q) count += whist[q * RADIX + tid];
    }
    uint32_t total;
    const uint32_t tile_excl = block_excl_scan<THREADS>(tid < RADIX ? count : 0u, scratch, &total);
    uint32_t* lbd = p.lookback + (size_t)tid * p.lb_stride;  // digit-major status words
    if (tid < RADIX) {
      if (!p.tile_offsets && tile + 1 != p.silent_tile1)
        st_relaxed(lbd + tile, (t_in == 0 ? LB_INC : LB_AGG) | count);
      tstart[tid] = tile_excl;
      uint32_t run = tile_excl;
#pragma unroll 4
      for (int q = 0; q < S::WARPS; ++q) {
        const uint32_t c = whist[q * RADIX + tid];
        whist[q * RADIX + tid] = run;
        run += c;
      }
    }
    BCF_SYNC();

    // Phase C -- rank and scatter into shared memory in digit order.  Peers with
    // the same digit come from one ballot per digit bit; the lowest peer claims the
    // run for all of them with one shared atomic.
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const bool valid = in_tile(wbase + j * 32 + lane);
      const uint32_t d = digit(j);
      unsigned peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
#if BCF_PEERS_MATCH == 2
      // Every lane sets its bit in its digit's word; the word then is the peer set.
      uint32_t* mb = mbins + warp * RADIX + d;
      if (valid) atomicOr(mb, 1u << lane);
      __syncwarp();
      peers = valid ? *mb : 0u;
#elif BCF_PEERS_MATCH
      peers &= __match_any_sync(0xffffffffu, valid ? d : 0xFFFFFFFFu);
#else
#pragma unroll
      for (int b = 0; b < BITS; ++b) {
        const unsigned bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
      }
#endif
      const int leader = valid ? __ffs(peers) - 1 : lane;
      uint32_t old = 0;
      if (valid && lane == leader) {
        BCF_TR(&wh[d], 4, 2, TS_CLAIM_ATOM);
        old = atomicAdd(&wh[d], (uint32_t)__popc(peers));
      }
      old = __shfl_sync(0xffffffffu, old, leader);
#if BCF_PEERS_MATCH == 2
      if (valid && lane == leader) *mb = 0u;  // every peer has read the word (shuffle above)
      __syncwarp();
#endif
      if (valid) {
        const uint32_t pos = old + __popc(peers & lt);
        if constexpr (SPLIT) sdig[pos] = (uint8_t)d;
        if constexpr (VB == 4) {
          BCF_TR(&kv_s[pos], 8, 1, TS_SCATTER);
          kv_s[pos] = ((unsigned long long)val[j] << 32) | key[j];
        } else {
          BCF_TR(&keys_s[pos], 4, 1, TS_SCATTER);
          keys_s[pos] = key[j];
          if (VB) BCF_TR(&vals_s[pos], VB, 1, TS_SCATTER);
          if (VB) vals_s[pos] = val[j];
        }
      }
    }
  };
  if (cnt == T) body(std::true_type{});
  else body(std::false_type{});

  // Global offsets.  Reduce-then-scan mode: the run start was scanned ahead of
  // this launch.  Otherwise decoupled look-back (one thread per digit): add
  // earlier tiles' counts until one has published its inclusive prefix; the
  // digit's status words of consecutive tiles are contiguous, so one read of
  // kLookbackWindow words covers that many tiles.
  uint32_t* lbd = p.lookback + (size_t)tid * p.lb_stride;
  if (tid < RADIX && p.tile_offsets) {
    const uint32_t* row = p.tile_offsets + (size_t)tid * p.lb_stride;
    uint32_t base = row[tile];
    if (segmented) {  // running sums cover all tiles: rebase at the segment's first tile
      const int first = tile - t_in;
      const uint32_t before = base - row[first];  // this digit in earlier tiles of the segment
      const uint32_t mine = (tid + 1 < RADIX ? tstart[tid + 1] : (uint32_t)cnt) - tstart[tid];
      if (p.balanced) {
        const int64_t len = hi - lo;
        base = (uint32_t)min(lo + (int64_t)tid * (len / max(w, 1)), hi) + before;
        if (last_tile) {
          const uint32_t expect = tid < w ? (uint32_t)(len / max(w, 1)) : 0u;
          if (before + mine != expect) set_status(p.status, DEV_NOT_BALANCED);
        }
      } else {
        base = p.seg_base[(size_t)p.seg_slot[seg] * RADIX + tid] + before;
      }
    }
    gofs[tid] = base - tstart[tid];
  } else if (tid < RADIX) {
    uint32_t excl = 0;
    const uint32_t count = ld_relaxed(lbd + tile) & LB_MASK;  // own aggregate, published above
    if (t_in > 0) {
      const int first = tile - t_in;
      int j = tile - 1;  // next tile to consume
      unsigned spins = 0;
      constexpr int W = kLookbackWindow;
      while (j >= first) {
        const int ws = j - (j % W);  // W-aligned window [ws, ws + W)
        uint32_t wv[W];
#pragma unroll
        for (int q = 0; q < W; q += 4) {
          const uint4 a = ld_relaxed_v4(lbd + ws + q);
          wv[q] = a.x;
          wv[q + 1] = a.y;
          wv[q + 2] = a.z;
          wv[q + 3] = a.w;
        }
        bool done = false, stalled = false;
#pragma unroll
        for (int q = W - 1; q >= 0; --q) {
          const int tt = ws + q;
          if (done || stalled || tt > j || tt < first) continue;
          const uint32_t f = wv[q] & ~LB_MASK;
          if (f == 0) {
            stalled = true;  // not published yet: poll this tile again
            continue;
          }
          excl += wv[q] & LB_MASK;
          j = tt - 1;
          if (f == LB_INC) done = true;
        }
        if (done) break;
        if (stalled && ++spins > (p.spin_limit ? p.spin_limit : kSpinLimit)) {
          set_status(p.status, DEV_TIMEOUT);
          break;
        }
        if (!stalled && j >= ws) j = ws - 1;  // window below `first`: finished
      }
      if (tile + 1 != p.silent_tile1) st_relaxed(lbd + tile, LB_INC | (excl + count));
    }
    uint32_t base;  // absolute start of this digit's block
    if (p.balanced) {
      const int64_t len = hi - lo;
      const int64_t b = lo + (int64_t)tid * (len / max(w, 1));
      base = (uint32_t)min(b, hi);
      if (last_tile) {
        const uint32_t expect = tid < w ? (uint32_t)(len / max(w, 1)) : 0u;
        if (excl + count != expect) set_status(p.status, DEV_NOT_BALANCED);
      }
    } else if (segmented) {
      base = p.seg_base[(size_t)p.seg_slot[seg] * RADIX + tid];
    } else {
      base = p.digit_base[tid];
    }
    gofs[tid] = base + excl - tstart[tid];
  }
  BCF_SYNC();

  // Write out: consecutive threads take consecutive sorted positions, so the
  // stores of one digit's run are contiguous in global memory.  Positions are
  // below 2^30, so 32-bit arithmetic suffices; dst outside [lo, hi) (only possible
  // with invalid labels) is never written.
  VT* vout = reinterpret_cast<VT*>(p.vals_out);
  const uint32_t lo32 = (uint32_t)lo, len32 = (uint32_t)(hi - lo);
  for (int i = tid; i < cnt; i += THREADS) {
    uint32_t k;
    VT v = VT(0);
    if constexpr (VB == 4) {
      BCF_TR(&kv_s[i], 8, 0, TS_WRITEOUT_READ);
      const unsigned long long x = kv_s[i];
      k = (uint32_t)x;
      v = (uint32_t)(x >> 32);
    } else {
      BCF_TR(&keys_s[i], 4, 0, TS_WRITEOUT_READ);
      k = keys_s[i];
      if (VB) BCF_TR(&vals_s[i], VB, 0, TS_WRITEOUT_READ);
      if (VB) v = vals_s[i];
    }
    uint32_t dk;
    if constexpr (SPLIT) dk = sdig[i];
    else dk = (k >> shift) & DMASK;
    BCF_TR(&gofs[dk], 4, 0, TS_OFFSET_READ);
    const uint32_t dst = gofs[dk] + (uint32_t)i;
    if (dst - lo32 < len32) {
      p.keys_out[dst] = k;
      if (VB) vout[dst] = v;
    }
  }
}

template <int BITS, int VB, int THREADS = kSweepThreads, int IPT = kSweepIPT, bool SPLIT = false>
inline cudaError_t launch_sweep(const SweepParams& p, int64_t grid, cudaStream_t s) {
  using S = SweepSmem<THREADS, IPT, BITS, VB, SPLIT>;
  auto kern = k_sweep<THREADS, IPT, BITS, VB, SPLIT>;
  // The shared-memory limit is raised on every launch that needs it, not once per
  // process: this launcher is instantiated in several translation units, and a
  // flag shared between them could stand for another unit's copy of the kernel.
  if (S::bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
  }
  if (grid <= 0) return cudaSuccess;
  kern<<<(unsigned)grid, THREADS, S::bytes, s>>>(p);
  return cudaGetLastError();
}

template <int BITS, int THREADS = kSweepThreads, int IPT = kSweepIPT, bool SPLIT = false>
inline cudaError_t sweep_dispatch(const SweepParams& p, int64_t grid, int vb, cudaStream_t s) {
  switch (vb) {
    case 0: return launch_sweep<BITS, 0, THREADS, IPT, SPLIT>(p, grid, s);
    case 4: return launch_sweep<BITS, 4, THREADS, IPT, SPLIT>(p, grid, s);
    case 8: return launch_sweep<BITS, 8, THREADS, IPT, SPLIT>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bcf
