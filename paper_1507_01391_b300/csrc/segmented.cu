// segmented.cu -- batched forms: many independent CSR segments in one call, and
// the tile sort (Lemma 1) on its own.
//
// Everything is planned on the device, so a call issues a fixed sequence of
// launches with no host synchronisation and no allocation (capturable in a CUDA
// graph):
//   1. k_seg_plan   one block scans the CSR offsets: segments up to one tile go to
//                   the small-segment queue, longer ones get a run of sweep tiles;
//   2. k_seg_small  (sort only) persistent blocks pull small segments from the
//                   queue and sort each whole in shared memory with the Lemma 1
//                   schedule (tile_sort.cuh): one read and one write per key.
//                   Segments of more than kTinyMax keys take a tile each; tiny ones
//                   are packed, in order, into bins of consecutive tiny segments
//                   whose key counts sum to less than a tile (a bin holds the
//                   segments whose running key offset lies in one kTinyMax-wide
//                   interval), and a bin is sorted as one tile of items ordered by
//                   (segment in the bin, key, position);
//   3. per digit pass: k_tile_counts over the long segments' tiles, k_scan_offsets
//                   (running sums over all tiles), k_seg_digit_base (each segment's
//                   digit starts from those sums), then k_sweep in segment mode: a
//                   tile's run start is its running sum minus the one at its
//                   segment's first tile, plus the segment's digit start.
// Launch grids are host-side upper bounds; blocks without work exit at once.
#include "common.cuh"
#include "internal.h"
#include "onesweep.cuh"
#include "sweep.cuh"
#include "tile_sort.cuh"

namespace bcf {

enum : int { C_NSMALL = 0, C_NLARGE = 1, C_NTILES = 2, C_QUEUE = 3, C_TICKET = 4 /* +pass */,
             C_NTINY = 8, C_NBINS = 9 };

// Tiny segments (1..kTinyMax keys) share tiles: a bin's keys sum to at most
// 2 * kTinyMax - 1 < kL1Tile.
constexpr int kTinyMax = kL1Tile / 2;

struct PlanParams {
  const int64_t* offs;
  int64_t nseg, n_total;
  int small_max;        // segments with 1..small_max keys go to the small queue
  int tile;             // sweep tile
  int64_t tiles_cap;    // capacity of tile_seg
  int64_t slots_cap;    // capacity of slot_seg
  const int32_t* seg_w; // partition widths (checked when given)
  int32_t* small_ids;   // segments of kTinyMax + 1 .. small_max keys (a tile each)
  int32_t* tiny_ids;    // segments of 1 .. kTinyMax keys, in order
  uint32_t* bin_first;  // per bin: ~(index in tiny_ids of its first segment), max-reduced
  int64_t bins_cap;
  int32_t* seg_slot;
  int32_t* seg_tile0;
  int32_t* tile_seg;
  int32_t* slot_seg;
  uint32_t* ctr;
  unsigned* status;
};

constexpr int kPlanThreads = 1024;

__global__ void __launch_bounds__(kPlanThreads) k_seg_plan(PlanParams p) {
  __shared__ uint32_t scratch[32];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = (p.nseg > 0 && (p.offs[0] != 0 || p.offs[p.nseg] != p.n_total)) ? 1 : 0;
  BCF_SYNC();
  uint32_t run_small = 0, run_large = 0, run_tiles = 0, run_tiny = 0, run_tiny_keys = 0;
  for (int64_t base = 0; base < p.nseg; base += kPlanThreads) {
    const int64_t s = base + tid;
    int64_t len = 0;
    if (s < p.nseg) {
      const int64_t a = p.offs[s], b = p.offs[s + 1];
      if (a < 0 || b < a || b > p.n_total) bad = 1;  // benign race: every writer stores 1
      else len = b - a;
      if (p.seg_w && (p.seg_w[s] < 1 || p.seg_w[s] > 256)) {
        bad = 1;
        len = 0;
      }
    }
    const bool tiny = len > 0 && len <= kTinyMax && p.small_max > 0;
    const bool small = len > kTinyMax && len <= p.small_max;
    const bool large = len > p.small_max;
    const uint32_t tiles = large ? (uint32_t)((len + p.tile - 1) / p.tile) : 0u;
    uint32_t tot;
    const uint32_t es = block_excl_scan<kPlanThreads>(small ? 1u : 0u, scratch, &tot);
    const uint32_t add_small = tot;
    const uint32_t ey = block_excl_scan<kPlanThreads>(tiny ? 1u : 0u, scratch, &tot);
    const uint32_t add_tiny = tot;
    const uint32_t ek = block_excl_scan<kPlanThreads>(tiny ? (uint32_t)len : 0u, scratch, &tot);
    const uint32_t add_tiny_keys = tot;
    const uint32_t el = block_excl_scan<kPlanThreads>(large ? 1u : 0u, scratch, &tot);
    const uint32_t add_large = tot;
    const uint32_t et = block_excl_scan<kPlanThreads>(tiles, scratch, &tot);
    const uint32_t add_tiles = tot;
    if (s < p.nseg) {
      p.seg_slot[s] = -1;
      p.seg_tile0[s] = -1;
      if (small) p.small_ids[run_small + es] = (int32_t)s;
      if (tiny) {
        // bin = running key offset / kTinyMax; offsets grow by at most kTinyMax per
        // segment, so bins are consecutive and each bin's first segment is the
        // smallest index mapped to it
        const uint32_t idx = run_tiny + ey;
        const uint32_t bin = (run_tiny_keys + ek) / kTinyMax;
        p.tiny_ids[idx] = (int32_t)s;
        if ((int64_t)bin < p.bins_cap) atomicMax(&p.bin_first[bin], ~idx);
        else bad = 1;
      }
      if (large) {
        const uint32_t slot = run_large + el, t0 = run_tiles + et;
        if ((int64_t)slot < p.slots_cap && (int64_t)(t0 + tiles) <= p.tiles_cap) {
          p.seg_slot[s] = (int32_t)slot;
          p.seg_tile0[s] = (int32_t)t0;
          p.slot_seg[slot] = (int32_t)s;
          for (uint32_t t = 0; t < tiles; ++t) p.tile_seg[t0 + t] = (int32_t)s;
        } else {
          bad = 1;
        }
      }
    }
    run_small += add_small;
    run_large += add_large;
    run_tiles += add_tiles;
    run_tiny += add_tiny;
    run_tiny_keys += add_tiny_keys;
  }
  BCF_SYNC();
  if (tid == 0) {
    // Bins in use: every id up to the last tiny segment's bin is taken (ids grow
    // by at most one per segment).  The total key count can reach one bin past
    // it; that bin has no first segment (its word is still zero).
    uint32_t nbins = 0;
    if (run_tiny > 0) {
      nbins = (uint32_t)min((int64_t)(run_tiny_keys / kTinyMax) + 1, p.bins_cap);
      while (nbins > 0 && p.bin_first[nbins - 1] == 0u) --nbins;
    }
    p.ctr[C_NTINY] = run_tiny;
    p.ctr[C_NBINS] = nbins;
    p.ctr[C_NSMALL] = run_small;
    p.ctr[C_NLARGE] = (int64_t)run_large <= p.slots_cap ? run_large : (uint32_t)p.slots_cap;
    p.ctr[C_NTILES] = (int64_t)run_tiles <= p.tiles_cap ? run_tiles : (uint32_t)p.tiles_cap;
    if (bad) set_status(p.status, DEV_BAD_SEGMENTS);
  }
}

// Digit starts of every long segment for one pass, from that pass's running
// tile sums: the segment holds run[d][t0 + tiles] - run[d][t0] keys of digit d;
// an exclusive scan over d, offset by the segment's start, gives the starts.
// seg_w != nullptr (a balanced partition): every label below the segment's width
// must hold len / w keys, else the status records it.
__global__ void __launch_bounds__(256) k_seg_digit_base(const uint32_t* __restrict__ run,
                                                        int64_t stride, uint32_t* __restrict__ seg_base,
                                                        const int32_t* __restrict__ slot_seg,
                                                        const int32_t* __restrict__ seg_tile0,
                                                        const int64_t* __restrict__ offs,
                                                        const uint32_t* __restrict__ ctr, int tile,
                                                        const int32_t* __restrict__ seg_w, unsigned* status) {
  __shared__ uint32_t scratch[32];
  const int64_t slot = blockIdx.x;
  if (slot >= (int64_t)ctr[C_NLARGE]) return;
  const int seg = slot_seg[slot];
  const int64_t lo = offs[seg], len = offs[seg + 1] - lo;
  const int t0 = seg_tile0[seg];
  const int t1 = t0 + (int)((len + tile - 1) / tile);
  const uint32_t* r = run + (size_t)threadIdx.x * stride;
  const uint32_t c = r[t1] - r[t0];
  if (seg_w) {
    const int w = max(seg_w[seg], 1);
    if (c != ((int)threadIdx.x < w ? (uint32_t)(len / w) : 0u)) set_status(status, DEV_NOT_BALANCED);
  }
  uint32_t tot;
  const uint32_t e = block_excl_scan<256>(c, scratch, &tot);
  seg_base[(size_t)slot * 256 + threadIdx.x] = (uint32_t)lo + e;
}

// One bin of tiny segments as one Lemma 1 tile.  Segment j of the bin (j < cnt)
// occupies packed positions [cum[j], cum[j+1]); its keys become items
// (j << 44 | key << 12 | packed position), whose order is (segment, key, input
// order), so sorted position t of segment j is its rank t - cum[j].
template <int VB>
__device__ __forceinline__ void sort_bin(const uint32_t* __restrict__ keys_in, const void* __restrict__ vals_in,
                                         uint32_t* __restrict__ keys_out, void* __restrict__ vals_out,
                                         const int64_t* __restrict__ offs, const int32_t* __restrict__ ids,
                                         int cnt, unsigned long long* X, unsigned long long* Y, uint16_t* cum,
                                         uint32_t* scratch) {
  using VT = typename ValT<VB>::type;
  constexpr int PER = kL1Tile / kL1Threads;  // bin segments per thread in the scan
  const int tid = threadIdx.x;
  uint32_t len[PER], sum = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid * PER + q;
    len[q] = j < cnt ? (uint32_t)(offs[ids[j] + 1] - offs[ids[j]]) : 0u;
    sum += len[q];
  }
  uint32_t total;
  uint32_t run = block_excl_scan<kL1Threads>(sum, scratch, &total);
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid * PER + q;
    if (j <= cnt) cum[j] = (uint16_t)run;  // cum[cnt] = total
    run += len[q];
  }
  BCF_SYNC();
  for (int q = tid; q < kL1Tile; q += kL1Threads) {
    unsigned long long it = ~0ull;  // padding sorts last
    if (q < (int)total) {
      int lo = 0, hi = cnt - 1;  // last j with cum[j] <= q
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int)cum[mid] <= q) lo = mid;
        else hi = mid - 1;
      }
      const uint32_t key = keys_in[offs[ids[lo]] + (q - (int)cum[lo])];
      it = ((unsigned long long)lo << 44) | ((unsigned long long)key << 12) | (unsigned)q;
    }
    BCF_TR(&X[q], 8, 1, TS_L1_IO);
    X[q] = it;
  }
  BCF_SYNC();
  lemma1_schedule(X, Y);
  const VT* vin = reinterpret_cast<const VT*>(vals_in);
  VT* vout = reinterpret_cast<VT*>(vals_out);
  for (int t = tid; t < (int)total; t += kL1Threads) {
    BCF_TR(&Y[t], 8, 0, TS_L1_IO);
    const unsigned long long it = Y[t];
    const int j = (int)(it >> 44), q = (int)(it & 0xFFFu);
    const int64_t lo = offs[ids[j]];
    const int c = (int)cum[j];
    keys_out[lo + (t - c)] = (uint32_t)(it >> 12);
    if (VB) vout[lo + (t - c)] = vin ? vin[lo + (q - c)] : VT(lo + (q - c));
  }
  BCF_SYNC();
}

// Persistent blocks: sort every small segment whole with the Lemma 1 schedule --
// first the segments that take a tile each, then the bins of tiny segments.
template <int VB>
__global__ void __launch_bounds__(kL1Threads, 3) k_seg_small(const uint32_t* __restrict__ keys_in,
                                                          const void* __restrict__ vals_in,
                                                          uint32_t* __restrict__ keys_out,
                                                          void* __restrict__ vals_out,
                                                          const int64_t* __restrict__ offs,
                                                          const int32_t* __restrict__ small_ids,
                                                          const int32_t* __restrict__ tiny_ids,
                                                          const uint32_t* __restrict__ bin_first,
                                                          uint32_t* ctr) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* X = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* Y = X + kL1Tile;
  uint16_t* cum = reinterpret_cast<uint16_t*>(Y + kL1Tile);  // kL1Tile + 1 entries
  __shared__ int item;
  __shared__ uint32_t scratch[32];
  const int nsmall = (int)ctr[C_NSMALL], nbins = (int)ctr[C_NBINS], ntiny = (int)ctr[C_NTINY];
  while (true) {
    if (threadIdx.x == 0) item = (int)atomicAdd(&ctr[C_QUEUE], 1u);
    BCF_SYNC();
    const int i = item;
    BCF_SYNC();
    if (i >= nsmall + nbins) break;
    if (i < nsmall) {
      const int seg = small_ids[i];
      const int64_t lo = offs[seg];
      lemma1_tile<VB>(keys_in, vals_in, keys_out, vals_out, lo, (int)(offs[seg + 1] - lo), X, Y);
    } else {
      const int b = i - nsmall;
      const int first = (int)~bin_first[b];
      const int last = b + 1 < nbins ? (int)~bin_first[b + 1] : ntiny;
      sort_bin<VB>(keys_in, vals_in, keys_out, vals_out, offs, tiny_ids + first, last - first, X, Y, cum,
                   scratch);
    }
  }
}

// Standalone tile sort: tile t = [t*4096, min(n, (t+1)*4096)).
template <int VB>
__global__ void __launch_bounds__(kL1Threads) k_sort_tiles(const uint32_t* __restrict__ keys_in,
                                                           const void* __restrict__ vals_in,
                                                           uint32_t* __restrict__ keys_out,
                                                           void* __restrict__ vals_out, int64_t n) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* X = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* Y = X + kL1Tile;
  const int64_t start = (int64_t)blockIdx.x * kL1Tile;
  lemma1_tile<VB>(keys_in, vals_in, keys_out, vals_out, start, (int)min((int64_t)kL1Tile, n - start), X, Y);
}

// ------------------------------------------------------------------ host
static int sms() {
  int dev = 0, c = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c;
}

SegLayout seg_layout(int64_t n_total, int64_t nseg, int vb, int passes, bool sort) {
  SegLayout L;
  const int64_t T = kSweepTile;
  L.small_max = sort ? kL1Tile : 0;
  // long segments hold more than small_max keys each
  const int64_t max_large = sort ? std::min<int64_t>(nseg, n_total / (L.small_max + 1) + 1) : nseg;
  L.slots_cap = max_large > 0 ? max_large : 1;
  L.tiles_cap = n_total / T + max_large + 1;
  L.lb_stride = (L.tiles_cap + kLookbackWindow) / kLookbackWindow * kLookbackWindow;  // > tiles
  L.passes = passes;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  L.keys_tmp = take((size_t)n_total * 4);
  L.vals_tmp = take((size_t)n_total * vb);
  L.small_ids = take((size_t)std::max<int64_t>(nseg, 1) * 4);
  L.tiny_ids = take((size_t)std::max<int64_t>(nseg, 1) * 4);
  L.seg_slot = take((size_t)std::max<int64_t>(nseg, 1) * 4);
  L.seg_tile0 = take((size_t)std::max<int64_t>(nseg, 1) * 4);
  L.slot_seg = take((size_t)L.slots_cap * 4);
  L.tile_seg = take((size_t)L.tiles_cap * 4);
  L.seg_base = take((size_t)L.slots_cap * 256 * 4);  // digit starts of the current pass
  L.zero_begin = off;
  L.ctr = take(16 * 4);
  L.bin_first = take((size_t)(n_total / kTinyMax + 2) * 4);  // zeroed: 0 = bin not started
  L.lookback = take((size_t)L.lb_stride * 256 * 4);  // tile counts -> running sums (one pass at a time)
  L.zero_bytes = off - L.zero_begin;
  L.total = off;
  return L;
}

constexpr size_t kSegSmallSmem = kL1SmemBytes + (kL1Tile + 8) * 2;  // items + packed offsets

template <int VB>
static cudaError_t small_sort(const uint32_t* ki, const void* vi, uint32_t* ko, void* vo,
                              const int64_t* offs, const int32_t* ids, const int32_t* tiny_ids,
                              const uint32_t* bin_first, uint32_t* ctr, int64_t nseg, cudaStream_t s) {
  auto k = k_seg_small<VB>;
  static bool ready[64] = {};
  cudaError_t e = set_smem_once(k, (int)kSegSmallSmem, ready);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(nseg, (int64_t)sms() * 3);
  if (grid <= 0) return cudaSuccess;
  k<<<(unsigned)grid, kL1Threads, kSegSmallSmem, s>>>(ki, vi, ko, vo, offs, ids, tiny_ids, bin_first, ctr);
  return cudaGetLastError();
}

static cudaError_t run_segments(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                                void* vals_out, int64_t n_total, const int64_t* offs, int64_t nseg,
                                const int32_t* seg_w, int vb, const PassPlan& plan, bool label,
                                bool balanced, unsigned char* ws, const SegLayout& L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  auto I32 = [&](size_t o) { return reinterpret_cast<int32_t*>(ws + o); };
  auto U32 = [&](size_t o) { return reinterpret_cast<uint32_t*>(ws + o); };
  uint32_t* ctr = U32(L.ctr);
  unsigned* st = status_word();

  PlanParams pp{};
  pp.offs = offs;
  pp.nseg = nseg;
  pp.n_total = n_total;
  pp.small_max = L.small_max;
  pp.tile = kSweepTile;
  pp.tiles_cap = L.tiles_cap;
  pp.slots_cap = L.slots_cap;
  pp.seg_w = seg_w;
  pp.small_ids = I32(L.small_ids);
  pp.tiny_ids = I32(L.tiny_ids);
  pp.bin_first = U32(L.bin_first);
  pp.bins_cap = n_total / kTinyMax + 2;
  pp.seg_slot = I32(L.seg_slot);
  pp.seg_tile0 = I32(L.seg_tile0);
  pp.tile_seg = I32(L.tile_seg);
  pp.slot_seg = I32(L.slot_seg);
  pp.ctr = ctr;
  pp.status = st;
  k_seg_plan<<<1, kPlanThreads, 0, s>>>(pp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  if (L.small_max > 0) {
    switch (vb) {
      case 0:
        e = small_sort<0>(keys_in, vals_in, keys_out, vals_out, offs, I32(L.small_ids), I32(L.tiny_ids),
                          U32(L.bin_first), ctr, nseg, s);
        break;
      case 4:
        e = small_sort<4>(keys_in, vals_in, keys_out, vals_out, offs, I32(L.small_ids), I32(L.tiny_ids),
                          U32(L.bin_first), ctr, nseg, s);
        break;
      case 8:
        e = small_sort<8>(keys_in, vals_in, keys_out, vals_out, offs, I32(L.small_ids), I32(L.tiny_ids),
                          U32(L.bin_first), ctr, nseg, s);
        break;
    }
    if (e != cudaSuccess) return e;
  }

  const int P = plan.passes;
  // Sorts and partitions take the pass form the tuning table names for this
  // batch size: the pass body fed scanned offsets (form 1) or the staged sweep
  // (form 2), both of 4096-key tiles.  The body takes every segment's digit
  // starts from the counts (a balanced partition's closed-form starts are the
  // same; k_seg_digit_base checks the counts); the staged sweep computes a
  // balanced partition's starts and checks itself.
  const bool body_form = cfg_form(tuned_config(kOpSegmentedSort, n_total)) == 1;
  uint32_t* kt = U32(L.keys_tmp);
  void* vt = vb ? (void*)(ws + L.vals_tmp) : nullptr;
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  uint32_t* offsets = U32(L.lookback);  // per-(digit, tile) counts, scanned in place
  for (int q = 0; q < P; ++q) {
    const bool to_out = ((P - 1 - q) % 2) == 0;
    uint32_t* dk = to_out ? keys_out : kt;
    void* dv = to_out ? vals_out : vt;
    // reduce-then-scan: tile counts of this pass, running sums over all tiles
    CountParams cp{};
    cp.keys = src_k;
    cp.n = n_total;
    cp.shift = plan.shift[q];
    cp.nbits = 8;
    cp.label_bits = label ? 8 : 0;
    cp.counts = offsets;
    cp.stride = L.lb_stride;
    cp.totals = nullptr;
    cp.seg_offs = offs;
    cp.tile_seg = I32(L.tile_seg);
    cp.seg_tile0 = I32(L.seg_tile0);
    cp.num_tiles = ctr + C_NTILES;
    cp.seg_w = label && body_form ? seg_w : nullptr;
    cp.status = st;
    const int64_t count_blocks = (L.tiles_cap + kCountTilesPerBlock - 1) / kCountTilesPerBlock;
    k_tile_counts<8, kSweepTile, false, false><<<(unsigned)count_blocks, 256, 0, s>>>(cp, L.tiles_cap);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launch_scan_offsets(256, offsets, L.tiles_cap, L.lb_stride, nullptr, 0, n_total, 1, st, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!balanced || body_form) {
      k_seg_digit_base<<<(unsigned)L.slots_cap, 256, 0, s>>>(offsets, L.lb_stride, U32(L.seg_base), I32(L.slot_seg),
                                                             I32(L.seg_tile0), offs, ctr, kSweepTile,
                                                             balanced ? seg_w : nullptr, st);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (body_form) {
      static_assert(kSweepTile == 256 * 16, "the batched sort's tiles are the 256 x 16 body's");
      OneSweepParams op{};
      op.keys_in = src_k;
      op.vals_in = src_v;
      op.keys_out = dk;
      op.vals_out = dv;
      op.n = n_total;
      op.shift = plan.shift[q];
      op.w = label ? 256 : 0;  // the tile counts check each segment's labels against seg_w
      op.tile_offsets = offsets;
      op.offs_stride = L.lb_stride;
      op.err = st;
      op.seg_offs = offs;
      op.tile_seg = I32(L.tile_seg);
      op.seg_tile0 = I32(L.seg_tile0);
      op.seg_slot = I32(L.seg_slot);
      op.seg_base = U32(L.seg_base);
      op.num_tiles = ctr + C_NTILES;
      if ((e = onesweep_dispatch<8, 256, 16, kOneCfgMinBlocks[kNumOneConfigs]>(op, L.tiles_cap, vb, s)) !=
          cudaSuccess)
        return e;
      src_k = dk;
      src_v = dv;
      continue;
    }
    SweepParams sp{};
    sp.tile_offsets = offsets;
    sp.keys_in = src_k;
    sp.vals_in = src_v;
    sp.keys_out = dk;
    sp.vals_out = dv;
    sp.n = n_total;
    sp.shift = plan.shift[q];
    sp.nbits = plan.nbits[q];
    sp.w = label ? 256 : 0;  // per-segment widths come from seg_w
    sp.balanced = balanced ? 1 : 0;
    sp.lookback = nullptr;
    sp.lb_stride = L.lb_stride;
    sp.ticket = ctr + C_TICKET + q;
    sp.status = st;
    sp.seg_offs = offs;
    sp.tile_seg = I32(L.tile_seg);
    sp.seg_tile0 = I32(L.seg_tile0);
    sp.seg_slot = I32(L.seg_slot);
    sp.seg_base = U32(L.seg_base);
    sp.seg_w = seg_w;
    sp.num_tiles = ctr + C_NTILES;
    if ((e = sweep_dispatch<8>(sp, L.tiles_cap, vb, s)) != cudaSuccess) return e;
    src_k = dk;
    src_v = dv;
  }
  return cudaSuccess;
}

cudaError_t segmented_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                           void* vals_out, int64_t n_total, const int64_t* offs, int64_t nseg,
                           int vb, const PassPlan& plan, unsigned char* ws, const SegLayout& L,
                           cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  return run_segments(keys_in, vals_in, keys_out, vals_out, n_total, offs, nseg, nullptr, vb, plan,
                      false, false, ws, L, s);
}

cudaError_t segmented_partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                                void* vals_out, int64_t n_total, const int64_t* offs,
                                const int32_t* w_per_seg, int64_t nseg, int vb, bool balanced,
                                unsigned char* ws, const SegLayout& L, cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  PassPlan one;
  one.passes = 1;
  one.shift[0] = 0;
  one.nbits[0] = 8;
  return run_segments(keys_in, vals_in, keys_out, vals_out, n_total, offs, nseg, w_per_seg, vb, one,
                      true, balanced, ws, L, s);
}

cudaError_t sort_tiles(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n, int vb, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t tiles = (n + kL1Tile - 1) / kL1Tile;
  cudaError_t e = cudaSuccess;
  switch (vb) {
#define BCF_TS(VB)                                                                                 \
  case VB: {                                                                                       \
    static bool ready[64] = {};                                                                    \
    e = set_smem_once(k_sort_tiles<VB>, (int)kL1SmemBytes, ready);                                 \
    if (e != cudaSuccess) return e;                                                                \
    k_sort_tiles<VB><<<(unsigned)tiles, kL1Threads, kL1SmemBytes, s>>>(keys_in, vals_in, keys_out, \
                                                                       vals_out, n);               \
    break;                                                                                         \
  }
    BCF_TS(0)
    BCF_TS(4)
    BCF_TS(8)
#undef BCF_TS
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

BCF_TRACE_INSTALLER(segmented)

}  // namespace bcf
