// onesweep.cuh -- single-launch digit passes (decoupled look-back) for the flat
// radix sort and the w-way partition, and the one-read histogram that precedes a
// sort.
//
// A pass is the paper's partition problem (Sec. 1) at GPU scale: every key moves to
// the block of its digit (or label), stably.  One block of threads handles one tile
// of keys in one launch:
//   1. keys (and payloads) are read warp-striped -- lane l of warp q holds tile
//      items q*32*IPT + 32j + l -- which is the conflict-free strided pattern of
//      Sec. 1 moved into registers: every warp-wide load is one 128-byte line;
//   2. each warp ranks its keys: the peers of a key (lanes of the same warp step
//      with the same digit) come from one ballot per digit bit; the lowest peer
//      claims the digit's next run slots in the warp's count row with one shared
//      atomic, and rank = claimed start + popc(peers below the lane) -- the row
//      "radix sort" of Corollary 1 done per warp step, stable by construction;
//   3. the tile's digit counts are published at once (decoupled look-back
//      status, tile-major: the 256 counts of one tile are one 1 KB row, so a warp
//      reads 32 digits of a predecessor with one coalesced load);
//   4. keys are scattered in shared memory into digit order, then one thread per
//      digit sums predecessors' published counts (several predecessors per round
//      trip) until it meets an inclusive prefix, and publishes its own;
//   5. the ordered tile is written out: consecutive threads take consecutive
//      positions, so every digit's run is a contiguous stretch of global memory.
// No per-pass count kernel re-reads the keys and no scan kernel runs between
// passes: a pass moves 16 bytes per key-value pair (read 8, write 8).
//
// The histogram kernel counts all digits of all passes in one read of the keys.
// Its counters are private to a lane: counter (pass, digit) of lane l sits at word
// ((pass * 256 + digit) * 32 + l), in bank l, so the 32 lanes of a counting
// instruction always touch 32 different banks -- the conflict avoidance condition
// of Sec. 1 met by construction, whatever the digits are.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"
#include "trace.cuh"

namespace bcf {

// ------------------------------------------------------------- histogram
struct OneHistParams {
  const uint32_t* keys;
  int64_t n;
  int passes;            // 1..4 digit passes of 8 bits
  int shift[4];
  uint32_t* hist;        // passes x 256 totals, zero on entry
  uint32_t* digit_base;  // passes x 256 exclusive starts, written by the last block
  uint32_t* done;        // zero on entry
  uint32_t* vary;        // nullptr, or [2] zero on entry: OR of the keys, OR of their complements
  uint32_t* zero;        // status region cleared for the first pass (16-byte aligned)
  int64_t zero_words;    // multiple of 4
};

constexpr int kHistThreads = 1024;
constexpr int kHistUnroll = 4;  // 16-byte loads in flight per thread

inline size_t onesweep_hist_smem(int passes) { return (size_t)passes * 256 * 32 * 4; }

// BYTES: the digits are the key's bytes 0..passes-1 (shifts 0, 8, 16, 24), taken
// with one byte permute each; otherwise shifts come from p.shift.
template <bool BYTES>
__global__ void __launch_bounds__(kHistThreads, 1) k_onesweep_hist(OneHistParams p) {
  extern __shared__ uint32_t hsm[];  // passes x 256 x 32 lane-private counters
  __shared__ uint32_t scratch[32];
  __shared__ int is_last;
  const int tid = threadIdx.x, lane = tid & 31;
  const int words = p.passes * 256 * 32;
  for (int i = tid; i < words; i += kHistThreads) hsm[i] = 0;
  if (p.zero) {
    uint4* z = reinterpret_cast<uint4*>(p.zero);
    const int64_t nz = p.zero_words / 4;
    for (int64_t i = (int64_t)blockIdx.x * kHistThreads + tid; i < nz; i += (int64_t)gridDim.x * kHistThreads)
      z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  BCF_SYNC();
  uint32_t* hl = hsm + lane;
  uint32_t o1 = 0, o0 = 0;
  auto count = [&](uint32_t k) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < p.passes) {
        const uint32_t d = BYTES ? __byte_perm(k, 0u, 0x4440u + q) : (k >> p.shift[q]) & 0xFFu;
        uint32_t* c = hl + ((q * 256 + d) << 5);
        BCF_TR(c, 4, 2, TS_HIST_ATOM);
        atomicAdd(c, 1u);
      }
  };
  auto count4 = [&](const uint4& x) {  // the OR words per 16 bytes, then four keys
    o1 |= x.x | x.y | x.z | x.w;
    o0 |= ~(x.x & x.y & x.z & x.w);
    count(x.x);
    count(x.y);
    count(x.z);
    count(x.w);
  };
  const int64_t nvec = p.n >> 2;
  const uint4* kv = reinterpret_cast<const uint4*>(p.keys);
  const int64_t stride = (int64_t)gridDim.x * kHistThreads;
  int64_t i = (int64_t)blockIdx.x * kHistThreads + tid;
  for (; i + (kHistUnroll - 1) * stride < nvec; i += kHistUnroll * stride) {
    uint4 x[kHistUnroll];
#pragma unroll
    for (int u = 0; u < kHistUnroll; ++u) x[u] = __ldcs(kv + i + u * stride);
#pragma unroll
    for (int u = 0; u < kHistUnroll; ++u) count4(x[u]);
  }
  for (; i < nvec; i += stride) count4(__ldcs(kv + i));
  for (int64_t e = nvec * 4 + (int64_t)blockIdx.x * kHistThreads + tid; e < p.n; e += stride) {
    const uint32_t k = p.keys[e];
    o1 |= k;
    o0 |= ~k;
    count(k);
  }
  if (p.vary) or_into_vary(o1, o0, p.vary, scratch);
  BCF_SYNC();
  // Sum the 32 lane counters of each (pass, digit): thread e reads lane (i + e) mod
  // 32 in step i, so the 32 threads of a warp read 32 different banks.
  for (int e = tid; e < p.passes * 256; e += kHistThreads) {
    uint32_t s = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const uint32_t* c = hsm + e * 32 + ((k + e) & 31);
      BCF_TR(c, 4, 0, TS_HIST_SUM);
      s += *c;
    }
    if (s) atomicAdd(&p.hist[e], s);
  }
  __threadfence();
  BCF_SYNC();
  if (tid == 0) is_last = (atomicAdd(p.done, 1u) == gridDim.x - 1);
  BCF_SYNC();
  if (!is_last) return;
  __threadfence();
  for (int q = 0; q < p.passes; ++q) {
    const uint32_t c = tid < 256 ? ld_relaxed(&p.hist[q * 256 + tid]) : 0u;
    uint32_t total;
    const uint32_t e = block_excl_scan<kHistThreads>(c, scratch, &total);
    if (tid < 256) p.digit_base[q * 256 + tid] = e;
  }
}

// ------------------------------------------------------------- one pass
struct OneSweepParams {
  const uint32_t* keys_in;
  const void* vals_in;         // nullptr with 4-byte payloads: payload = input position
  uint32_t* keys_out;
  void* vals_out;
  int64_t n;
  int shift;                   // digit = (key >> shift) & (RADIX - 1)
  int w;                       // > 0: partition, digit = label, labels must be < w
  int balanced;                // partition: label b starts at b * (n / w)
  const uint32_t* digit_base;  // RADIX exclusive global starts (unused when balanced)
  uint32_t* status;            // tiles x RADIX look-back words (tile-major), zero on entry
  // offsets mode (tile_offsets != nullptr): the absolute start of every (digit,
  // tile) run, digit-major with stride offs_stride, scanned ahead of the launch;
  // no ticket, no status words, no look-back
  const uint32_t* tile_offsets;
  int64_t offs_stride;
  uint32_t* zero_next;         // tiles x RADIX words cleared for the next pass, or nullptr
  uint32_t* ticket;            // tile counter, zero on entry
  unsigned* err;
  unsigned spin_limit;         // polls before a wait gives up (0: kSpinLimit)
  int silent_tile1;            // testing aid: 1 + a tile that never publishes (0: none)
  PassSel sel;                 // sel.vary != nullptr: buffers (or a skip) decided on the device
  // direct (partitions by at most 32 labels): every key goes from its registers
  // straight to its global place; no digit-order staging in shared memory, so
  // every shared access of the pass is conflict-free (label = bank)
  int direct;
  // segment mode (seg_offs != nullptr; offsets mode): tile t is
  // piece t - seg_tile0[s] of segment s = tile_seg[t] (tiles past *num_tiles do
  // nothing), tile_offsets holds running sums over all tiles, and a tile's run
  // start is its running sum minus the one at its segment's first tile plus the
  // segment's digit start seg_base[seg_slot[s] * RADIX + digit].
  const int64_t* seg_offs;
  const int32_t* tile_seg;
  const int32_t* seg_tile0;
  const int32_t* seg_slot;
  const uint32_t* seg_base;
  const uint32_t* num_tiles;
};

// Look-back predecessors read per round trip (one coalesced row load each).
#ifndef BCF_OS_LBW
#define BCF_OS_LBW 8
#endif
constexpr int kOneLookback = BCF_OS_LBW;

template <int BITS, int THREADS, int IPT, int VB>
struct OneSmem {
  static constexpr int T = THREADS * IPT;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int RADIX = 1 << BITS;
  // The tile in digit order: with 4-byte payloads (payload << 32 | key) pairs,
  // then the staging area the payloads' bulk copy fills; otherwise keys, then
  // payloads.
  static constexpr size_t keys = 0;
  static constexpr size_t vals = (size_t)T * 4;                     // 8-byte payloads
  static constexpr size_t stage = (size_t)T * 8;                    // 4-byte payloads (+ 3 words of
                                                                    // a segment's misalignment)
  static constexpr size_t whist = (size_t)T * (4 + VB) + (VB == 4 ? (size_t)T * 4 + 16 : 0);
  static constexpr size_t gofs = whist + (size_t)WARPS * RADIX * 4;
  static constexpr size_t scratch = gofs + (size_t)RADIX * 4;  // scan scratch
  static constexpr size_t mbar = scratch + 32 * 4;
  static constexpr size_t info = mbar + 16;   // ints: tile, route, segment, piece, slot; then lo, hi
  static constexpr size_t bytes = info + 48;
  static_assert(mbar % 8 == 0, "mbarrier alignment");
};

template <int BITS, int THREADS, int IPT, int VB, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_onesweep(OneSweepParams p) {
  using VT = typename ValT<VB>::type;
  using S = OneSmem<BITS, THREADS, IPT, VB>;
  constexpr int T = S::T, RADIX = S::RADIX, WARPS = S::WARPS;
  constexpr uint32_t DMASK = RADIX - 1;
  constexpr int LO = BITS < 5 ? BITS : 5;  // digit bits resolved by the first peer table
  static_assert(RADIX <= THREADS && THREADS >= 64, "one thread per digit");
  static_assert(BITS <= 10, "two peer tables of at most 5 bits");
  static_assert(IPT % 2 == 0, "ranks are kept two to a register");
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* kv_s = reinterpret_cast<unsigned long long*>(smem + S::keys);
  uint32_t* keys_s = reinterpret_cast<uint32_t*>(smem + S::keys);
  VT* vals_s = reinterpret_cast<VT*>(smem + S::vals);
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem + S::stage);
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + S::whist);
  uint32_t* gofs = reinterpret_cast<uint32_t*>(smem + S::gofs);
  uint32_t* scratch = reinterpret_cast<uint32_t*>(smem + S::scratch);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::mbar);
  int* s_info = reinterpret_cast<int*>(smem + S::info);
  int64_t* s_bounds = reinterpret_cast<int64_t*>(smem + S::info + 32);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool segmented = p.seg_offs != nullptr;

  // The next pass's status row of this block is cleared whatever this pass does:
  // the previous pass (the row's last user) has finished, and the next one needs
  // it zero even when this pass is skipped.
  if (p.zero_next)
    for (int d = tid; d < RADIX; d += THREADS) p.zero_next[(size_t)blockIdx.x * RADIX + d] = 0u;

  // Two global round trips overlap: thread 0 takes the tile ticket while thread 32
  // decides the pass's route (which buffers it reads and writes, or a skip).
  // Tiles are taken in launch order (atomic ticket), so every tile a look-back
  // waits on belongs to a block that is already running.
  if (tid == 0) {
    mbar_init(mbar, 1);
    s_info[0] = p.tile_offsets ? (int)blockIdx.x : (int)atomicAdd(p.ticket, 1u);
  }
  if (tid == 32) {
    const int route = p.sel.vary ? pass_route(p.sel, vary_bits(p.sel)) : 3 * 0 + 1;
    if (route >= 0 && p.sel.vary && blockIdx.x == 0) atomicOr(p.sel.ran, 1u << p.sel.q);
    s_info[1] = route;
  }
  if (segmented && tid == 64) {  // the tile's segment, piece and bounds (two round trips)
    const int tile = (int)blockIdx.x;
    const int seg = (uint32_t)tile < ld_relaxed(p.num_tiles) ? p.tile_seg[tile] : -1;
    s_info[2] = seg;
    if (seg >= 0) {
      s_info[3] = tile - p.seg_tile0[seg];
      s_info[4] = p.seg_slot[seg];
      s_bounds[0] = p.seg_offs[seg];
      s_bounds[1] = p.seg_offs[seg + 1];
    }
  }
  // In offsets mode the flat tile is the block's own and its run starts were
  // scanned before the launch: fetch them now, so that the round trip overlaps the
  // key loads and the ranking instead of holding the block after its scatter.
  uint32_t pre_base = 0;
  if (p.tile_offsets && !segmented && tid < RADIX)
    pre_base = __ldcg(p.tile_offsets + (size_t)tid * p.offs_stride + blockIdx.x);
  static_assert(S::whist % 16 == 0, "count rows are cleared 16 bytes at a time");
  for (int i = tid; i < WARPS * RADIX / 4; i += THREADS)
    reinterpret_cast<uint4*>(whist)[i] = make_uint4(0u, 0u, 0u, 0u);
  // 1. warp-striped key loads, every warp-wide load one contiguous 128-byte line.
  // They are issued for tile blockIdx.x from the launch's input before the ticket
  // and the route are known: blocks start in index order and passes are rarely
  // skipped, so this is almost always the tile the ticket names, and the load
  // latency overlaps the two round trips; otherwise the keys are read again.
  const int wbase = warp * 32 * IPT;
  uint32_t key[IPT];
  auto load_keys = [&](const uint32_t* src, int64_t st, int c) {
    const uint32_t* kin = src + st + wbase + lane;
    if (c == T) {  // full tile: no per-key test
#pragma unroll
      for (int j = 0; j < IPT; ++j) key[j] = __ldcs(kin + 32 * j);
    } else {
#pragma unroll
      for (int j = 0; j < IPT; ++j) key[j] = wbase + j * 32 + lane < c ? __ldcs(kin + 32 * j) : 0xFFFFFFFFu;
    }
  };
  if (!segmented) {
    const int64_t st = (int64_t)blockIdx.x * T;
    load_keys(p.keys_in, st, (int)min((int64_t)T, p.n - st));
  }
  BCF_SYNC();
  const int route = s_info[1];
  if (route < 0) return;  // skipped pass: nothing to move
  if (segmented && s_info[2] < 0) return;  // more blocks than tiles this time
  const uint32_t* keys_in = p.keys_in;
  const void* vals_in = p.vals_in;
  uint32_t* keys_out = p.keys_out;
  void* vals_out = p.vals_out;
  if (p.sel.vary) route_buffers(p.sel, route, keys_in, vals_in, keys_out, vals_out);
  const int tile = s_info[0];
  const int64_t start = segmented ? s_bounds[0] + (int64_t)s_info[3] * T : (int64_t)tile * T;
  const int cnt = (int)min((int64_t)T, (segmented ? s_bounds[1] : p.n) - start);
  const bool label_mode = p.w > 0;
  const bool iota = VB == 4 && vals_in == nullptr;
  const int shift = label_mode ? 0 : p.shift;
  // An 8-bit digit is a whole key byte (the host plans passes at shifts 8q and
  // refuses others), taken with one byte permute.
  const uint32_t psel = 0x4440u + ((uint32_t)shift >> 3);
  auto digit = [&](uint32_t k) -> uint32_t {
    if constexpr (BITS == 8) return __byte_perm(k, 0u, psel);
    else return (k >> shift) & DMASK;
  };
  uint32_t* wh = whist + warp * RADIX;
  if (segmented || tile != (int)blockIdx.x || keys_in != p.keys_in) load_keys(keys_in, start, cnt);
  // 4-byte payloads arrive by one bulk copy into the staging area while the keys
  // are ranked.  The copy starts at the 16-byte boundary at or below the tile's
  // first payload, vsh words early (0 but for a segment's pieces), so item i of
  // the tile is stage[vsh + i]; the ragged end past the copy is read directly.
  const uint32_t* vin4 = reinterpret_cast<const uint32_t*>(vals_in);
  const int vsh = (VB == 4 && !iota) ? (int)((reinterpret_cast<uintptr_t>(vin4 + start) & 15u) >> 2) : 0;
  const int vcopy = (VB == 4 && !iota) ? ((vsh + cnt) & ~3) : 0;  // words copied
  const int vcov = vcopy > 0 ? vcopy - vsh : 0;                    // tile items they cover
  if (VB == 4 && !iota && tid == 0) {
    mbar_arrive_expect_tx(mbar, (unsigned)vcopy * 4u);
    if (vcopy) bulk_g2s(stage, vin4 + start - vsh, (unsigned)vcopy * 4u, mbar);
  }
  // Lane l holds entry l of the peer table of the low digit bits, and (its low
  // bits reused) entry l mod 2^(BITS - LO) of the table of the high bits.
  uint32_t rep[LO];
#pragma unroll
  for (int k = 0; k < LO; ++k) rep[k] = ((lane >> k) & 1) ? 0xffffffffu : 0u;

  // The last tile, if ragged, runs the same code: its missing keys read as
  // 0xFFFFFFFF, whose digit is the largest, so they rank after every real key of
  // that digit -- at the tile's last T - cnt positions, which are never written
  // out -- and that digit's published count leaves them out.
  const bool full = cnt == T;
  {
    auto valid_at = [&](int j) { return full || wbase + j * 32 + lane < cnt; };
    if (label_mode) {
      bool bad = false;
#pragma unroll
      for (int j = 0; j < IPT; ++j) bad |= valid_at(j) && key[j] >= (uint32_t)p.w;
      if (bad) set_status(p.err, DEV_BAD_KEY);
    }

    // 2. per-warp ranking.  One ballot per digit bit; each lane turns them into
    // its entries of two tables -- the lanes whose low digit bits equal the lane
    // index, and those whose high bits equal it -- and a key's peers (same
    // digit, same warp step) are the AND of the two entries fetched from the
    // lanes its digit names.  The highest peer claims the run for all of them.
    const unsigned lt = lanemask_lt();
    uint32_t rk[IPT / 2];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t d = digit(key[j]);
      unsigned bal[BITS];
#pragma unroll
      for (int b = 0; b < BITS; ++b) bal[b] = __ballot_sync(0xffffffffu, (d >> b) & 1u);
      unsigned tlo = ~(bal[0] ^ rep[0]);
#pragma unroll
      for (int k = 1; k < LO; ++k) tlo &= ~(bal[k] ^ rep[k]);
      unsigned peers = __shfl_sync(0xffffffffu, tlo, (int)(d & 31u));
      if constexpr (BITS > 5) {
        unsigned thi = ~(bal[5] ^ rep[0]);
#pragma unroll
        for (int k = 1; k < BITS - 5; ++k) thi &= ~(bal[5 + k] ^ rep[k]);
        peers &= __shfl_sync(0xffffffffu, thi, (int)(d >> 5));
      }
      const int leader = 31 - __clz(peers);
      uint32_t old = 0;
      if (lane == leader) {
        BCF_TR(&wh[d], 4, 2, TS_CLAIM_ATOM);
        old = atomicAdd(&wh[d], (uint32_t)__popc(peers));
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      const uint32_t r = old + (uint32_t)__popc(peers & lt);
      if (j & 1) rk[j >> 1] |= r << 16;
      else rk[j >> 1] = r;
    }
    // A ragged tile's payloads past the bulk copy are read into the staging area
    // directly, so that the scatter below reads every payload from there.
    if (VB == 4 && !iota && vcov < cnt)
      for (int i = vcov + tid; i < cnt; i += THREADS) stage[vsh + i] = vin4[start + i];
    BCF_SYNC();

    // 3. per digit: tile count (published at once), tile-exclusive start, and each
    // warp's start inside the tile.
    uint32_t count = 0;
    uint32_t wc[WARPS];  // this digit's warp counts, reused for the warps' starts below
    if (tid < RADIX) {
#pragma unroll
      for (int q = 0; q < WARPS; ++q) {
        BCF_TR(&whist[q * RADIX + tid], 4, 0, TS_WARP_OFFSETS);
        wc[q] = whist[q * RADIX + tid];
        count += wc[q];
      }
      if (tid == RADIX - 1) count -= (uint32_t)(T - cnt);  // the ragged tile's padding
      if (!p.tile_offsets && tile + 1 != p.silent_tile1)
        st_relaxed(p.status + (size_t)tile * RADIX + tid, (tile == 0 ? LB_INC : LB_AGG) | count);
    }
    // Decoupled look-back, one thread per digit, at once: the sooner a tile
    // publishes its inclusive prefix, the shorter its successors' look-backs.
    // Predecessors' counts are added (kOneLookback rows per round trip) until one
    // has published its inclusive prefix; a row not yet published is polled again.
    uint32_t excl = 0;
    if (tid < RADIX && tile > 0 && !p.tile_offsets) {
      int j = tile - 1;  // nearest predecessor not yet added
      unsigned spins = 0;
      const unsigned limit = p.spin_limit ? p.spin_limit : kSpinLimit;
      while (true) {
        uint32_t lbv[kOneLookback];
#pragma unroll
        for (int k = 0; k < kOneLookback; ++k)
          lbv[k] = j - k >= 0 ? ld_relaxed(p.status + (size_t)(j - k) * RADIX + tid) : LB_INC;
        int used = 0;
        bool done = false;
#pragma unroll
        for (int k = 0; k < kOneLookback; ++k) {
          if (done || used < k) continue;  // stopped at an unpublished row
          const uint32_t f = lbv[k] & ~LB_MASK;
          if (f == 0) continue;
          excl += lbv[k] & LB_MASK;
          used = k + 1;
          done = f == LB_INC;
        }
        if (done) break;
        j -= used;
        if (used < kOneLookback && ++spins > limit) {
          set_status(p.err, DEV_TIMEOUT);
          break;
        }
      }
      if (tile + 1 != p.silent_tile1) st_relaxed(p.status + (size_t)tile * RADIX + tid, LB_INC | (excl + count));
    }
    uint32_t total;
    const uint32_t tile_excl = block_excl_scan<THREADS>(tid < RADIX ? count : 0u, scratch, &total);
    if (tid < RADIX) {
      uint32_t run = tile_excl;
#pragma unroll
      for (int q = 0; q < WARPS; ++q) {
        BCF_TR(&whist[q * RADIX + tid], 4, 1, TS_WARP_OFFSETS);
        whist[q * RADIX + tid] = run;
        run += wc[q];
      }
    }
    BCF_SYNC();

    // 4a. keys (with 4-byte payloads: pairs) into digit order in shared memory;
    // the payload comes from the staging area (padding slots carry stale words,
    // which are never written out) or is the input position
    if (VB == 4 && !iota) mbar_wait(mbar, 0, p.err);
    auto scatter = [&](auto iota_tag) {
      constexpr bool IOTA = decltype(iota_tag)::value;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t half = (rk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
        const uint32_t d = digit(key[j]);
        BCF_TR(&wh[d], 4, 0, TS_OFFSET_READ);
        const uint32_t pos = wh[d] + half;  // < T, padding included
        if constexpr (VB == 4) {
          const int idx = wbase + j * 32 + lane;
          uint32_t v;
          if constexpr (IOTA) {
            v = (uint32_t)(start + idx);
          } else {
            BCF_TR(&stage[vsh + idx], 4, 0, TS_STAGE_READ);
            v = stage[vsh + idx];
          }
          BCF_TR(&kv_s[pos], 8, 1, TS_SCATTER);
          kv_s[pos] = ((unsigned long long)v << 32) | key[j];
        } else {
          BCF_TR(&keys_s[pos], 4, 1, TS_SCATTER);
          keys_s[pos] = key[j];
        }
        if constexpr (VB == 8) {  // the ranks become positions for the payload stores
          if (j & 1) rk[j >> 1] = (rk[j >> 1] & 0xFFFFu) | (pos << 16);
          else rk[j >> 1] = (rk[j >> 1] & 0xFFFF0000u) | pos;
        }
      }
    };
    if (!p.direct) {
      if (VB == 4 && iota) scatter(std::true_type{});
      else scatter(std::false_type{});
    }
    // 4b. 8-byte payloads: loaded now (the keys' registers are free), in flight
    // during the look-back, then stored at their keys' positions
    VT val[VB == 8 ? IPT : 1];
    asm volatile("" ::: "memory");
    if constexpr (VB == 8) {
      const VT* vin = reinterpret_cast<const VT*>(vals_in) + start + wbase + lane;
#pragma unroll
      for (int j = 0; j < IPT; ++j) val[j] = valid_at(j) ? __ldcs(vin + 32 * j) : VT(0);
    }

    // 4c. global offsets of the tile's digit runs
    if (tid < RADIX) {
      uint32_t base;
      if (p.tile_offsets) {  // balanced counts were checked by the scan
        const uint32_t* row = p.tile_offsets + (size_t)tid * p.offs_stride;
        base = pre_base;
        if (segmented)  // running sums over all tiles: rebase at the segment's first tile
          base = p.seg_base[(size_t)s_info[4] * RADIX + tid] + (row[tile] - row[tile - s_info[3]]);
      } else if (label_mode && p.balanced) {
        const int64_t per = p.n / p.w;
        base = (uint32_t)min((int64_t)tid * per, p.n);
        if (start + cnt >= p.n && excl + count != (tid < p.w ? (uint32_t)per : 0u))
          set_status(p.err, DEV_NOT_BALANCED);
      } else {
        base = p.digit_base[tid];
      }
      gofs[tid] = base + excl - tile_excl;
    }
    if (VB == 8 && !p.direct) {
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const uint32_t pos = (rk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
        BCF_TR(&vals_s[pos], VB, 1, TS_SCATTER);
        vals_s[pos] = val[j];
      }
    }
    BCF_SYNC();
    if (p.direct) {
      // global place = the run start of the key's label in this tile, plus its
      // warp's start inside the run, plus its rank among the warp's peers
      VT* vo = reinterpret_cast<VT*>(vals_out);
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (!valid_at(j)) continue;
        const uint32_t half = (rk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
        const uint32_t d = digit(key[j]);
        BCF_TR(&wh[d], 4, 0, TS_OFFSET_READ);
        BCF_TR(&gofs[d], 4, 0, TS_OFFSET_READ);
        const uint32_t dst = gofs[d] + wh[d] + half;
        if (dst >= (uint32_t)p.n) continue;
        keys_out[dst] = key[j];
        if constexpr (VB == 4) {
          const int idx = wbase + j * 32 + lane;
          uint32_t v;
          if (iota) {
            v = (uint32_t)(start + idx);
          } else {
            BCF_TR(&stage[vsh + idx], 4, 0, TS_STAGE_READ);
            v = stage[vsh + idx];
          }
          vo[dst] = v;
        } else if constexpr (VB == 8) {
          vo[dst] = val[j];
        }
      }
      return;
    }
  }

  // 5. write-out: consecutive threads take consecutive ordered positions, so the
  // stores of one digit's run are contiguous; positions outside [0, n) (possible
  // only after a wait gave up or with bad labels) are never written.
  VT* vout = reinterpret_cast<VT*>(vals_out);
  const uint32_t n32 = (uint32_t)p.n;
  auto emit = [&](int i) {
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
      if constexpr (VB == 8) {
        BCF_TR(&vals_s[i], VB, 0, TS_WRITEOUT_READ);
        v = vals_s[i];
      }
    }
    const uint32_t d = digit(k);
    BCF_TR(&gofs[d], 4, 0, TS_OFFSET_READ);
    const uint32_t dst = gofs[d] + (uint32_t)i;
    if (dst < n32) {
      keys_out[dst] = k;
      if constexpr (VB != 0) vout[dst] = v;
    }
  };
  if (full) {
#pragma unroll 4
    for (int q = 0; q < IPT; ++q) emit(q * THREADS + tid);
  } else {
    for (int i = tid; i < cnt; i += THREADS) emit(i);
  }
}

template <int BITS, int THREADS, int IPT, int VB, int MINB>
inline cudaError_t launch_onesweep(const OneSweepParams& p, int64_t grid, cudaStream_t s) {
  using S = OneSmem<BITS, THREADS, IPT, VB>;
  auto kern = k_onesweep<BITS, THREADS, IPT, VB, MINB>;
  if (BITS == 8 && p.w == 0 && (p.shift & 7)) return cudaErrorInvalidValue;  // digits are whole bytes
  // raised on every launch that needs it (see launch_sweep: no flag shared
  // between translation units)
  if (S::bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
  }
  if (grid <= 0) return cudaSuccess;
  kern<<<(unsigned)grid, THREADS, S::bytes, s>>>(p);
  return cudaGetLastError();
}

template <int BITS, int THREADS, int IPT, int MINB>
inline cudaError_t onesweep_dispatch(const OneSweepParams& p, int64_t grid, int vb, cudaStream_t s) {
  switch (vb) {
    case 0: return launch_onesweep<BITS, THREADS, IPT, 0, MINB>(p, grid, s);
    case 4: return launch_onesweep<BITS, THREADS, IPT, 4, MINB>(p, grid, s);
    case 8: return launch_onesweep<BITS, THREADS, IPT, 8, MINB>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bcf
