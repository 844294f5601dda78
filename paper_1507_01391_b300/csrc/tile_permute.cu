// tile_permute.cu -- permutation inside shared-memory tiles (Sec. 3).
//
// A tile of T keys is the paper's w x m matrix with w = 32 rows (banks) and
// m = T/32 columns: the key at tile position q sits in bank q mod 32, slot q/32,
// and its label p = lpi[q] names bank p mod 32 ("row i") and slot p/32 ("j").
//
// Two schedules, same result:
//  * scatter  -- every thread writes out_s[p] = in_s[q] (k_tile_scatter_stream,
//                persistent blocks over many tiles); a warp's 32 stores land
//                in arbitrary banks, so they conflict (about 3.5 wavefronts each
//                for a random permutation).
//  * coloured -- the randomized algorithm of Sec. 3.  A random hash h: [32] -> [m]
//                colours label (i, j) with k = (j - h(i)) mod m.  Within one
//                colour class every destination bank appears exactly once, so a
//                warp request that sends only colour-k items never conflicts
//                (the CAC argument of the Communication step).  Each row sends
//                at most one item of each colour per round; items whose colour
//                was already taken are retried next round with a fresh h (the
//                Synchronization loop).  The few left after the last round are
//                either sent greedily, one item per destination bank per request,
//                or (sorted finish) packed into a matrix sorted by destination and
//                sent in the three groups of the paper's finishing step: labels
//                whose destination bank is private to their row go first in any
//                order, then a row's first and last destination banks, the label
//                of slot j in step j.
#include "common.cuh"
#include "internal.h"
#include "trace.cuh"

namespace bcf {

#ifndef BCF_TP_THREADS
#define BCF_TP_THREADS 512
#endif
constexpr int kTPThreads = BCF_TP_THREADS;  // warps per tile: each lane owns M / warps slots of its row
#ifndef BCF_TP_ROUNDS
#define BCF_TP_ROUNDS 3
#endif
constexpr int kTPRounds = BCF_TP_ROUNDS;     // colouring rounds before the finish

__device__ __forceinline__ uint32_t mix32(uint64_t x) {
  // splitmix64 finaliser (Steele, Lea & Flood 2014), folded to 32 bits
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (uint32_t)x;
}

template <int T>
struct TPSmem {
  static constexpr int M = T / 32;
  static constexpr size_t in = 0;
  static constexpr size_t lpi = in + (size_t)T * 4;
  static constexpr size_t out = lpi + (size_t)T * 2;
  static constexpr size_t mbar = out + (size_t)T * 4;
  static constexpr size_t bytes = mbar + 8;             // direct scatter
  static constexpr size_t tbl = mbar + 16;
  static constexpr size_t lab = tbl + (size_t)T * 4;    // labels widened to one word each
  static constexpr size_t bytes_coloured = lab + (size_t)T * 4;
  // sorted finish: bitmap of the (bank, slot) label space and scan scratch; the
  // source positions reuse lpi, the packed labels lab and the packed keys tbl
  static constexpr size_t bits = bytes_coloured;
  static constexpr size_t scr = bits + (size_t)(T / 32) * 4;           // one word per warp
  static constexpr size_t bytes_sorted = scr + (size_t)(kTPThreads / 32) * 4;
};

// Stage the tile's keys and local labels into shared memory.  Returns len.
template <int T>
__device__ __forceinline__ int stage_tile(const uint32_t* src, const uint16_t* lpi,
                                          int64_t n, int64_t tile, uint32_t* in_s,
                                          uint16_t* lpi_s, uint64_t* mbar, unsigned* status) {
  const int64_t start = tile * T;
  const int len = (int)min((int64_t)T, n - start);
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    const unsigned bk = (unsigned)(len * 4) & ~15u;
    const unsigned bl = (unsigned)(len * 2) & ~15u;
    mbar_arrive_expect_tx(mbar, bk + bl);
    if (bk) bulk_g2s(in_s, src + start, bk, mbar);
    if (bl) bulk_g2s(lpi_s, lpi + start, bl, mbar);
  }
  BCF_SYNC();
  for (int i = (((len * 4) & ~15) >> 2) + threadIdx.x; i < len; i += blockDim.x) in_s[i] = src[start + i];
  for (int i = (((len * 2) & ~15) >> 1) + threadIdx.x; i < len; i += blockDim.x) lpi_s[i] = lpi[start + i];
  mbar_wait(mbar, 0, status);
  BCF_SYNC();
  return len;
}

template <int T>
__device__ __forceinline__ void write_tile(uint32_t* dst, int64_t start, int len,
                                          const uint32_t* out_s) {
  if (len == T) {
    const uint4* o4 = reinterpret_cast<const uint4*>(out_s);
    uint4* d4 = reinterpret_cast<uint4*>(dst + start);
    for (int i = threadIdx.x; i < T / 4; i += blockDim.x) {
      BCF_TR(&o4[i], 16, 0, TS_WRITEOUT_READ);
      __stcs(d4 + i, o4[i]);
    }
  } else {
    for (int i = threadIdx.x; i < len; i += blockDim.x) dst[start + i] = out_s[i];
  }
}

// Direct scatter, streamed: persistent blocks take tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...; the keys and labels of the next kTSBuffers - 1 tiles arrive by
// bulk copies into a ring of buffers while this one is scattered, and each
// finished tile leaves by a bulk store from shared memory that the block only
// waits on before it scatters the next tile.
constexpr int kTSThreads = 256;
#ifndef BCF_TS_BUFFERS
#define BCF_TS_BUFFERS 3
#endif
constexpr int kTSBuffers = BCF_TS_BUFFERS;  // tiles in flight per block: kTSBuffers - 1 ahead

template <int T>
struct TSSmem {
  static constexpr size_t in = 0;                                     // [kTSBuffers][T] keys
  static constexpr size_t lpi = in + kTSBuffers * (size_t)T * 4;      // [kTSBuffers][T] labels
  static constexpr size_t out = lpi + kTSBuffers * (size_t)T * 2;     // [T] scattered tile
  static constexpr size_t mbar = out + (size_t)T * 4;                 // [kTSBuffers]
  static constexpr size_t bytes = mbar + 8 * kTSBuffers;
};

template <int T>
__global__ void __launch_bounds__(kTSThreads) k_tile_scatter_stream(const uint32_t* __restrict__ src,
                                                                    uint32_t* __restrict__ dst,
                                                                    const uint16_t* __restrict__ lpi,
                                                                    int64_t n, int64_t tiles,
                                                                    unsigned* status) {
  using S = TSSmem<T>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* out_s = reinterpret_cast<uint32_t*>(smem + S::out);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::mbar);
  auto in_set = [&](int b) { return reinterpret_cast<uint32_t*>(smem + S::in) + b * T; };
  auto lpi_set = [&](int b) { return reinterpret_cast<uint16_t*>(smem + S::lpi) + b * T; };
  const int tid = threadIdx.x;
  auto issue = [&](int64_t t, int b) {  // one thread: bulk copies of tile t into buffer b
    const int len = (int)min((int64_t)T, n - t * T);
    const unsigned bk = (unsigned)(len * 4) & ~15u, bl = (unsigned)(len * 2) & ~15u;
    mbar_arrive_expect_tx(&mbar[b], bk + bl);
    if (bk) bulk_g2s(in_set(b), src + t * T, bk, &mbar[b]);
    if (bl) bulk_g2s(lpi_set(b), lpi + t * T, bl, &mbar[b]);
  };
  if (tid == 0) {
    for (int b = 0; b < kTSBuffers; ++b) mbar_init(&mbar[b], 1);
    for (int b = 0; b < kTSBuffers - 1; ++b)
      if ((int64_t)blockIdx.x + (int64_t)b * gridDim.x < tiles) issue(blockIdx.x + (int64_t)b * gridDim.x, b);
  }
  BCF_SYNC();
  int it = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
    const int b = it % kTSBuffers;
    uint32_t* in_s = in_set(b);
    uint16_t* lpi_s = lpi_set(b);
    const int len = (int)min((int64_t)T, n - t * T);
    if (len < T) {  // ragged last tile: the words past the bulk copies by plain loads
      for (int i = (((len * 4) & ~15) >> 2) + tid; i < len; i += kTSThreads) in_s[i] = src[t * T + i];
      for (int i = (((len * 2) & ~15) >> 1) + tid; i < len; i += kTSThreads) lpi_s[i] = lpi[t * T + i];
    }
    mbar_wait(&mbar[b], (it / kTSBuffers) & 1, status);  // bounded: a lost copy is recorded, not waited on
    if (tid == 0) {
      bulk_s2g_wait_read();  // the previous tile's store has read out_s
      // the buffer of the previous round is free again: refill it kTSBuffers - 1 tiles ahead
      const int64_t ahead = t + (int64_t)(kTSBuffers - 1) * gridDim.x;
      if (ahead < tiles) issue(ahead, (it + kTSBuffers - 1) % kTSBuffers);
    }
    BCF_SYNC();
#pragma unroll 4
    for (int q = tid; q < len; q += kTSThreads) {
      BCF_TR_WORD(&lpi_s[q], 0, TS_STAGE_READ);
      const uint32_t p = lpi_s[q];
      BCF_TR(&in_s[q], 4, 0, TS_STAGE_READ);
      if ((int)p < len) {
        BCF_TR(&out_s[p], 4, 1, TS_SCATTER);
        out_s[p] = in_s[q];
      } else {
        set_status(status, DEV_BAD_PERM);
      }
    }
    fence_proxy_async_smem();
    BCF_SYNC();
    const unsigned bo = (unsigned)(len * 4) & ~15u;
    if (tid == 0 && bo) {
      bulk_s2g(dst + t * T, out_s, bo);
      bulk_s2g_commit();
    }
    for (int i = (int)(bo >> 2) + tid; i < len; i += kTSThreads) dst[t * T + i] = out_s[i];
  }
  if (tid == 0) bulk_s2g_wait_read();  // shared memory stays valid until read out
}

// Coloured schedule.  Thread (warp g, lane l) owns row l's slots [g*M/4, (g+1)*M/4)
// and, in the send phase, colours [g*M/4, (g+1)*M/4).  Table entry tbl[k*32 + l]
// holds the item of colour k that row l sends this round: (label << 8) | slot.
// Sorted finish for the items still pending after the colouring rounds (the
// finishing step of Sec. 3).  The pending labels (i, j) -- destination bank i,
// slot j -- are ordered lexicographically by counting over the label space (a
// bitmap; labels are distinct integers below T), packed row-major into ceil(L/32)
// columns with row r in bank r, and sent in three conflict-free phases:
//  * middle labels of row r (bank neither r's first nor its last destination):
//    no other row holds a label for that bank, so every row sends one per step;
//  * first-group labels (bank = the row's first destination), label (i, j) in
//    step j: two rows sending in one step would need the same (i, j);
//  * last-group labels, likewise.
// Returns nothing; every pending item is written to out_s.
template <int T>
__device__ __forceinline__ void sorted_finish(uint32_t pending, const uint32_t* in_s, uint32_t* out_s,
                                              unsigned char* smem) {
  using S = TPSmem<T>;
  constexpr int M = S::M, WARPS = kTPThreads / 32, SPW = M / WARPS, NW = T / 32;
  const uint32_t* lab = reinterpret_cast<const uint32_t*>(smem + S::lab);
  uint16_t* src_of = reinterpret_cast<uint16_t*>(smem + S::lpi);  // staged labels no longer needed
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + S::bits);
  uint32_t* pkl = reinterpret_cast<uint32_t*>(smem + S::lab);     // filled after lab is read
  uint32_t* pkk = reinterpret_cast<uint32_t*>(smem + S::tbl);     // colour table no longer needed
  uint32_t* scr = reinterpret_cast<uint32_t*>(smem + S::scr);
  static_assert(S::bytes_sorted - S::scr == WARPS * 4, "one scan word per warp");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int w = tid; w < NW; w += kTPThreads) {
    BCF_TR(&bits[w], 4, 1, TS_COL_TABLE);
    bits[w] = 0;
  }
  BCF_SYNC();
  // Key of label p = j*32 + i in destination order: i*M + j.
  for (uint32_t pend = pending; pend; pend &= pend - 1) {
    const int s = warp * SPW + __ffs(pend) - 1, q = s * 32 + lane;
    BCF_TR(&lab[q], 4, 0, TS_COL_READ);
    const uint32_t p = lab[q];
    const uint32_t key = (p & 31u) * M + (p >> 5);
    BCF_TR(&bits[key >> 5], 4, 2, TS_COL_PACK);
    atomicOr(&bits[key >> 5], 1u << (key & 31));
    BCF_TR_WORD(&src_of[key], 1, TS_COL_PACK);
    src_of[key] = (uint16_t)q;
  }
  BCF_SYNC();
  // Ranks: exclusive scan of the words' popcounts (one word per thread).
  uint32_t word = 0;
  if (tid < NW) {
    BCF_TR(&bits[tid], 4, 0, TS_COL_TABLE);
    word = bits[tid];
  }
  const uint32_t c = __popc(word);
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scr[warp] = x;
  BCF_SYNC();
  uint32_t before = 0, total = 0;
#pragma unroll
  for (int g = 0; g < WARPS; ++g) {
    const uint32_t t = scr[g];
    if (g < warp) before += t;
    total += t;
  }
  BCF_SYNC();
  const int L = (int)total;
  if (L == 0) return;
  const int C = (L + 31) / 32;  // columns of the packed matrix
  uint32_t rank = before + x - c;
  for (uint32_t b = word; b; b &= b - 1, ++rank) {
    const uint32_t key = (uint32_t)tid * 32 + (uint32_t)(__ffs(b) - 1);
    const uint32_t p = (key % M) * 32 + key / M;  // back to the label
    const int r = (int)rank / C, t = (int)rank % C;
    BCF_TR_WORD(&src_of[key], 0, TS_COL_PACK);
    const uint32_t q = src_of[key];
    BCF_TR(&in_s[q], 4, 0, TS_COL_PACK);
    BCF_TR(&pkl[t * 32 + r], 4, 1, TS_COL_PACK);
    pkl[t * 32 + r] = p;
    BCF_TR(&pkk[t * 32 + r], 4, 1, TS_COL_PACK);
    pkk[t * 32 + r] = in_s[q];
  }
  BCF_SYNC();
  if (warp != 0) return;
  // Row `lane` of the packed matrix lives in bank `lane`.
  const int nr = max(0, min(C, L - lane * C));
  uint32_t i_first = 32, i_last = 32;
  if (nr > 0) {
    BCF_TR(&pkl[lane], 4, 0, TS_COL_READ);
    i_first = pkl[lane] & 31u;
    BCF_TR(&pkl[(nr - 1) * 32 + lane], 4, 0, TS_COL_READ);
    i_last = pkl[(nr - 1) * 32 + lane] & 31u;
  }
  auto send = [&](int t) {
    BCF_TR(&pkl[t * 32 + lane], 4, 0, TS_COL_READ);
    const uint32_t p = pkl[t * 32 + lane];
    BCF_TR(&pkk[t * 32 + lane], 4, 0, TS_COL_READ);
    const uint32_t v = pkk[t * 32 + lane];
    BCF_TR(&out_s[p], 4, 1, TS_COL_FINISH);
    out_s[p] = v;
  };
  for (int t = 0; t < C; ++t) {  // middle labels, one per row per step
    bool go = false;
    if (t < nr) {
      BCF_TR(&pkl[t * 32 + lane], 4, 0, TS_COL_READ);
      const uint32_t i = pkl[t * 32 + lane] & 31u;
      go = i != i_first && i != i_last;
    }
    if (go) send(t);
  }
  // First group: a prefix sorted by slot; label (i_first, j) goes in step j.
  // Steps past every row's last first-group label are skipped.
  int nf = 0;
  while (nf < nr && (pkl[nf * 32 + lane] & 31u) == i_first) ++nf;
  int cur = 0;
  for (int j = 0; j < M && __any_sync(0xffffffffu, cur < nf); ++j) {
    bool go = false;
    if (cur < nf) {
      BCF_TR(&pkl[cur * 32 + lane], 4, 0, TS_COL_READ);
      go = (int)(pkl[cur * 32 + lane] >> 5) == j;
    }
    if (go) send(cur++);
  }
  // Last group (when the row has a different last destination): a suffix.
  int beg = nr;
  if (i_last != i_first)
    while (beg > 0 && (pkl[(beg - 1) * 32 + lane] & 31u) == i_last) --beg;
  for (int j = 0; j < M && __any_sync(0xffffffffu, beg < nr); ++j) {
    bool go = false;
    if (beg < nr) {
      BCF_TR(&pkl[beg * 32 + lane], 4, 0, TS_COL_READ);
      go = (int)(pkl[beg * 32 + lane] >> 5) == j;
    }
    if (go) send(beg++);
  }
}

template <int T>
__global__ void __launch_bounds__(kTPThreads, kTPThreads >= 1024 ? 2 : 3) k_tile_coloured(const uint32_t* __restrict__ src,
                                                              uint32_t* __restrict__ dst,
                                                              const uint16_t* __restrict__ lpi,
                                                              int64_t n, uint64_t seed,
                                                              int rounds, int sorted, unsigned* status) {
  using S = TPSmem<T>;
  constexpr int M = S::M;          // columns (slots per bank) = colours
  constexpr int WARPS = kTPThreads / 32;
  constexpr int SPW = M / WARPS;   // slots (and colours) per warp
  static_assert(SPW <= 32, "one pending bit per owned slot");
  constexpr uint32_t EMPTY = 0xFFFFFFFFu;
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* in_s = reinterpret_cast<uint32_t*>(smem + S::in);
  uint16_t* lpi_s = reinterpret_cast<uint16_t*>(smem + S::lpi);
  uint32_t* out_s = reinterpret_cast<uint32_t*>(smem + S::out);
  uint32_t* tbl = reinterpret_cast<uint32_t*>(smem + S::tbl);
  uint32_t* lab = reinterpret_cast<uint32_t*>(smem + S::lab);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::mbar);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = blockIdx.x;
  const int len = stage_tile<T>(src, lpi, n, tile, in_s, lpi_s, mbar, status);
  // This thread's labels, read once into registers.  All lanes of a warp read the
  // same slot at once, so the two lanes of each 16-bit pair read one word and a
  // request touches 16 distinct banks.  Pending slots of this thread: labels
  // outside the tile are dropped (and flagged).
  uint32_t labr[SPW];
  uint32_t pending = 0;
#pragma unroll
  for (int c = 0; c < SPW; ++c) {
    const int q = (warp * SPW + c) * 32 + lane;
    labr[c] = 0u;
    if (q < len) {
      BCF_TR_WORD(&lpi_s[q], 0, TS_COL_READ);
      labr[c] = lpi_s[q];
      if ((int)labr[c] < len) pending |= 1u << c;
      else set_status(status, DEV_BAD_PERM);
    }
  }
  // The sorted finish reads pending labels by slot, from lanes at different slots:
  // it gets them widened to one word each, so row l's labels sit in bank l.
  if (sorted) {
    for (int q = threadIdx.x; q < T; q += kTPThreads) {
      if (q < len) BCF_TR_WORD(&lpi_s[q], 0, TS_COL_READ);
      BCF_TR(&lab[q], 4, 1, TS_COL_READ);
      lab[q] = q < len ? (uint32_t)lpi_s[q] : 0u;
    }
  }

  // The colour table starts empty; afterwards every send step empties the entry it
  // has just sent, so each round begins with an empty table.
  for (int k = warp * SPW; k < (warp + 1) * SPW; ++k) {
    BCF_TR(&tbl[k * 32 + lane], 4, 1, TS_COL_TABLE);
    tbl[k * 32 + lane] = EMPTY;
  }
  BCF_SYNC();
  for (int r = 0; r < rounds; ++r) {
    // Coloring: h(i) for destination bank i, drawn fresh every round (held by lane i).
    const uint32_t h_lane = mix32(seed ^ ((uint64_t)tile << 20) ^ ((uint64_t)r << 8) ^ (uint64_t)lane) & (M - 1);
    // Claim the first free entry of each colour in this row; an item whose colour
    // is already taken stays pending for the next round.  Slot by slot, in the
    // same order on every lane, so the loop has no divergent trip count.
#pragma unroll
    for (int c = 0; c < SPW; ++c) {
      const uint32_t p = labr[c];
      const uint32_t hi = __shfl_sync(0xffffffffu, h_lane, (int)(p & 31u));  // h(i), i = p mod 32
      if ((pending >> c) & 1u) {
        const uint32_t k = ((p >> 5) - hi) & (M - 1);
        BCF_TR(&tbl[k * 32 + lane], 4, 2, TS_COL_TABLE);
        if (atomicCAS(&tbl[k * 32 + lane], EMPTY, (p << 8) | (uint32_t)(warp * SPW + c)) == EMPTY)
          pending &= ~(1u << c);
      }
    }
    BCF_SYNC();
    // Communication: in step k every row sends its colour-k item (if any); the
    // destination banks of one step are distinct.
#pragma unroll 4
    for (int k = warp * SPW; k < (warp + 1) * SPW; ++k) {
      BCF_TR(&tbl[k * 32 + lane], 4, 0, TS_COL_TABLE);
      const uint32_t e = tbl[k * 32 + lane];
      if (e != EMPTY) {
        BCF_TR(&in_s[(e & 0xFFu) * 32 + lane], 4, 0, TS_COL_READ);
        BCF_TR(&out_s[e >> 8], 4, 1, TS_COL_SEND);
        out_s[e >> 8] = in_s[(e & 0xFFu) * 32 + lane];
        BCF_TR(&tbl[k * 32 + lane], 4, 1, TS_COL_TABLE);
        tbl[k * 32 + lane] = EMPTY;
      }
    }
    BCF_SYNC();
  }

  if (sorted) {
    sorted_finish<T>(pending, in_s, out_s, smem);
    pending = 0;
  }
  // Finish: greedy conflict-free sends.  Each lane offers its next pending item;
  // among lanes aiming at one destination bank only the lowest sends.
  while (__any_sync(0xffffffffu, pending != 0)) {
    const int c = pending ? __ffs(pending) - 1 : 0;
    const int s = warp * SPW + c;
    uint32_t p = 0u;
#pragma unroll
    for (int u = 0; u < SPW; ++u)  // the label of slot c, from registers
      if (u == c && pending) p = labr[u];
    const uint32_t bank = pending ? (p & 31u) : 32u + (uint32_t)lane;  // idle lanes never collide
    const unsigned peers = __match_any_sync(0xffffffffu, bank);
    if (pending && lane == __ffs(peers) - 1) {
      BCF_TR(&in_s[s * 32 + lane], 4, 0, TS_COL_READ);
      BCF_TR(&out_s[p], 4, 1, TS_COL_FINISH);
      out_s[p] = in_s[s * 32 + lane];
      pending &= ~(1u << c);
    }
  }
  BCF_SYNC();
  write_tile<T>(dst, tile * T, len, out_s);
}

template <int T>
static cudaError_t launch_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi,
                                int64_t n, bool coloured, bool sorted, uint64_t seed, cudaStream_t s) {
  using S = TPSmem<T>;
  const int64_t tiles = (n + T - 1) / T;
  if (coloured) {
    auto k = k_tile_coloured<T>;
    const int bytes = (int)(sorted ? S::bytes_sorted : S::bytes_coloured);
    static bool ready[64] = {};
    const cudaError_t e = set_smem_once(k, (int)S::bytes_sorted, ready);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)tiles, kTPThreads, bytes, s>>>(src, dst, lpi, n, seed, kTPRounds, sorted ? 1 : 0, status_word());
  } else {
    using SS = TSSmem<T>;
    auto k = k_tile_scatter_stream<T>;
    static int resident[64] = {0};  // per device: blocks resident at once (shared-memory limit set)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!resident[dev]) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS::bytes);
      if (e != cudaSuccess) return e;
      int sms = 148, per_sm = 1;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTSThreads, SS::bytes);
      resident[dev] = sms * std::max(per_sm, 1);
    }
    const int64_t grid = std::min<int64_t>(tiles, resident[dev]);
    k<<<(unsigned)grid, kTSThreads, SS::bytes, s>>>(src, dst, lpi, n, tiles, status_word());
  }
  return cudaGetLastError();
}

cudaError_t permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi, int64_t n,
                          int tile, bool coloured, bool sorted, uint64_t seed, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  switch (tile) {
    case 1024: return launch_tiles<1024>(src, dst, lpi, n, coloured, sorted, seed, s);
    case 2048: return launch_tiles<2048>(src, dst, lpi, n, coloured, sorted, seed, s);
    case 4096: return launch_tiles<4096>(src, dst, lpi, n, coloured, sorted, seed, s);
  }
  return cudaErrorInvalidValue;
}

BCF_TRACE_INSTALLER(tile_permute)

}  // namespace bcf
