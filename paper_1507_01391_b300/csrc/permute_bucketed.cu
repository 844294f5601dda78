// permute_bucketed.cu -- the permutation dst[pi[i]] = src[i] (Sec. 1) in two
// coalesced passes through a workspace, instead of one scattered store per element.
//
// A scattered 4-byte store costs one L2 sector operation however few bytes it
// carries, and L2 accepts only so many of those per second; that rate, not HBM
// bandwidth, bounds the one-pass scatter.  Here every store is part of a run:
//
//  Pass 1 (k_pb_bucket): persistent blocks take tiles of kPbTile elements; a tile's
//    pi, keys and payloads stream into shared memory by bulk copies while the
//    previous tile is processed.  Element i belongs to destination block
//    b = pi[i] / len (len destinations each, len <= kPbMaxLen).  A tile is counted
//    per block, reordered into block order in shared memory, and each run is
//    written to the block's region of the workspace at an offset claimed with one
//    global atomic per (tile, block).  Only the offset pi[i] - b * len (16 bits)
//    travels with the element.  The order inside a region is whatever the claims
//    produced; pass 2 does not depend on it.
//  Pass 2 (k_pb_place): one thread block per destination block reads the region in
//    order, stores every element at its offset in shared memory (len x 4 bytes),
//    then writes the block of dst with 16-byte stores; payloads take a second round.
//
// The block length is chosen so that the number of destination blocks is a
// multiple of the SM count: pass 2 then runs in whole waves of one block per SM,
// with no partly filled last wave.
//
// Traffic per element: pass 1 reads 4 + 4 + vb bytes and writes 2 + 4 + vb, pass 2
// reads them back (plus the offsets again for the payload round) and writes
// 4 + vb -- about twice the one-pass bytes, but in whole sectors.
#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"

namespace bcf {

int sm_count_cached() {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!sms[dev]) {
    int c = 148;
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = c;
  }
  return sms[dev];
}

namespace {

constexpr int kPbMaxLen = 53248;   // destinations per block at most (shared memory of pass 2)
constexpr int kPbMinLen = 4096;    // ... and at least
constexpr int kPbMagicShift = 42;  // b = (pi * magic) >> 42 is pi / len for pi < 2^26, len < 2^16
constexpr int kPbThreads = 1024, kPbIPT = 8;
constexpr int kPbTile = kPbThreads * kPbIPT;  // 8192 elements per pass-1 tile
constexpr int kPbMaxBlocks = 2048;
constexpr int64_t kPbMaxN = (int64_t)1 << 26;
constexpr int kPlaceThreads = 1024;
constexpr int kBulkChunk = 1 << 16;  // bytes per bulk store of the pass-2 write-out
#ifndef BCF_PB_UNROLL
#define BCF_PB_UNROLL 2
#endif
#ifndef BCF_PB_GROUPS
#define BCF_PB_GROUPS 1
#endif
constexpr int kPlaceGroups = BCF_PB_GROUPS;  // pass 2: groups of 8 elements in flight per thread
#ifndef BCF_PB_EVICT_FIRST
#define BCF_PB_EVICT_FIRST 1
#endif
constexpr uint32_t kNone = 0xFFFFFFFFu;

// Destination blocks: nb blocks of len positions (len a multiple of 8, so every
// block's region starts 16-byte aligned in all three workspace arrays).
struct PbGeom {
  int nb = 0;
  uint32_t len = 0;
  unsigned long long magic = 0;  // ceil(2^42 / len)
};

PbGeom pb_geometry(int64_t n) {
  const int64_t sms = std::max(1, sm_count_cached());
  const int64_t waves = std::max<int64_t>(1, (n + sms * kPbMaxLen - 1) / (sms * kPbMaxLen));
  int64_t len = (n + sms * waves - 1) / (sms * waves);
  len = std::max<int64_t>((len + 7) / 8 * 8, kPbMinLen);
  if ((n + len - 1) / len > kPbMaxBlocks) len = ((n + kPbMaxBlocks - 1) / kPbMaxBlocks + 7) / 8 * 8;
  PbGeom g;
  g.len = (uint32_t)len;
  g.nb = (int)((n + len - 1) / len);
  g.magic = ((1ull << kPbMagicShift) + (unsigned long long)len - 1) / (unsigned long long)len;
  return g;
}

struct PbLayout {
  size_t k1 = 0, v1 = 0, p1 = 0, fill = 0, total = 0;
};

PbLayout pb_layout(int64_t n, int vb) {
  PbLayout L;
  size_t off = 0;
  L.k1 = off;
  off = align_up(off + (size_t)n * 4);
  L.v1 = off;
  off = align_up(off + (size_t)n * vb);
  L.p1 = off;
  off = align_up(off + (size_t)n * 2 + 16);
  L.fill = off;
  off = align_up(off + (size_t)kPbMaxBlocks * 4);
  L.total = off;
  return L;
}

template <int NB>
constexpr int pb_smem_bytes() {
  // in: pi, keys, payloads; reordered: (key | payload << 32), (offset | block << 16);
  // per-block counts and write offsets; scan scratch; mbarrier
  return kPbTile * 4 * 3 + kPbTile * 8 + kPbTile * 4 + NB * 4 * 2 + 32 * 4 + 16;
}

template <int VB, int NB>
__global__ void __launch_bounds__(kPbThreads, 1)
    k_pb_bucket(const uint32_t* __restrict__ pi, const uint32_t* __restrict__ sk,
                const uint32_t* __restrict__ sv, uint32_t* __restrict__ K1, uint32_t* __restrict__ V1,
                uint16_t* __restrict__ P1, uint32_t* __restrict__ fill, int64_t n, int64_t row_len,
                int ntiles, uint32_t len, unsigned long long magic, unsigned* status) {
  constexpr int T = kPbTile;
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* in_p = reinterpret_cast<uint32_t*>(smem);
  uint32_t* in_k = in_p + T;
  uint32_t* in_v = in_k + T;
  unsigned long long* skv = reinterpret_cast<unsigned long long*>(in_v + T);
  uint32_t* spb = reinterpret_cast<uint32_t*>(skv + T);
  uint32_t* cur = spb + T;  // per-block count, then start, then cursor
  uint32_t* gofs = cur + NB;
  uint32_t* scratch = gofs + NB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(scratch + 32);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  auto bulk_elems = [&](int t) { return (int)min((int64_t)T, n - (int64_t)t * T) & ~3; };
  auto issue = [&](int t) {  // one thread: stream tile t into the in-buffers
    const int e = bulk_elems(t);
    const int64_t o = (int64_t)t * T;
    if (e > 0) {
      mbar_arrive_expect_tx(bar, (VB ? 3u : 2u) * (unsigned)e * 4u);
      bulk_g2s(in_p, pi + o, e * 4, bar);
      bulk_g2s(in_k, sk + o, e * 4, bar);
      if (VB) bulk_g2s(in_v, sv + o, e * 4, bar);
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int64_t base = (int64_t)t * T;
    const int cnt = (int)min((int64_t)T, n - base);
    const int be = bulk_elems(t);
    if (!mbar_wait(bar, it & 1, status)) {
      mbar_wait(bar, it & 1, status);  // give the copy in flight a last chance to land
      return;
    }
    // Each warp takes 32 consecutive elements per step: conflict-free reads.
    uint32_t d[kPbIPT], k[kPbIPT], v[kPbIPT];
#pragma unroll
    for (int j = 0; j < kPbIPT; ++j) {
      const int li = warp * (kPbIPT * 32) + j * 32 + lane;
      v[j] = 0;
      if (li < be) {
        d[j] = in_p[li];
        k[j] = in_k[li];
        if (VB) v[j] = in_v[li];
      } else if (li < cnt) {  // ragged end of the last tile
        d[j] = pi[base + li];
        k[j] = sk[base + li];
        if (VB) v[j] = sv[base + li];
      } else {
        d[j] = kNone;
        continue;
      }
      if (row_len > 0) {  // pi local to rows of row_len elements
        const int64_t i = base + li;
        const int64_t g = (int64_t)d[j] < row_len ? (i / row_len) * row_len + d[j] : n;
        d[j] = g < n ? (uint32_t)g : (uint32_t)n;
      }
      if ((int64_t)d[j] >= n) {
        set_status(status, DEV_BAD_PERM);
        d[j] = kNone;
        continue;
      }
      // (offset | block << 16): block = d / len, offset = d - block * len
      const uint32_t b = (uint32_t)(((unsigned long long)d[j] * magic) >> kPbMagicShift);
      d[j] = (d[j] - b * len) | (b << 16);
    }
    __syncthreads();  // in-buffers read; the previous tile's write-out is done
    for (int b = tid; b < NB; b += kPbThreads) cur[b] = 0;
    if (tid == 0 && t + (int)gridDim.x < ntiles) issue(t + gridDim.x);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPbIPT; ++j)
      if (d[j] != kNone) atomicAdd(&cur[d[j] >> 16], 1u);
    __syncthreads();

    // Block starts inside the tile; one claim per non-empty block, whose latency
    // the shared-memory reorder below hides.
    constexpr int PER = (NB + kPbThreads - 1) / kPbThreads;
    uint32_t c[PER], sum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int b = tid * PER + q;
      c[q] = b < NB ? cur[b] : 0u;
      sum += c[q];
    }
    uint32_t total;
    uint32_t run = block_excl_scan<kPbThreads>(sum, scratch, &total);
    uint32_t claim[PER], start[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int b = tid * PER + q;
      claim[q] = 0;
      start[q] = run;
      if (b < NB) {
        cur[b] = run;
        if (c[q]) claim[q] = atomicAdd(&fill[b], c[q]);
        run += c[q];
      }
    }
    __syncthreads();
    {
      uint32_t pos[kPbIPT];
#pragma unroll
      for (int j = 0; j < kPbIPT; ++j)  // every claim first, so none waits behind a store
        pos[j] = d[j] != kNone ? atomicAdd(&cur[d[j] >> 16], 1u) : 0u;
#pragma unroll
      for (int j = 0; j < kPbIPT; ++j) {
        if (d[j] == kNone) continue;
        skv[pos[j]] = ((unsigned long long)v[j] << 32) | k[j];
        spb[pos[j]] = d[j];
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int b = tid * PER + q;
      if (b < NB && c[q]) {
        const int64_t lo = (int64_t)b * len;
        const int64_t cap = min((int64_t)len, n - lo);
        if ((int64_t)claim[q] + c[q] > cap) {  // more elements than destinations: pi is no bijection
          set_status(status, DEV_BAD_PERM);
          gofs[b] = kNone;
        } else {
          gofs[b] = (uint32_t)(lo + claim[q]) - start[q];
        }
      }
    }
    __syncthreads();
    // Write-out: consecutive threads take consecutive reordered elements, so the
    // stores of one run are contiguous.  Only the `total` elements that passed the
    // range check were reordered; entries past them are stale.
    const int tot = (int)total;
    constexpr int U = BCF_PB_UNROLL;  // loads of U elements first, then their stores
    for (int i0 = tid; i0 < tot; i0 += U * kPbThreads) {
      uint32_t pb[U], g[U];
      unsigned long long kv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * kPbThreads;
        pb[u] = i < tot ? spb[i] : 0u;
        kv[u] = i < tot ? skv[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) g[u] = gofs[pb[u] >> 16];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * kPbThreads;
        if (i >= tot || g[u] == kNone) continue;
        const uint32_t dst = g[u] + (uint32_t)i;
        K1[dst] = (uint32_t)kv[u];
        if (VB) V1[dst] = (uint32_t)(kv[u] >> 32);
        P1[dst] = (uint16_t)pb[u];
      }
    }
  }
}

// Pass 2: destination block blockIdx.x.  CHECK: a bitmap of the block's offsets
// finds a destination hit twice (with no block over-full, that is the only way pi
// can fail to be a bijection).  Offsets are clamped below len: with a pi that is
// no bijection a region can hold entries no claim wrote, and those must not
// reach outside the shared buffer.
template <int VB, bool CHECK>
__global__ void __launch_bounds__(kPlaceThreads, 1)
    k_pb_place(const uint32_t* __restrict__ K1, const uint32_t* __restrict__ V1,
               const uint16_t* __restrict__ P1, uint32_t* __restrict__ dk, uint32_t* __restrict__ dv,
               int64_t n, uint32_t len, unsigned* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* xs = reinterpret_cast<uint32_t*>(smem);
  uint32_t* seen = xs + len;  // CHECK only
  const int tid = threadIdx.x;
  const int64_t lo = (int64_t)blockIdx.x * len;
  const int cap = (int)min((int64_t)len, n - lo);
  const uint32_t top = len - 1;
  if (CHECK) {
    for (int i = tid; i < (int)(len + 31) / 32; i += kPlaceThreads) seen[i] = 0;
    __syncthreads();
  }
  auto mark = [&](uint32_t o) {
    const uint32_t bit = 1u << (o & 31);
    if (atomicOr(&seen[o >> 5], bit) & bit) set_status(status, DEV_BAD_PERM);
  };
  const int nv = cap / 8;
  const int mv = cap / 4;
  // kPlaceGroups groups of 8 per thread per step, every load issued before any store.
  constexpr int G = kPlaceGroups;
  uint4 p[G], a[G], b[G];
  auto load = [&](const uint32_t* X, int t) {
#pragma unroll
    for (int h = 0; h < G; ++h) {
      const int th = t + h * kPlaceThreads;
      const int64_t i = lo + (int64_t)(th < nv ? th : t) * 8;
      p[h] = __ldcs(reinterpret_cast<const uint4*>(P1 + i));
      a[h] = __ldcs(reinterpret_cast<const uint4*>(X + i));
      b[h] = __ldcs(reinterpret_cast<const uint4*>(X + i + 4));
    }
  };
  auto place = [&](int t, bool marking) {
#pragma unroll
    for (int h = 0; h < G; ++h) {
      if (t + h * kPlaceThreads >= nv) break;
      const uint32_t o[8] = {min(p[h].x & 0xFFFFu, top), min(p[h].x >> 16, top),
                             min(p[h].y & 0xFFFFu, top), min(p[h].y >> 16, top),
                             min(p[h].z & 0xFFFFu, top), min(p[h].z >> 16, top),
                             min(p[h].w & 0xFFFFu, top), min(p[h].w >> 16, top)};
      const uint32_t x[8] = {a[h].x, a[h].y, a[h].z, a[h].w, b[h].x, b[h].y, b[h].z, b[h].w};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        xs[o[c]] = x[c];
        if (CHECK && marking) mark(o[c]);
      }
    }
  };
#pragma unroll 1
  for (int round = 0; round < (VB ? 2 : 1); ++round) {
    const uint32_t* X = round ? V1 : K1;
    uint32_t* D = round ? dv : dk;
    int t = tid;
    if (t < nv) load(X, t);
    if (round > 0) {  // the previous round's bulk write-out must have read xs
      if (tid == 0) bulk_s2g_wait_read();
      __syncthreads();
    }
    while (t < nv) {
      place(t, round == 0);
      t += G * kPlaceThreads;
      if (t < nv) load(X, t);
    }
    for (int i = nv * 8 + tid; i < cap; i += kPlaceThreads) {
      const uint32_t o = min((uint32_t)P1[lo + i], top);
      xs[o] = X[lo + i];
      if (CHECK && round == 0) mark(o);
    }
    // Write-out: one thread hands the block to the bulk-copy engine, which writes
    // it while the next round's first loads are in flight.
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && mv > 0) {
      for (int c = 0; c < mv; c += kBulkChunk / 16)
#if BCF_PB_EVICT_FIRST
        bulk_s2g_evict_first(D + lo + (int64_t)c * 4, xs + c * 4, (unsigned)min(kBulkChunk, (mv - c) * 16));
#else
        bulk_s2g(D + lo + (int64_t)c * 4, xs + c * 4, (unsigned)min(kBulkChunk, (mv - c) * 16));
#endif
      bulk_s2g_commit();
    }
    for (int j = mv * 4 + tid; j < cap; j += kPlaceThreads) D[lo + j] = xs[j];
  }
  if (tid == 0) bulk_s2g_wait_read();  // shared memory stays valid until read out
}

template <int VB, int NB>
cudaError_t run_bucketed(const uint32_t* sk, const uint32_t* sv, uint32_t* dk, uint32_t* dv,
                         const uint32_t* pi, int64_t n, int64_t row_len, bool check, const PbGeom& g,
                         unsigned char* ws, cudaStream_t s) {
  const PbLayout L = pb_layout(n, VB);
  uint32_t* K1 = reinterpret_cast<uint32_t*>(ws + L.k1);
  uint32_t* V1 = reinterpret_cast<uint32_t*>(ws + L.v1);
  uint16_t* P1 = reinterpret_cast<uint16_t*>(ws + L.p1);
  uint32_t* fill = reinterpret_cast<uint32_t*>(ws + L.fill);
  const int ntiles = (int)((n + kPbTile - 1) / kPbTile);
  cudaError_t e = cudaMemsetAsync(fill, 0, (size_t)g.nb * 4, s);
  if (e != cudaSuccess) return e;
  constexpr int sm1 = pb_smem_bytes<NB>();
  static bool ready1[64] = {};
  if ((e = set_smem_once(k_pb_bucket<VB, NB>, sm1, ready1)) != cudaSuccess) return e;
  const int grid = std::min(ntiles, sm_count_cached());
  k_pb_bucket<VB, NB><<<grid, kPbThreads, sm1, s>>>(pi, sk, sv, K1, V1, P1, fill, n, row_len, ntiles, g.len,
                                                    g.magic, status_word());
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the limit is raised once, to the largest block; a launch takes what its block needs
  constexpr int sm2_max = kPbMaxLen * 4 + kPbMaxLen / 8;
  const int sm2 = (int)g.len * 4 + (check ? (int)(g.len + 31) / 32 * 4 : 0);
  if (check) {
    static bool ready2[64] = {};
    if ((e = set_smem_once(k_pb_place<VB, true>, sm2_max, ready2)) != cudaSuccess) return e;
    k_pb_place<VB, true><<<g.nb, kPlaceThreads, sm2, s>>>(K1, V1, P1, dk, dv, n, g.len, status_word());
  } else {
    static bool ready2[64] = {};
    if ((e = set_smem_once(k_pb_place<VB, false>, sm2_max, ready2)) != cudaSuccess) return e;
    k_pb_place<VB, false><<<g.nb, kPlaceThreads, sm2, s>>>(K1, V1, P1, dk, dv, n, g.len, status_word());
  }
  return cudaGetLastError();
}

}  // namespace

bool permute_bucketed_supported(int64_t n, int kb, int vb) {
  return kb == 4 && (vb == 0 || vb == 4) && n > 0 && n <= kPbMaxN;
}

size_t permute_bucketed_workspace(int64_t n, int vb) { return pb_layout(n, vb).total; }

cudaError_t permute_bucketed(const uint32_t* sk, const uint32_t* sv, uint32_t* dk, uint32_t* dv,
                             const uint32_t* pi, int64_t n, int64_t row_len, int vb, bool check,
                             unsigned char* ws, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const PbGeom g = pb_geometry(n);
  const bool few = g.nb <= 512;
  if (vb == 4)
    return few ? run_bucketed<4, 512>(sk, sv, dk, dv, pi, n, row_len, check, g, ws, s)
               : run_bucketed<4, 2048>(sk, sv, dk, dv, pi, n, row_len, check, g, ws, s);
  return few ? run_bucketed<0, 512>(sk, sv, dk, dv, pi, n, row_len, check, g, ws, s)
             : run_bucketed<0, 2048>(sk, sv, dk, dv, pi, n, row_len, check, g, ws, s);
}

}  // namespace bcf
