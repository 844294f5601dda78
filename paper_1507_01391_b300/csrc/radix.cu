// radix.cu -- stable digit sweeps: LSD radix sort and w-way partition.
//
// One sweep moves every key to the block of its digit (or partition label).  It
// is the paper's partition problem (Sec. 1) at GPU scale: each block of threads
// ranks one tile of keys in shared memory -- the per-row "radix sort" of
// Corollary 1 done per warp -- and finds the tile's global offsets with a
// decoupled look-back over earlier tiles.  Keys and payloads are staged into
// shared memory by bulk copies (TMA engine), read back with the conflict-free
// strided pattern of Sec. 1 (lane t reads word 32i + t), and written out in
// digit order so that global stores form contiguous runs.
#include "common.cuh"
#include "internal.h"

namespace bcf {

constexpr uint32_t LB_AGG = 1u << 30;   // tile aggregate published
constexpr uint32_t LB_INC = 2u << 30;   // inclusive prefix published
constexpr uint32_t LB_MASK = (1u << 30) - 1;

struct SweepParams {
  const uint32_t* keys_in;
  const void* vals_in;
  uint32_t* keys_out;
  void* vals_out;
  int64_t n;
  int shift, nbits;            // radix digit = (key >> shift) & (2^nbits - 1)
  int w;                       // > 0: partition by label, labels must be < w
  int balanced;                // partition: block b starts at b * n / w
  const uint32_t* digit_base;  // exclusive global start of every digit
  uint32_t* lookback;          // tiles x RADIX status words, zero on entry
  uint32_t* ticket;            // tile counter, zero on entry
  unsigned* status;
};

template <int BITS>
__device__ __forceinline__ uint32_t digit_of(uint32_t key, int w, int shift, int nbits) {
  if (w > 0) return key & ((1u << BITS) - 1u);
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
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < WARPS ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < WARPS) scratch[lane] = s;
  }
  __syncthreads();
  const uint32_t before = warp ? scratch[warp - 1] : 0u;
  *total = scratch[WARPS - 1];
  __syncthreads();
  return before + x - v;
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
};

// Counts every digit of every pass in one read of the keys; the last block to
// finish turns the counts into exclusive starts.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_histogram(HistParams p) {
  __shared__ uint32_t h[4 * 256];
  __shared__ uint32_t scratch[32];
  __shared__ int is_last;
  const int tid = threadIdx.x;
  for (int i = tid; i < 4 * 256; i += THREADS) h[i] = 0;
  __syncthreads();
  uint32_t mask[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    mask[q] = p.label_bits ? ((1u << p.label_bits) - 1u) : ((1u << p.nbits[q]) - 1u);
  const int64_t nvec = p.n >> 2;
  const uint4* kv = reinterpret_cast<const uint4*>(p.keys);
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  for (int64_t i = (int64_t)blockIdx.x * THREADS + tid; i < nvec; i += stride) {
    uint4 k4 = __ldcs(kv + i);
    uint32_t k[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < p.passes) atomicAdd(&h[q * 256 + ((k[c] >> p.shift[q]) & mask[q])], 1u);
    }
  }
  for (int64_t i = nvec * 4 + (int64_t)blockIdx.x * THREADS + tid; i < p.n; i += stride) {
    uint32_t k = p.keys[i];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < p.passes) atomicAdd(&h[q * 256 + ((k >> p.shift[q]) & mask[q])], 1u);
  }
  __syncthreads();
  for (int i = tid; i < p.passes * 256; i += THREADS)
    if (h[i]) atomicAdd(&p.hist[i], h[i]);
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(p.done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int q = 0; q < p.passes; ++q) {
    uint32_t c = tid < 256 ? ld_relaxed(&p.hist[q * 256 + tid]) : 0u;
    uint32_t total;
    uint32_t e = block_excl_scan<THREADS>(c, scratch, &total);
    if (tid < 256) p.digit_base[q * 256 + tid] = e;
  }
}

// ------------------------------------------------------------- one sweep
template <int THREADS, int IPT, int BITS, int VB>
struct SweepSmem {
  static constexpr int T = THREADS * IPT;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int RADIX = 1 << BITS;
  static constexpr size_t keys = 0;
  static constexpr size_t vals = keys + (size_t)T * 4;
  static constexpr size_t whist = vals + (size_t)T * VB;
  static constexpr size_t tstart = whist + (size_t)WARPS * RADIX * 4;
  static constexpr size_t gofs = tstart + (size_t)RADIX * 4;
  static constexpr size_t scratch = gofs + (size_t)RADIX * 4;
  static constexpr size_t mbar = scratch + 32 * 4;
  static constexpr size_t tile = mbar + 8;
  static constexpr size_t bytes = tile + 8;
};

template <int THREADS, int IPT, int BITS, int VB>
__global__ void __launch_bounds__(THREADS) k_sweep(SweepParams p) {
  using VT = typename ValT<VB>::type;
  using S = SweepSmem<THREADS, IPT, BITS, VB>;
  constexpr int T = S::T, RADIX = S::RADIX;
  static_assert(RADIX <= THREADS, "one thread per digit");
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* keys_s = reinterpret_cast<uint32_t*>(smem + S::keys);
  VT* vals_s = reinterpret_cast<VT*>(smem + S::vals);
  uint32_t* whist = reinterpret_cast<uint32_t*>(smem + S::whist);
  uint32_t* tstart = reinterpret_cast<uint32_t*>(smem + S::tstart);
  uint32_t* gofs = reinterpret_cast<uint32_t*>(smem + S::gofs);
  uint32_t* scratch = reinterpret_cast<uint32_t*>(smem + S::scratch);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::mbar);
  int* s_tile = reinterpret_cast<int*>(smem + S::tile);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // Tiles are taken in launch order so that every tile a look-back waits on
  // belongs to a block that is already running.
  if (tid == 0) {
    const int tile = (int)atomicAdd(p.ticket, 1u);
    *s_tile = tile;
    mbar_init(mbar, 1);
    const int64_t start = (int64_t)tile * T;
    const int cnt = (int)min((int64_t)T, p.n - start);
    const unsigned bk = (unsigned)(cnt * 4) & ~15u;
    const unsigned bv = VB ? ((unsigned)(cnt * VB) & ~15u) : 0u;
    mbar_arrive_expect_tx(mbar, bk + bv);
    if (bk) bulk_g2s(keys_s, p.keys_in + start, bk, mbar);
    if (VB && bv) bulk_g2s(vals_s, reinterpret_cast<const VT*>(p.vals_in) + start, bv, mbar);
  }
  for (int i = tid; i < S::WARPS * RADIX; i += THREADS) whist[i] = 0;
  __syncthreads();
  const int tile = *s_tile;
  const int64_t start = (int64_t)tile * T;
  const int cnt = (int)min((int64_t)T, p.n - start);
  // the last few elements that do not fill a 16-byte chunk: plain loads
  for (int i = ((cnt * 4) & ~15) / 4 + tid; i < cnt; i += THREADS) keys_s[i] = p.keys_in[start + i];
  if (VB) {
    for (int i = ((cnt * VB) & ~15) / VB + tid; i < cnt; i += THREADS)
      vals_s[i] = reinterpret_cast<const VT*>(p.vals_in)[start + i];
  }
  mbar_wait(mbar, 0, p.status);
  __syncthreads();

  // Registers, warp-striped: lane l of warp q holds tile items q*32*IPT + 32j + l.
  // Reading them is the strided pattern: lane l always in bank l.
  uint32_t key[IPT], dig[IPT], rank[IPT];
  VT val[IPT];
  const int wbase = warp * 32 * IPT;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const int idx = wbase + j * 32 + lane;
    const bool valid = idx < cnt;
    key[j] = valid ? keys_s[idx] : 0u;
    if (VB) val[j] = valid ? vals_s[idx] : VT(0);
    if (valid && p.w > 0 && key[j] >= (uint32_t)p.w) set_status(p.status, DEV_BAD_KEY);
    dig[j] = valid ? digit_of<BITS>(key[j], p.w, p.shift, p.nbits) : (uint32_t)RADIX;
  }

  // Warp ranking: peers with the same digit, stable rank = earlier peers plus
  // this warp's running count of the digit (kept per warp in shared memory).
  uint32_t* wh = whist + warp * RADIX;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t d = dig[j];
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && d < (uint32_t)RADIX) {
      old = wh[d];
      wh[d] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[j] = old + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();

  // Per digit: warp counts -> exclusive warp offsets; tile count per digit.
  uint32_t count = 0;
  if (tid < RADIX) {
#pragma unroll 4
    for (int q = 0; q < S::WARPS; ++q) {
      const uint32_t c = whist[q * RADIX + tid];
      whist[q * RADIX + tid] = count;
      count += c;
    }
  }
  uint32_t total;
  const uint32_t tile_excl = block_excl_scan<THREADS>(tid < RADIX ? count : 0u, scratch, &total);
  if (tid < RADIX) {
    tstart[tid] = tile_excl;
    // Decoupled look-back: publish this tile's count, then add up earlier
    // tiles' counts until one has published its inclusive prefix.
    uint32_t* lb = p.lookback + (size_t)tile * RADIX + tid;
    uint32_t excl = 0;
    if (tile == 0) {
      st_relaxed(lb, LB_INC | count);
    } else {
      st_relaxed(lb, LB_AGG | count);
      int pred = tile - 1;
      unsigned spins = 0;
      while (true) {
        const uint32_t v = ld_relaxed(p.lookback + (size_t)pred * RADIX + tid);
        const uint32_t f = v & ~LB_MASK;
        if (f == 0) {
          if (++spins > kSpinLimit) {
            set_status(p.status, DEV_TIMEOUT);
            break;
          }
          continue;
        }
        excl += v & LB_MASK;
        if (f == LB_INC || pred == 0) break;
        --pred;
      }
      st_relaxed(lb, LB_INC | (excl + count));
    }
    uint32_t base;
    if (p.balanced) {
      const int64_t b = (int64_t)tid * (p.n / p.w);
      base = (uint32_t)min(b, p.n);
      if (tile == (int)gridDim.x - 1) {
        const uint32_t expect = tid < p.w ? (uint32_t)(p.n / p.w) : 0u;
        if (excl + count != expect) set_status(p.status, DEV_NOT_BALANCED);
      }
    } else {
      base = p.digit_base[tid];
    }
    gofs[tid] = base + excl - tile_excl;
  }
  __syncthreads();

  // Scatter into shared memory in digit order.
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t d = dig[j];
    if (d < (uint32_t)RADIX) {
      const uint32_t pos = tstart[d] + wh[d] + rank[j];
      keys_s[pos] = key[j];
      if (VB) vals_s[pos] = val[j];
    }
  }
  __syncthreads();

  // Write out: consecutive threads take consecutive sorted positions, so the
  // stores of one digit's run are contiguous in global memory.
  VT* vout = reinterpret_cast<VT*>(p.vals_out);
  for (int i = tid; i < cnt; i += THREADS) {
    const uint32_t k = keys_s[i];
    const uint32_t d = digit_of<BITS>(k, p.w, p.shift, p.nbits);
    const uint32_t dst = gofs[d] + (uint32_t)i;
    if ((int64_t)dst < p.n) {
      p.keys_out[dst] = k;
      if (VB) vout[dst] = vals_s[i];
    }
  }
}

// ------------------------------------------------------------- host side
PassPlan plan_passes(int key_bits) {
  PassPlan pl;
  pl.passes = (key_bits + 7) / 8;
  int shift = 0;
  for (int q = 0; q < pl.passes; ++q) {
    int bits = key_bits / pl.passes + (q < key_bits % pl.passes ? 1 : 0);
    pl.shift[q] = shift;
    pl.nbits[q] = bits;
    shift += bits;
  }
  return pl;
}

SweepLayout sweep_layout(int64_t n, int val_bytes, int passes, int radix, bool need_tmp) {
  SweepLayout L;
  L.radix = radix;
  L.tiles = (n + kSweepTile - 1) / kSweepTile;
  size_t off = 0;
  if (need_tmp) {
    L.keys_tmp = off;
    off = align_up(off + (size_t)n * 4);
    L.vals_tmp = off;
    off = align_up(off + (size_t)n * val_bytes);
  }
  L.digit_base = off;
  off = align_up(off + 4 * 256 * 4);
  L.zero_begin = off;
  L.hist = off;
  off = align_up(off + 4 * 256 * 4);
  L.counters = off;
  off = align_up(off + 8 * 4);
  L.lookback = off;
  off = align_up(off + (size_t)(passes > 0 ? passes : 1) * L.tiles * radix * 4);
  L.zero_bytes = off - L.zero_begin;
  L.total = off;
  return L;
}

template <int BITS, int VB>
static cudaError_t launch_sweep(const SweepParams& p, int64_t tiles, cudaStream_t s) {
  using S = SweepSmem<kSweepThreads, kSweepIPT, BITS, VB>;
  auto kern = k_sweep<kSweepThreads, kSweepIPT, BITS, VB>;
  static bool configured = false;  // attribute is per device function; idempotent
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  kern<<<(unsigned)tiles, kSweepThreads, S::bytes, s>>>(p);
  return cudaGetLastError();
}

template <int BITS>
static cudaError_t sweep_dispatch(const SweepParams& p, int64_t tiles, int vb, cudaStream_t s) {
  switch (vb) {
    case 0: return launch_sweep<BITS, 0>(p, tiles, s);
    case 4: return launch_sweep<BITS, 4>(p, tiles, s);
    case 8: return launch_sweep<BITS, 8>(p, tiles, s);
  }
  return cudaErrorInvalidValue;
}

static int hist_grid(int64_t n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (n / 4 + 255) / 256;
  int64_t g = sms * 4;
  if (want < g) g = want > 0 ? want : 1;
  return (int)g;
}

cudaError_t radix_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n, int vb, const PassPlan& plan,
                       unsigned char* ws, const SweepLayout& L, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* base = reinterpret_cast<uint32_t*>(ws + L.digit_base);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(ws + L.counters);
  uint32_t* lb = reinterpret_cast<uint32_t*>(ws + L.lookback);

  HistParams hp{};
  hp.keys = keys_in;
  hp.n = n;
  hp.passes = plan.passes;
  for (int q = 0; q < 4; ++q) {
    hp.shift[q] = plan.shift[q];
    hp.nbits[q] = plan.nbits[q] ? plan.nbits[q] : 1;
  }
  hp.label_bits = 0;
  hp.hist = hist;
  hp.digit_base = base;
  hp.done = ctr + 4;
  k_histogram<256><<<hist_grid(n), 256, 0, s>>>(hp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // Ping-pong so that the last pass lands in keys_out.  When sorting in place
  // with an odd pass count, every pass alternates tmp/out starting from tmp and
  // a final copy brings the result home.
  uint32_t* kt = reinterpret_cast<uint32_t*>(ws + L.keys_tmp);
  void* vt = vb ? (void*)(ws + L.vals_tmp) : nullptr;
  const bool in_place = (keys_in == keys_out);
  const int P = plan.passes;
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  bool odd_in_place = in_place && (P % 2 == 1);
  for (int q = 0; q < P; ++q) {
    bool to_out = odd_in_place ? (q % 2 == 1) : (((P - 1 - q) % 2) == 0);
    uint32_t* dk = to_out ? keys_out : kt;
    void* dv = to_out ? vals_out : vt;
    SweepParams sp{};
    sp.keys_in = src_k;
    sp.vals_in = src_v;
    sp.keys_out = dk;
    sp.vals_out = dv;
    sp.n = n;
    sp.shift = plan.shift[q];
    sp.nbits = plan.nbits[q];
    sp.w = 0;
    sp.balanced = 0;
    sp.digit_base = base + q * 256;
    sp.lookback = lb + (size_t)q * L.tiles * 256;
    sp.ticket = ctr + q;
    sp.status = status_word();
    if ((e = sweep_dispatch<8>(sp, L.tiles, vb, s)) != cudaSuccess) return e;
    src_k = dk;
    src_v = dv;
  }
  if (odd_in_place) {
    if ((e = cudaMemcpyAsync(keys_out, kt, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    if (vb && (e = cudaMemcpyAsync(vals_out, vt, (size_t)n * vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

cudaError_t partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                      void* vals_out, int64_t n, int w, int vb, bool balanced,
                      unsigned char* ws, const SweepLayout& L, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  const int bits = (L.radix == 32) ? 5 : 8;
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* base = reinterpret_cast<uint32_t*>(ws + L.digit_base);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(ws + L.counters);
  uint32_t* lb = reinterpret_cast<uint32_t*>(ws + L.lookback);
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  if (keys_in == keys_out) {  // in place: sweep from a copy of the input
    uint32_t* kt = reinterpret_cast<uint32_t*>(ws + L.keys_tmp);
    if ((e = cudaMemcpyAsync(kt, keys_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    src_k = kt;
    if (vb) {
      void* vt = ws + L.vals_tmp;
      if ((e = cudaMemcpyAsync(vt, vals_in, (size_t)n * vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
      src_v = vt;
    }
  }
  if (!balanced) {
    HistParams hp{};
    hp.keys = src_k;
    hp.n = n;
    hp.passes = 1;
    hp.shift[0] = 0;
    hp.nbits[0] = bits;
    hp.label_bits = bits;
    hp.hist = hist;
    hp.digit_base = base;
    hp.done = ctr + 4;
    k_histogram<256><<<hist_grid(n), 256, 0, s>>>(hp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  SweepParams sp{};
  sp.keys_in = src_k;
  sp.vals_in = src_v;
  sp.keys_out = keys_out;
  sp.vals_out = vals_out;
  sp.n = n;
  sp.shift = 0;
  sp.nbits = bits;
  sp.w = w;
  sp.balanced = balanced ? 1 : 0;
  sp.digit_base = base;
  sp.lookback = lb;
  sp.ticket = ctr;
  sp.status = status_word();
  if (bits == 5) return sweep_dispatch<5>(sp, L.tiles, vb, s);
  return sweep_dispatch<8>(sp, L.tiles, vb, s);
}

}  // namespace bcf
