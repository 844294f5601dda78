// partition_l1.cu -- w-way partition with the Lemma 1 tile schedule
// (BCF_PARTITION_LEMMA1).
//
// Same result as the digit sweep (a stable partition), but the order inside each
// 4096-key tile comes from Lemma 1 (Sec. 2) applied to (label, position) items:
// rows sorted inside their own bank pairs, diagonal row <-> column conversions, no
// bank conflicts by construction.  The global position of every (label, tile) run
// comes from the same tile counts and per-label scan as the sweep.  Corollary 1's
// O(m) row sorts (counting by label alone) would not keep equal labels in input
// order, which this library promises, so the rows are compared on the full item.
#include "common.cuh"
#include "internal.h"
#include "sweep.cuh"
#include "tile_sort.cuh"

namespace bcf {

template <int VB>
__global__ void __launch_bounds__(kL1Threads) k_partition_l1(const uint32_t* __restrict__ keys_in,
                                                             const void* __restrict__ vals_in,
                                                             uint32_t* __restrict__ keys_out,
                                                             void* __restrict__ vals_out, int64_t n,
                                                             int w, const uint32_t* __restrict__ offsets,
                                                             int64_t stride, unsigned* status) {
  using VT = typename ValT<VB>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* X = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* Y = X + kL1Tile;
  __shared__ uint32_t tstart[256];
  __shared__ uint32_t scratch[32];
  const int tid = threadIdx.x;
  const int64_t tile = blockIdx.x;
  const int64_t start = tile * kL1Tile;
  const int len = (int)min((int64_t)kL1Tile, n - start);
  tstart[tid] = 0;  // kL1Threads == 256 labels
  BCF_SYNC();
  for (int q = tid; q < kL1Tile; q += kL1Threads) {
    unsigned long long d = 0x100ull;  // padding sorts after every label
    if (q < len) {
      const uint32_t key = keys_in[start + q];
      if (key >= (uint32_t)w) set_status(status, DEV_BAD_KEY);
      d = key & 0xFFu;  // the label the tile counts used
      atomicAdd(&tstart[d], 1u);
    }
    BCF_TR(&X[q], 8, 1, TS_L1_IO);
    X[q] = (d << 32) | (unsigned)q;
  }
  BCF_SYNC();
  uint32_t total;
  const uint32_t c = tstart[tid];
  const uint32_t e = block_excl_scan<kL1Threads>(c, scratch, &total);
  tstart[tid] = e;  // first sorted position of label tid in this tile
  lemma1_schedule(X, Y);
  const VT* vin = reinterpret_cast<const VT*>(vals_in);
  VT* vout = reinterpret_cast<VT*>(vals_out);
  for (int t = tid; t < len; t += kL1Threads) {
    BCF_TR(&Y[t], 8, 0, TS_L1_IO);
    const unsigned long long it = Y[t];
    const uint32_t d = (uint32_t)(it >> 32), q = (uint32_t)it;
    const uint32_t dst = offsets[(size_t)d * stride + tile] + ((uint32_t)t - tstart[d]);
    if ((int64_t)dst < n) {
      keys_out[dst] = keys_in[start + q];
      if (VB) vout[dst] = vin ? vin[start + q] : VT(start + q);
    }
  }
}

cudaError_t partition_lemma1(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                             void* vals_out, int64_t n, int w, int vb, bool balanced,
                             unsigned char* ws, const SweepLayout& L, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(ws + L.lookback);
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  if (keys_in == keys_out) {  // in place: work from a copy of the input
    uint32_t* kt = reinterpret_cast<uint32_t*>(ws + L.keys_tmp);
    if ((e = cudaMemcpyAsync(kt, keys_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    src_k = kt;
    if (vb && vals_in) {
      void* vt = ws + L.vals_tmp;
      if ((e = cudaMemcpyAsync(vt, vals_in, (size_t)n * vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
      src_v = vt;
    }
  }
  const int64_t tiles = (n + kL1Tile - 1) / kL1Tile;
  const int64_t stride = (tiles + kLookbackWindow) / kLookbackWindow * kLookbackWindow;  // > tiles
  CountParams cp{};
  cp.keys = src_k;
  cp.n = n;
  cp.label_bits = 8;
  cp.counts = offsets;
  cp.stride = stride;
  cp.totals = totals;
  const int64_t count_blocks = (tiles + kCountTilesPerBlock - 1) / kCountTilesPerBlock;
  k_tile_counts<8, kL1Tile><<<(unsigned)count_blocks, 256, 0, s>>>(cp, tiles);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  launch_scan_offsets(256, offsets, tiles, stride, totals, balanced ? 1 : 0, n, w, status_word(), s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (vb) {
#define BCF_PL1(VB)                                                                                  \
  case VB: {                                                                                         \
    static bool ready[64] = {};                                                                      \
    if ((e = set_smem_once(k_partition_l1<VB>, (int)kL1SmemBytes, ready)) != cudaSuccess) return e;  \
    k_partition_l1<VB><<<(unsigned)tiles, kL1Threads, kL1SmemBytes, s>>>(                            \
        src_k, src_v, keys_out, vals_out, n, w, offsets, stride, status_word());                     \
    break;                                                                                           \
  }
    BCF_PL1(0)
    BCF_PL1(4)
    BCF_PL1(8)
#undef BCF_PL1
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

BCF_TRACE_INSTALLER(partition_l1)

}  // namespace bcf
