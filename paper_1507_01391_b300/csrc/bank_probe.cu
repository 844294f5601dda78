// bank_probe.cu -- probe kernels for reading a profiler's shared-memory bank
// conflict counters pattern by pattern (trace build only, libbcf_trace.so).
//
// Each probe repeats one shared-memory access pattern of the Lemma 1 tile sort
// (Sec. 2) on the same 64 KB tile it uses (two buffers of 16 x 256 64-bit items,
// item (r, c) at index c*16 + r, so row r lives in bank pair {2r, 2r+1}), alone or
// with global-memory traffic issued between its shared accesses.  A traced copy
// of every probe records its shared accesses (site TS_PROBE) so the bank model of
// Sec. 1 can replay them; the untraced copy touches no global memory except the
// traffic it is asked for and one store of its checksum at the end, so a
// profiler's counters for it belong to the pattern and that traffic alone.
#ifdef BCF_TRACE
#include <cuda_runtime.h>

#include "bcf.h"
#include "bcf_trace.h"
#include "common.cuh"
#include "trace.cuh"

namespace bcf {
namespace {

constexpr int kPrThreads = 256;
constexpr int kPrRows = 16;
constexpr int kPrItems = 4096;
constexpr size_t kPrSmem = 2ull * kPrItems * 8;

template <bool TR>
__device__ __forceinline__ void rec(const void* p, uint32_t width, uint32_t store) {
  if constexpr (TR) trace_access(p, width, store, TS_PROBE);
}

template <bool TR>
__device__ __forceinline__ void block_sync() {
  __syncthreads();
  if constexpr (TR) trace_barrier();
}

__device__ __forceinline__ uint32_t mix(uint32_t x) {
  x *= 0x9E3779B1u;
  return x ^ (x >> 15);
}

// Global traffic issued beside a shared access: a gather from the block's 4096
// words of gin through L1 (traffic 1) or from L2 only (traffic 2), or a streaming
// store of a lane-contiguous word (traffic 3).
template <int G>
__device__ __forceinline__ void beside(const uint32_t* gin, uint32_t* gout, int blk, uint32_t key, uint32_t q,
                                       uint32_t& acc) {
  if constexpr (G == BCF_PROBE_GATHER) acc += gin[(size_t)blk * kPrItems + (mix(key) & (kPrItems - 1))];
  if constexpr (G == BCF_PROBE_GATHER_L2) acc += __ldcg(gin + (size_t)blk * kPrItems + (mix(key) & (kPrItems - 1)));
  if constexpr (G == BCF_PROBE_STORE) gout[(size_t)blk * kPrItems + q] = key;
}

template <int P, int G, bool TR>
__global__ void __launch_bounds__(kPrThreads) k_bank_probe(const uint32_t* __restrict__ gin,
                                                           uint32_t* __restrict__ gout, int reps) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* X = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* Y = X + kPrItems;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, blk = blockIdx.x;
  const int r = lane & 15, tm = warp * 2 + (lane >> 4);  // row, and team member (Lemma 1's row sort)
  for (int q = tid; q < kPrItems; q += kPrThreads) {
    X[q] = ((unsigned long long)mix(q) << 32) | (unsigned)q;
    Y[q] = ((unsigned long long)mix(q + kPrItems) << 32) | (unsigned)q;
  }
  block_sync<TR>();
  uint32_t acc = 0;
#pragma unroll 1
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      if constexpr (P == BCF_PROBE_READOUT) {  // the write-out's read: Y[t], t lane-contiguous
        const int t = tid + i * kPrThreads;
        rec<TR>(&Y[t], 8, 0);
        const unsigned long long v = Y[t];
        acc ^= (uint32_t)v ^ (uint32_t)(v >> 32);
        beside<G>(gin, gout, blk, (uint32_t)v, (uint32_t)t, acc);
      } else if constexpr (P == BCF_PROBE_BUILD) {  // building the items: X[q], q lane-contiguous
        const int q = tid + i * kPrThreads;
        rec<TR>(&X[q], 8, 1);
        X[q] = ((unsigned long long)(acc + rep) << 32) | (unsigned)q;
        beside<G>(gin, gout, blk, (uint32_t)q + rep, (uint32_t)q, acc);
      } else if constexpr (P == BCF_PROBE_ROW_LD) {  // row sort load: 16 items of row r
        const int idx = (tm * 16 + i) * kPrRows + r;
        rec<TR>(&X[idx], 8, 0);
        const unsigned long long v = X[idx];
        acc ^= (uint32_t)v ^ (uint32_t)(v >> 32);
        beside<G>(gin, gout, blk, (uint32_t)v, (uint32_t)(tid + i * kPrThreads), acc);
      } else if constexpr (P == BCF_PROBE_ROW_ST) {  // row sort store, same cells
        const int idx = (tm * 16 + i) * kPrRows + r;
        rec<TR>(&Y[idx], 8, 1);
        Y[idx] = ((unsigned long long)acc << 32) | (unsigned)(idx + rep);
        beside<G>(gin, gout, blk, (uint32_t)idx + rep, (uint32_t)(tid + i * kPrThreads), acc);
      } else if constexpr (P == BCF_PROBE_CONVERT) {  // row-major -> column-major along a diagonal
        const int p = r, R = (p + tm) & 15;
        const int src = (i * 16 + p) * kPrRows + R, dst = (R * 16 + i) * kPrRows + p;
        rec<TR>(&X[src], 8, 0);
        const unsigned long long v = X[src];
        rec<TR>(&Y[dst], 8, 1);
        Y[dst] = v + rep;
        beside<G>(gin, gout, blk, (uint32_t)v, (uint32_t)(tid + i * kPrThreads), acc);
      } else if constexpr (P == BCF_PROBE_MERGE) {  // merge-path search: any column of the lane's own row
        const int col = (int)(mix((uint32_t)(tid * 16 + i) + (uint32_t)rep * 4096u) & 255u);
        rec<TR>(&X[col * kPrRows + r], 8, 0);
        const unsigned long long v = X[col * kPrRows + r];
        acc ^= (uint32_t)v ^ (uint32_t)(v >> 32);
        beside<G>(gin, gout, blk, (uint32_t)v, (uint32_t)(tid + i * kPrThreads), acc);
      } else if constexpr (P == BCF_PROBE_FROM_ROWS) {  // cell (t, 16i + r), t = (r + half-warp) mod 16
        const int t = (r + tm) & 15, c = 16 * ((t & 1) ? 15 - i : i) + r;
        rec<TR>(&X[c * kPrRows + t], 8, 0);
        const unsigned long long v = X[c * kPrRows + t];
        acc ^= (uint32_t)v ^ (uint32_t)(v >> 32);
        beside<G>(gin, gout, blk, (uint32_t)v, (uint32_t)(tid + i * kPrThreads), acc);
      } else if constexpr (P == BCF_PROBE_FROM_COLS) {  // cell ((i + r) mod 16, 16r + t)
        const int t = (r + tm) & 15, idx = (r * 16 + t) * kPrRows + ((i + r) & 15);
        rec<TR>(&X[idx], 8, 0);
        const unsigned long long v = X[idx];
        acc ^= (uint32_t)v ^ (uint32_t)(v >> 32);
        beside<G>(gin, gout, blk, (uint32_t)v, (uint32_t)(tid + i * kPrThreads), acc);
      } else if constexpr (P == BCF_PROBE_READ32) {  // 32-bit lane-contiguous read
        const uint32_t* W = reinterpret_cast<const uint32_t*>(Y);
        const int t = tid + i * kPrThreads;
        rec<TR>(&W[t], 4, 0);
        const uint32_t v = W[t];
        acc ^= v;
        beside<G>(gin, gout, blk, v, (uint32_t)t, acc);
      }
    }
    block_sync<TR>();
  }
  const unsigned long long last = Y[tid] ^ X[tid];
  gout[(size_t)gridDim.x * kPrItems + (size_t)blk * kPrThreads + tid] = acc ^ (uint32_t)last ^ (uint32_t)(last >> 32);
}

using ProbeFn = void (*)(const uint32_t*, uint32_t*, int);

template <int P, int G>
ProbeFn pick(int traced) {
  return traced ? k_bank_probe<P, G, true> : k_bank_probe<P, G, false>;
}

template <int P>
ProbeFn pick_g(int traffic, int traced) {
  switch (traffic) {
    case BCF_PROBE_NONE: return pick<P, BCF_PROBE_NONE>(traced);
    case BCF_PROBE_GATHER: return pick<P, BCF_PROBE_GATHER>(traced);
    case BCF_PROBE_GATHER_L2: return pick<P, BCF_PROBE_GATHER_L2>(traced);
    default: return pick<P, BCF_PROBE_STORE>(traced);
  }
}

ProbeFn pick_probe(int pattern, int traffic, int traced) {
  switch (pattern) {
    case BCF_PROBE_READOUT: return pick_g<BCF_PROBE_READOUT>(traffic, traced);
    case BCF_PROBE_BUILD: return pick_g<BCF_PROBE_BUILD>(traffic, traced);
    case BCF_PROBE_ROW_LD: return pick_g<BCF_PROBE_ROW_LD>(traffic, traced);
    case BCF_PROBE_ROW_ST: return pick_g<BCF_PROBE_ROW_ST>(traffic, traced);
    case BCF_PROBE_CONVERT: return pick_g<BCF_PROBE_CONVERT>(traffic, traced);
    case BCF_PROBE_MERGE: return pick_g<BCF_PROBE_MERGE>(traffic, traced);
    case BCF_PROBE_FROM_ROWS: return pick_g<BCF_PROBE_FROM_ROWS>(traffic, traced);
    case BCF_PROBE_FROM_COLS: return pick_g<BCF_PROBE_FROM_COLS>(traffic, traced);
    default: return pick_g<BCF_PROBE_READ32>(traffic, traced);
  }
}

}  // namespace

BCF_TRACE_INSTALLER(bank_probe)
}  // namespace bcf

extern "C" int bcf_trace_bank_probe(int pattern, int traffic, int traced, const uint32_t* gin, uint32_t* gout,
                                    int blocks, int reps, void* stream) {
  if (pattern < 0 || pattern >= BCF_PROBE_PATTERNS || traffic < 0 || traffic >= BCF_PROBE_TRAFFICS)
    return BCF_E_INVAL;
  if (!gin || !gout || blocks < 1 || blocks > 65535 || reps < 1) return BCF_E_INVAL;
  const bcf::ProbeFn k = bcf::pick_probe(pattern, traffic, traced);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bcf::kPrSmem) != cudaSuccess)
    return BCF_E_CUDA;
  k<<<(unsigned)blocks, bcf::kPrThreads, bcf::kPrSmem, static_cast<cudaStream_t>(stream)>>>(gin, gout, reps);
  return cudaGetLastError() == cudaSuccess ? BCF_OK : BCF_E_CUDA;
}
#endif
