// trace.cuh -- optional shared-memory access tracing (builds with -DBCF_TRACE).
//
// In a trace build every instrumented shared-memory access appends one record per
// active lane to a caller-provided device buffer: (request id, thread index |
// block index << 16, shared-window byte address, width | store << 8 | site << 16),
// and every barrier taken through BCF_SYNC() (block-wide) or BCF_SYNCWARP()
// (warp-wide) one record per warp.  All lanes of one warp-wide access share the
// request id, so the trace can be replayed through the bank model of Sec. 1 (32
// banks of 4-byte words; a request conflicts when two of its lanes need different
// words of one bank).  Without BCF_TRACE the macro is empty and the kernels are
// unchanged.
#pragma once

#include "common.cuh"

namespace bcf {

// Access sites (the `site` field of a record).
enum TraceSite : uint32_t {
  TS_STAGE_READ = 1,    // strided read of a staged tile into registers
  TS_COUNT_ATOM = 2,    // per-warp digit count
  TS_CLAIM_ATOM = 3,    // leader claims a digit run
  TS_SCATTER = 4,       // store into digit / label order
  TS_WRITEOUT_READ = 5, // read of the ordered tile for the global write-out
  TS_OFFSET_READ = 6,   // per-digit offset lookup
  TS_HIST_ATOM = 7,     // one-read histogram: lane-private digit count
  TS_HIST_SUM = 8,      // one-read histogram: diagonal sum of the lane counters
  TS_WARP_OFFSETS = 9,  // per-(warp, digit) count row read / rewritten as offsets
  TS_TILE_COUNT_ATOM = 14,  // per-tile counts: lane-private byte counters
  TS_TILE_COUNT_SUM = 15,   // per-tile counts: diagonal sum of the lane words
  TS_L1_ROW_LD = 10,    // Lemma 1: row sort loads (register sort and merges)
  TS_L1_ROW_ST = 11,    // Lemma 1: row sort stores
  TS_L1_CONVERT = 12,   // Lemma 1: row <-> column conversions
  TS_L1_IO = 13,        // Lemma 1: building the items / final read
  TS_COL_TABLE = 20,    // colouring: table reset / claims
  TS_COL_SEND = 21,     // colouring: conflict-free sends
  TS_COL_READ = 22,     // colouring: reading own row (labels, items)
  TS_COL_FINISH = 23,   // colouring: finishing sends (greedy or sorted)
  TS_COL_PACK = 24,     // colouring, sorted finish: ordering and packing the leftovers
  TS_L2_SQUARE = 40,    // Lemma 2: balancing round 0 (column-major square sorts)
  TS_L2_CONVERT = 41,   // Lemma 2: balancing round 1 composed with the conversion
  TS_L2_DIVIDE = 42,    // Lemma 2: 8-row sub-problems sorted row-major
  TS_L2_COLUMN = 43,    // Lemma 2: column sorts (counts and moves)
  TS_L2_ROWS = 44,      // Lemma 2: squares of 32 contiguous rows, row-major
  TS_L2_SHIFTED = 45,   // Lemma 2: the same squares shifted down by 16 rows
  TS_L2_IO = 47,        // Lemma 2: the padded row-major write-out copy
  TS_BARRIER = 30,      // a barrier (one record per warp; store field 3 block-wide, 4 warp-wide)
  TS_PROBE = 50,        // the bank-conflict probe kernels
};

#ifdef BCF_TRACE
struct TraceState {
  unsigned long long* count;  // records written so far (may exceed cap)
  uint32_t* rec;              // 4 words per record
  unsigned long long cap;     // records that fit
};
// One copy per translation unit (no relocatable device code); each unit that
// includes this header installs its copy through BCF_TRACE_INSTALLER.
static __device__ TraceState g_bcf_trace;
#define BCF_TRACE_INSTALLER(name)                                        \
  cudaError_t trace_install_##name(const ::bcf::TraceState& t) {         \
    return cudaMemcpyToSymbol(::bcf::g_bcf_trace, &t, sizeof(t));       \
  }

__device__ __forceinline__ void trace_access(const void* p, uint32_t width, uint32_t store,
                                             uint32_t site) {
  const TraceState t = g_bcf_trace;
  if (!t.count) return;
  const unsigned mask = __activemask();
  const int lane = (int)(threadIdx.x & 31u);
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(t.count, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  const unsigned long long r = base + (unsigned long long)__popc(mask & lanemask_lt());
  if (r < t.cap) {
    uint32_t* o = t.rec + 4 * r;
    o[0] = (uint32_t)base;
    o[1] = (uint32_t)threadIdx.x | ((uint32_t)blockIdx.x << 16);
    o[2] = smem_u32(p);
    o[3] = width | (store << 8) | (site << 16);
  }
}

// After a block-wide barrier every warp appends one barrier record (store field 3),
// and after a warp-wide barrier the warp appends one (store field 4), so a replay
// can split each warp's accesses into the segments between barriers.
__device__ __forceinline__ void trace_barrier(uint32_t kind = 3u) {
  const TraceState t = g_bcf_trace;
  if (!t.count || (threadIdx.x & 31u) != (uint32_t)(__ffs(__activemask()) - 1)) return;
  const unsigned long long r = atomicAdd(t.count, 1ull);
  if (r < t.cap) {
    uint32_t* o = t.rec + 4 * r;
    o[0] = (uint32_t)r;
    o[1] = (uint32_t)threadIdx.x | ((uint32_t)blockIdx.x << 16);
    o[2] = 0;
    o[3] = 0u | (kind << 8) | ((uint32_t)TS_BARRIER << 16);
  }
}
#define BCF_TR(ptr, width, store, site) ::bcf::trace_access((ptr), (width), (store), (site))
#define BCF_SYNC()               \
  do {                           \
    __syncthreads();             \
    ::bcf::trace_barrier();      \
  } while (0)
#define BCF_SYNCWARP()           \
  do {                           \
    __syncwarp();                \
    ::bcf::trace_barrier(4u);    \
  } while (0)
#else
#define BCF_TR(ptr, width, store, site) ((void)0)
#define BCF_TRACE_INSTALLER(name)
#define BCF_SYNC() __syncthreads()
#define BCF_SYNCWARP() __syncwarp()
#endif
// Sub-word accesses are traced as the 4-byte word that holds them.
#define BCF_TR_WORD(ptr, store, site) \
  BCF_TR(reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(ptr) & ~(uintptr_t)3), 4, (store), (site))

}  // namespace bcf
