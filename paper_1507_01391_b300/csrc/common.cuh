// common.cuh -- shared device helpers for libbcf (sm_103a).
//
// Device status word, shared-memory bulk staging (cp.async.bulk + mbarrier) and
// bounded waits.  Every wait in this library has an iteration limit: when it runs
// out the kernel records BCF_DEV_TIMEOUT and carries on, so no launch can hang.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bcf {

// Bits of the device status word (see bcf_get_status()).
enum : unsigned {
  DEV_BAD_KEY = 1u << 0,
  DEV_NOT_BALANCED = 1u << 1,
  DEV_BAD_PERM = 1u << 2,
  DEV_TIMEOUT = 1u << 3,
  DEV_BAD_SEGMENTS = 1u << 4,  // CSR offsets or per-segment w out of range
};

// Polls before a wait gives up (each poll also backs off a little).
constexpr unsigned kSpinLimit = 1u << 24;

__device__ __forceinline__ void set_status(unsigned* status, unsigned bit) {
  atomicOr(status, bit);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- relaxed gpu-scope loads/stores for inter-block flags ----
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t* p) {  // 16-byte aligned
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- mbarrier + bulk copy (the TMA engine's non-tensor form) ----
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (after recording a timeout)
// if the phase never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* status) {
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  set_status(status, DEV_TIMEOUT);
  return false;
}

// Global -> shared bulk copy completed on `bar`.  dst, src and bytes must be
// multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared -> global bulk copy, tracked by the issuing thread's bulk groups.  dst,
// src and bytes must be multiples of 16.  Before the generic proxy's writes to
// the source are visible to the copy, the writers need fence_proxy_async_smem()
// and a barrier.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
// The same with an L2 evict-first hint, for output that no later step of the
// kernel reads.
__device__ __forceinline__ void bulk_s2g_evict_first(void* dst, const void* src, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
      "cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, pol;\n\t}" ::"l"(dst),
      "r"(smem_u32(src)), "r"(bytes)
      : "memory");
}
// Ask L2 to fetch [src, src + bytes) ahead of its use (16-byte aligned, bytes a
// multiple of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_s2g_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until every committed bulk store of this thread has read its source.
__device__ __forceinline__ void bulk_s2g_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int VB>
struct ValT {
  using type = uint32_t;
};
template <>
struct ValT<8> {
  using type = unsigned long long;
};

__host__ __device__ constexpr int ceil_div_i(int a, int b) { return (a + b - 1) / b; }

}  // namespace bcf
