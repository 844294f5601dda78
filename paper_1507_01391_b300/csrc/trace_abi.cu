// trace_abi.cu -- C entry points of the shared-memory access trace (libbcf_trace.so).
//
// Compiled only into the trace build (-DBCF_TRACE); the product library has no
// tracing code.  Declared in include/bcf_trace.h.
#ifdef BCF_TRACE
#include <cuda_runtime.h>

#include "bcf.h"
#include "bcf_trace.h"
#include "trace.cuh"

namespace bcf {
cudaError_t trace_install_radix(const TraceState& t);
cudaError_t trace_install_segmented(const TraceState& t);
cudaError_t trace_install_tile_permute(const TraceState& t);
cudaError_t trace_install_partition_l1(const TraceState& t);
cudaError_t trace_install_partition_l2(const TraceState& t);
cudaError_t trace_install_bank_probe(const TraceState& t);
}  // namespace bcf

namespace {
unsigned long long* g_count = nullptr;

int install(const bcf::TraceState& t) {
  if (bcf::trace_install_radix(t) != cudaSuccess) return BCF_E_CUDA;
  if (bcf::trace_install_segmented(t) != cudaSuccess) return BCF_E_CUDA;
  if (bcf::trace_install_tile_permute(t) != cudaSuccess) return BCF_E_CUDA;
  if (bcf::trace_install_partition_l1(t) != cudaSuccess) return BCF_E_CUDA;
  if (bcf::trace_install_partition_l2(t) != cudaSuccess) return BCF_E_CUDA;
  if (bcf::trace_install_bank_probe(t) != cudaSuccess) return BCF_E_CUDA;
  return BCF_OK;
}
}  // namespace

extern "C" int bcf_trace_begin(void* buf, size_t buf_bytes) {
  if (!buf || (reinterpret_cast<uintptr_t>(buf) & 15u) || buf_bytes < 32) return BCF_E_INVAL;
  if (cudaMemset(buf, 0, 16) != cudaSuccess) return BCF_E_CUDA;
  bcf::TraceState t;
  t.count = static_cast<unsigned long long*>(buf);
  t.rec = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(buf) + 16);
  t.cap = (buf_bytes - 16) / 16;
  g_count = t.count;
  return install(t);
}

extern "C" int bcf_trace_end(uint64_t* records) {
  if (!records || !g_count) return BCF_E_INVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return BCF_E_CUDA;
  unsigned long long n = 0;
  if (cudaMemcpy(&n, g_count, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess) return BCF_E_CUDA;
  *records = n;
  bcf::TraceState off;
  off.count = nullptr;
  off.rec = nullptr;
  off.cap = 0;
  g_count = nullptr;
  return install(off);
}
#endif
