// noalloc.cu -- bcf_partition_noalloc: the w-way partition with its scratch in a
// fixed device array instead of a caller workspace.
//
// Who needs it: callers that cannot allocate device memory when they call us --
// code running inside CUDA stream capture (cudaMalloc is not allowed while a
// global-mode capture is active), plugins living inside a host framework that
// owns all device memory through its own pool, and latency-critical loops that
// must never enter the driver's allocator.  They still pass their own inputs and
// outputs; only the scratch (per-tile label counts and label totals) moves here.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes (about
// 1 MiB), enough for n <= kNoAllocMaxN keys.  Every device that loads libbcf.so
// holds it until the process exits.  All calls share it and it keeps the last
// call's contents: the part that must start at zero is cleared on the stream by
// every call, and two calls whose work overlaps on the GPU (different streams,
// no ordering between them) race on it.
#include <cuda_runtime.h>

#include <atomic>

#include "bcf.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int64_t kNoAllocMaxN = BCF_NOALLOC_MAX_N;
// Largest workspace the partition needs without an in-place copy, reached at
// kNoAllocMaxN keys: label starts and label totals (4 x 256 words each, 256-byte
// aligned), the tile tickets (256 bytes) and 256 x tiles counts.  (Inputs small
// enough for the single-launch look-back path add status words instead, far fewer.)
constexpr size_t kNoAllocTiles = (size_t)((kNoAllocMaxN + bcf::kSweepTile - 1) / bcf::kSweepTile);
constexpr size_t kNoAllocStride =
    (kNoAllocTiles + bcf::kLookbackWindow) / bcf::kLookbackWindow * bcf::kLookbackWindow;
constexpr size_t kNoAllocScratchBytes = 2 * 4 * 256 * 4 + 256 + kNoAllocStride * 256 * 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name only stands for the symbol; the address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.  The
// per-device cache is atomic: host threads that make their first call at the same
// time may each look the address up, and they store the same value.
unsigned char* scratch_address(int* rc) {
  static std::atomic<unsigned char*> addr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *rc = BCF_E_CUDA;
    return nullptr;
  }
  unsigned char* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      *rc = BCF_E_CUDA;
      return nullptr;
    }
    a = static_cast<unsigned char*>(p);
    addr[dev].store(a, std::memory_order_release);
  }
  *rc = BCF_OK;
  return a;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool disjoint(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return na == 0 || nb == 0 || x + na <= y || y + nb <= x;
}

}  // namespace

extern "C" int bcf_partition_noalloc(const uint32_t* keys_in, const void* vals_in,
                                     uint32_t* keys_out, void* vals_out, int64_t n, int w,
                                     int val_bytes, int flags, bcf_stream_t stream) {
  if (n < 0 || w < 1 || (val_bytes != 0 && val_bytes != 4 && val_bytes != 8)) return BCF_E_INVAL;
  if (n > kNoAllocMaxN || w > 256) return BCF_E_UNSUPPORTED;
  if (flags & ~BCF_ASSUME_BALANCED) return BCF_E_UNSUPPORTED;  // e.g. BCF_PARTITION_LEMMA1
  const bool balanced = (flags & BCF_ASSUME_BALANCED) != 0;
  if (balanced && n % w) return BCF_E_INVAL;
  if (n == 0) return BCF_OK;
  if (!keys_in || !keys_out || !aligned16(keys_in) || !aligned16(keys_out)) return BCF_E_INVAL;
  const bool iota = (val_bytes == 4 && !vals_in);
  if (val_bytes && (!vals_out || !aligned16(vals_out) || (!iota && (!vals_in || !aligned16(vals_in)))))
    return BCF_E_INVAL;
  if (!val_bytes && (vals_in || vals_out)) return BCF_E_INVAL;
  // out of place only: the in-place form needs a copy of the input
  if (!disjoint(keys_in, (size_t)n * 4, keys_out, (size_t)n * 4)) return BCF_E_INVAL;
  if (val_bytes && !iota && !disjoint(vals_in, (size_t)n * val_bytes, vals_out, (size_t)n * val_bytes))
    return BCF_E_INVAL;
  const bcf::SweepLayout L = bcf::sweep_layout(n, val_bytes, 1, w <= 32 ? 32 : 256, false, bcf::kSweepTile, false);
  if (L.total > kNoAllocScratchBytes) return BCF_E_UNSUPPORTED;
  int rc = BCF_OK;
  unsigned char* scratch = scratch_address(&rc);
  if (rc != BCF_OK) return rc;
  if (!bcf::status_word()) return BCF_E_CUDA;
  // bcf::partition clears the counters it needs on `stream` before using them.
  const cudaError_t e = bcf::partition(keys_in, vals_in, keys_out, vals_out, n, w, val_bytes, balanced,
                                       scratch, L, (cudaStream_t)stream, bcf::kRtsCfg0);
  return e == cudaSuccess ? BCF_OK : BCF_E_CUDA;
}
