// internal.h -- host-side interfaces between the C ABI (abi.cu) and the kernel
// translation units.  Not installed; the public interface is include/bcf.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace bcf {

// Device status word of the current device (a module variable in abi.cu).
unsigned* status_word();

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- digit sweeps
constexpr int kSweepThreads = 256;
constexpr int kSweepIPT = 16;
constexpr int kSweepTile = kSweepThreads * kSweepIPT;  // keys per tile

struct PassPlan {
  int passes = 0;
  int shift[4] = {0, 0, 0, 0};
  int nbits[4] = {0, 0, 0, 0};
};
PassPlan plan_passes(int key_bits);

// Workspace carve-up of a radix sort / partition.
struct SweepLayout {
  size_t keys_tmp = 0, vals_tmp = 0;   // ping-pong buffers (0 bytes when unused)
  size_t zero_begin = 0, zero_bytes = 0;  // region cleared before the passes
  size_t hist = 0, counters = 0, lookback = 0, digit_base = 0;
  size_t total = 0;
  int64_t tiles = 0;
  int radix = 256;
};
SweepLayout sweep_layout(int64_t n, int val_bytes, int passes, int radix, bool need_tmp);

// Radix sort launch sequence (see bcf_sort in include/bcf.h).
cudaError_t radix_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n, int val_bytes, const PassPlan& plan,
                       unsigned char* ws, const SweepLayout& L, cudaStream_t s);

// Single-pass stable partition by label (see bcf_partition).
cudaError_t partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                      void* vals_out, int64_t n, int w, int val_bytes, bool balanced,
                      unsigned char* ws, const SweepLayout& L, cudaStream_t s);

// ---------------------------------------------------------------- permutations
cudaError_t permute(const void* src_k, const void* src_v, void* dst_k, void* dst_v,
                    const uint32_t* pi, int64_t n, int kbytes, int vbytes,
                    uint32_t* seen_bitmap, cudaStream_t s);
cudaError_t gather(const void* src, void* dst, const uint32_t* idx, int64_t n, int64_t n_src,
                   int elem_bytes, cudaStream_t s);
cudaError_t permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi, int64_t n,
                          int tile, bool coloured, uint64_t seed, cudaStream_t s);

}  // namespace bcf
