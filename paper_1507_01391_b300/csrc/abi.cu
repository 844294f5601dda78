// abi.cu -- extern "C" entry points of libbcf.so (declared in include/bcf.h).
//
// Argument checking, workspace carving and launch sequencing only; all data work
// happens in the kernels of radix.cu, permute.cu, tile_permute.cu, tile_sort.cu and
// segmented.cu.  No entry point allocates device memory.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "bcf.h"
#include "common.cuh"
#include "internal.h"

// Device status word: bits of bcf::DEV_* OR-ed in by kernels.
static __device__ unsigned g_bcf_status;

namespace bcf {

unsigned* status_word() {
  // Cached per device; cudaGetSymbolAddress only looks the address up.
  static unsigned* addr[64] = {nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bcf_status) == cudaSuccess) addr[dev] = static_cast<unsigned*>(p);
  }
  return addr[dev];
}

}  // namespace bcf

namespace {

constexpr int64_t kMaxSweepN = (int64_t)1 << 30;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool valid_vb(int vb) { return vb == 0 || vb == 4 || vb == 8; }

// [a, a+na) and [b, b+nb) either coincide exactly or do not overlap at all.
bool same_or_disjoint(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  if (x == y) return true;
  return x + na <= y || y + nb <= x;
}
bool disjoint(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return na == 0 || nb == 0 || x + na <= y || y + nb <= x;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? BCF_OK : BCF_E_CUDA; }

// Kernels record errors through the status word; without its address (no usable
// device) nothing may be launched.
bool device_ready() { return bcf::status_word() != nullptr; }

int check_kv(const uint32_t* ki, const void* vi, const uint32_t* ko, const void* vo, int64_t n,
             int vb) {
  if (n < 0 || !valid_vb(vb)) return BCF_E_INVAL;
  if (n == 0) return BCF_OK;
  if (!ki || !ko || !aligned16(ki) || !aligned16(ko)) return BCF_E_INVAL;
  // vi == NULL with 4-byte payloads: index payload (item i carries i)
  const bool iota = (vb == 4 && !vi);
  if (vb && (!vo || !aligned16(vo) || (!iota && (!vi || !aligned16(vi))))) return BCF_E_INVAL;
  if (!vb && (vi || vo)) return BCF_E_INVAL;
  const size_t kb = (size_t)n * 4, vbb = (size_t)n * vb;
  if (!same_or_disjoint(ki, kb, ko, kb)) return BCF_E_INVAL;
  if (vb && !iota && !same_or_disjoint(vi, vbb, vo, vbb)) return BCF_E_INVAL;
  if (vb && !iota && ((ki == ko) != (vi == vo))) return BCF_E_INVAL;  // both in place or neither
  return BCF_OK;
}

}  // namespace

extern "C" {

const char* bcf_status_string(int status) {
  switch (status) {
    case BCF_OK: return "ok";
    case BCF_E_INVAL: return "invalid argument (null pointer, size, width, alignment or overlap)";
    case BCF_E_WORKSPACE: return "workspace smaller than the *_workspace_size() result";
    case BCF_E_UNSUPPORTED: return "request outside what the library supports";
    case BCF_E_CUDA: return "a CUDA launch or copy failed";
    case BCF_E_TIMEOUT: return "a bounded inter-block wait gave up on the device";
    case BCF_E_NOT_BALANCED: return "balanced partition: a label count differs from n/w";
    case BCF_E_BAD_PERM: return "permutation index out of range or repeated";
    case BCF_E_BAD_KEY: return "partition label >= w";
  }
  return "unknown status";
}

int bcf_version(void) { return 10000 * 1 + 100 * 0 + 0; }

int bcf_get_status(bcf_stream_t stream, int* out) {
  if (!out) return BCF_E_INVAL;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BCF_E_CUDA;
  unsigned bits = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&bits, g_bcf_status, sizeof(bits)) != cudaSuccess) return BCF_E_CUDA;
  if (bits && cudaMemcpyToSymbol(g_bcf_status, &zero, sizeof(zero)) != cudaSuccess) return BCF_E_CUDA;
  if (bits & bcf::DEV_TIMEOUT) *out = BCF_E_TIMEOUT;
  else if (bits & bcf::DEV_BAD_SEGMENTS) *out = BCF_E_INVAL;
  else if (bits & bcf::DEV_BAD_PERM) *out = BCF_E_BAD_PERM;
  else if (bits & bcf::DEV_NOT_BALANCED) *out = BCF_E_NOT_BALANCED;
  else if (bits & bcf::DEV_BAD_KEY) *out = BCF_E_BAD_KEY;
  else *out = BCF_OK;
  return BCF_OK;
}

// ------------------------------------------------------------------ sort
int bcf_sort_workspace_size(int64_t n, int val_bytes, int key_bits, size_t* bytes) {
  if (!bytes || n < 0 || !valid_vb(val_bytes) || key_bits < 1 || key_bits > 32) return BCF_E_INVAL;
  if (n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  const bcf::PassPlan pl = bcf::plan_passes(key_bits);
  *bytes = bcf::sweep_layout(n, val_bytes, pl.passes, 256, true).total;
  return BCF_OK;
}

int bcf_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out, void* vals_out,
             int64_t n, int val_bytes, int key_bits, void* ws, size_t ws_bytes,
             bcf_stream_t stream) {
  int rc = check_kv(keys_in, vals_in, keys_out, vals_out, n, val_bytes);
  if (rc) return rc;
  if (key_bits < 1 || key_bits > 32) return BCF_E_INVAL;
  if (n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  if (n == 0) return BCF_OK;
  const bcf::PassPlan pl = bcf::plan_passes(key_bits);
  const bcf::SweepLayout L = bcf::sweep_layout(n, val_bytes, pl.passes, 256, true);
  if (!ws || !aligned16(ws)) return BCF_E_INVAL;
  if (ws_bytes < L.total) return BCF_E_WORKSPACE;
  if (!disjoint(ws, ws_bytes, keys_in, (size_t)n * 4) || !disjoint(ws, ws_bytes, keys_out, (size_t)n * 4))
    return BCF_E_INVAL;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::radix_sort(keys_in, vals_in, keys_out, vals_out, n, val_bytes, pl,
                                 static_cast<unsigned char*>(ws), L, (cudaStream_t)stream,
                                 bcf::tuned_config(BCF_OP_SORT, n)));
}

int bcf_sort_passes_run(const void* ws, int64_t n, int val_bytes, int key_bits, int* passes,
                        bcf_stream_t stream) {
  if (!ws || !passes || n < 0 || !valid_vb(val_bytes) || key_bits < 1 || key_bits > 32) return BCF_E_INVAL;
  if (n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  *passes = 0;
  if (n == 0) return BCF_OK;
  if (!device_ready()) return BCF_E_CUDA;
  const bcf::PassPlan pl = bcf::plan_passes(key_bits);
  const bcf::SweepLayout L = bcf::sweep_layout(n, val_bytes, pl.passes, 256, true);
  return bcf::sort_passes_run(static_cast<const unsigned char*>(ws), L, pl, (cudaStream_t)stream, passes) == 0
             ? BCF_OK
             : BCF_E_CUDA;
}

// ------------------------------------------------------------- partition
static bcf::SweepLayout partition_layout(int64_t n, int w, int vb) {
  return bcf::sweep_layout(n, vb, 1, w <= 32 ? 32 : 256, true);
}

int bcf_partition_workspace_size(int64_t n, int w, int val_bytes, int flags, size_t* bytes) {
  if (!bytes || n < 0 || w < 1 || !valid_vb(val_bytes)) return BCF_E_INVAL;
  if (w > 256 || n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  *bytes = partition_layout(n, w, val_bytes).total;
  if (flags & BCF_PARTITION_LEMMA1) {
    const size_t l1 = bcf::sweep_layout(n, val_bytes, 1, 256, true).total;
    if (l1 > *bytes) *bytes = l1;
  }
  return BCF_OK;
}

int bcf_partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                  void* vals_out, int64_t n, int w, int val_bytes, int flags, void* ws,
                  size_t ws_bytes, bcf_stream_t stream) {
  int rc = check_kv(keys_in, vals_in, keys_out, vals_out, n, val_bytes);
  if (rc) return rc;
  if (w < 1) return BCF_E_INVAL;
  if (w > 256 || n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  if ((flags & BCF_PARTITION_DIRECT) && (w > 32 || (flags & BCF_PARTITION_LEMMA1))) return BCF_E_UNSUPPORTED;
  const bool balanced = (flags & BCF_ASSUME_BALANCED) != 0;
  if (balanced && n % w) return BCF_E_INVAL;
  if (n == 0) return BCF_OK;
  const bcf::SweepLayout L = partition_layout(n, w, val_bytes);
  if (!ws || !aligned16(ws)) return BCF_E_INVAL;
  if (ws_bytes < L.total) return BCF_E_WORKSPACE;
  if (flags & BCF_PARTITION_LEMMA1) {
    if (!device_ready()) return BCF_E_CUDA;
    // 256-label counts at 4096-key tiles fit the workspace sized for the sweeps
    const bcf::SweepLayout L1 = bcf::sweep_layout(n, val_bytes, 1, 256, true);
    if (ws_bytes < L1.total) return BCF_E_WORKSPACE;
    return cuda_rc(bcf::partition_lemma1(keys_in, vals_in, keys_out, vals_out, n, w, val_bytes, balanced,
                                         static_cast<unsigned char*>(ws), L1, (cudaStream_t)stream));
  }
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::partition(keys_in, vals_in, keys_out, vals_out, n, w, val_bytes, balanced,
                                static_cast<unsigned char*>(ws), L, (cudaStream_t)stream,
                                bcf::tuned_config(BCF_OP_PARTITION, n), (flags & BCF_PARTITION_DIRECT) != 0));
}

// Splitter partition: the sweep layout of a 256-bucket partition, always with
// room for an in-place copy and for the reduce-then-scan counts at any size,
// plus one byte per key for the buckets and the splitter search's prefix table.
static bcf::SweepLayout splitter_layout(int64_t n, int val_bytes) {
  bcf::SweepLayout L = bcf::sweep_layout(n, val_bytes, 1, 256, true, bcf::kMinSweepTile, false);
  L.labels = L.total;  // each key's bucket, kept by the tile counts for the sweep
  L.split_table = bcf::align_up(L.total + (size_t)n);
  L.total = bcf::align_up(L.split_table + (size_t)bcf::kSplitPrefixes * 2 + 8);  // 16 bits per prefix, window
  return L;
}

int bcf_partition_splitters_workspace_size(int64_t n, int nsplit, int val_bytes, int flags, size_t* bytes) {
  (void)flags;
  if (!bytes || n < 0 || nsplit < 0 || !valid_vb(val_bytes)) return BCF_E_INVAL;
  if (nsplit > 255 || n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  *bytes = splitter_layout(n, val_bytes).total;
  return BCF_OK;
}

int bcf_partition_splitters(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                            void* vals_out, int64_t n, const uint32_t* splitters, int nsplit,
                            int val_bytes, int flags, void* ws, size_t ws_bytes, bcf_stream_t stream) {
  int rc = check_kv(keys_in, vals_in, keys_out, vals_out, n, val_bytes);
  if (rc) return rc;
  if (nsplit < 0 || (nsplit > 0 && !splitters)) return BCF_E_INVAL;
  if (nsplit > 255 || n >= kMaxSweepN) return BCF_E_UNSUPPORTED;
  const bool balanced = (flags & BCF_ASSUME_BALANCED) != 0;
  if (balanced && n % (nsplit + 1)) return BCF_E_INVAL;
  if (n == 0) return BCF_OK;
  const bcf::SweepLayout L = splitter_layout(n, val_bytes);
  if (!ws || !aligned16(ws)) return BCF_E_INVAL;
  if (ws_bytes < L.total) return BCF_E_WORKSPACE;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::partition_splitters(keys_in, vals_in, keys_out, vals_out, n, splitters, nsplit, val_bytes,
                                          balanced, static_cast<unsigned char*>(ws), L, (cudaStream_t)stream));
}

// ------------------------------------------------------------ permutations
// Workspace: [bucketed-form region (BCF_PERMUTE_BUCKETED)][seen bitmap (BCF_CHECK_PERM)].
static size_t permute_bucket_bytes(int64_t n, int vb, int flags) {
  return ((flags & BCF_PERMUTE_BUCKETED) && bcf::permute_bucketed_supported(n, 4, vb))
             ? bcf::permute_bucketed_workspace(n, vb)
             : 0;
}

int bcf_permute_workspace_size(int64_t n, int val_bytes, int flags, size_t* bytes) {
  if (!bytes || n < 0 || !valid_vb(val_bytes)) return BCF_E_INVAL;
  *bytes = permute_bucket_bytes(n, val_bytes, flags) +
           ((flags & BCF_CHECK_PERM) ? bcf::align_up((size_t)((n + 31) / 32) * 4) : 0);
  return BCF_OK;
}

static int permute_common(const void* sk, const void* sv, void* dk, void* dv, const uint32_t* pi,
                          int64_t n, int64_t row_len, int kb, int vb, int flags, void* ws,
                          size_t ws_bytes, cudaStream_t s) {
  if (n < 0 || row_len < 0 || (kb != 4 && kb != 8) || !valid_vb(vb)) return BCF_E_INVAL;
  if (n > (int64_t)0xFFFFFFFFLL) return BCF_E_UNSUPPORTED;
  if (n == 0) return BCF_OK;
  if (!sk || !dk || !pi || !aligned16(sk) || !aligned16(dk) || !aligned16(pi)) return BCF_E_INVAL;
  if (vb && (!sv || !dv || !aligned16(sv) || !aligned16(dv))) return BCF_E_INVAL;
  if (!disjoint(sk, (size_t)n * kb, dk, (size_t)n * kb)) return BCF_E_INVAL;
  if (vb && !disjoint(sv, (size_t)n * vb, dv, (size_t)n * vb)) return BCF_E_INVAL;
  // bcf_permute sizes its workspace with val_bytes 0 whatever its element size
  const int ws_vb = sv ? vb : 0;
  size_t need = 0;
  bcf_permute_workspace_size(n, ws_vb, flags, &need);
  if (need) {
    if (!ws || !aligned16(ws)) return BCF_E_INVAL;
    if (ws_bytes < need) return BCF_E_WORKSPACE;
  }
  const size_t bucket_bytes = permute_bucket_bytes(n, ws_vb, flags);
  const bool check = (flags & BCF_CHECK_PERM) != 0;
  if (!device_ready()) return BCF_E_CUDA;
  if ((flags & BCF_PERMUTE_BUCKETED) && bcf::permute_bucketed_supported(n, kb, vb))
    return cuda_rc(bcf::permute_bucketed(static_cast<const uint32_t*>(sk), static_cast<const uint32_t*>(sv),
                                         static_cast<uint32_t*>(dk), static_cast<uint32_t*>(dv), pi, n,
                                         row_len, vb, check, static_cast<unsigned char*>(ws), s));
  uint32_t* seen = check ? reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ws) + bucket_bytes) : nullptr;
  return cuda_rc(bcf::permute(sk, sv, dk, dv, pi, n, row_len, kb, vb, seen,
                              (flags & BCF_PERMUTE_FUSED) != 0, s));
}

int bcf_permute(const void* src, void* dst, const uint32_t* pi, int64_t n, int64_t row_len,
                int elem_bytes, int flags, void* ws, size_t ws_bytes, bcf_stream_t stream) {
  return permute_common(src, nullptr, dst, nullptr, pi, n, row_len, elem_bytes, 0, flags, ws,
                        ws_bytes, (cudaStream_t)stream);
}

int bcf_permute_kv(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                   const uint32_t* pi, int64_t n, int64_t row_len, int val_bytes, int flags,
                   void* ws, size_t ws_bytes, bcf_stream_t stream) {
  if (!val_bytes && (src_v || dst_v)) return BCF_E_INVAL;
  return permute_common(src_k, src_v, dst_k, dst_v, pi, n, row_len, 4, val_bytes, flags, ws,
                        ws_bytes, (cudaStream_t)stream);
}

int bcf_permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi, int64_t n,
                      int tile, int flags, uint64_t seed, bcf_stream_t stream) {
  if (n < 0 || (tile != 1024 && tile != 2048 && tile != 4096)) return BCF_E_INVAL;
  if (n >= ((int64_t)1 << 40)) return BCF_E_UNSUPPORTED;
  if (n == 0) return BCF_OK;
  if (!src || !dst || !lpi || !aligned16(src) || !aligned16(dst) || !aligned16(lpi)) return BCF_E_INVAL;
  if (!disjoint(src, (size_t)n * 4, dst, (size_t)n * 4)) return BCF_E_INVAL;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::permute_tiles(src, dst, lpi, n, tile, (flags & BCF_TILES_COLOURED) != 0,
                                    (flags & BCF_TILES_SORTED_FINISH) != 0,
                                    seed, (cudaStream_t)stream));
}

int bcf_gather(const void* src, void* dst, const uint32_t* idx, int64_t n, int64_t n_src,
               int64_t row_len, int elem_bytes, bcf_stream_t stream) {
  if (n < 0 || n_src < 0 || row_len < 0 || (elem_bytes != 4 && elem_bytes != 8)) return BCF_E_INVAL;
  if (n_src > (int64_t)0xFFFFFFFFLL) return BCF_E_UNSUPPORTED;
  if (n == 0) return BCF_OK;
  if (!dst || !idx || !aligned16(dst) || !aligned16(idx)) return BCF_E_INVAL;
  if (n_src > 0 && !src) return BCF_E_INVAL;
  if (!disjoint(src, (size_t)n_src * elem_bytes, dst, (size_t)n * elem_bytes)) return BCF_E_INVAL;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::gather(src, dst, idx, n, n_src, row_len, elem_bytes, (cudaStream_t)stream));
}

// ------------------------------------------------------- tiles / segments
int bcf_sort_tiles(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                   void* vals_out, int64_t n, int tile, int val_bytes, bcf_stream_t stream) {
  if (tile != 4096) return BCF_E_INVAL;
  int rc = check_kv(keys_in, vals_in, keys_out, vals_out, n, val_bytes);
  if (rc) return rc;
  if (n >= ((int64_t)1 << 40)) return BCF_E_UNSUPPORTED;
  if (n == 0) return BCF_OK;
  if (!disjoint(keys_in, (size_t)n * 4, keys_out, (size_t)n * 4)) return BCF_E_INVAL;
  if (val_bytes && !disjoint(vals_in, (size_t)n * val_bytes, vals_out, (size_t)n * val_bytes))
    return BCF_E_INVAL;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::sort_tiles(keys_in, vals_in, keys_out, vals_out, n, val_bytes, (cudaStream_t)stream));
}

int bcf_partition_lemma2(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                         uint32_t* vals_out, int64_t n, bcf_stream_t stream) {
  if (n < 0 || n % 32768 != 0) return BCF_E_INVAL;
  if (n >= ((int64_t)1 << 32)) return BCF_E_UNSUPPORTED;
  int rc = check_kv(keys_in, vals_in, keys_out, vals_out, n, 4);
  if (rc) return rc;
  if (n == 0) return BCF_OK;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::partition_lemma2(keys_in, vals_in, keys_out, vals_out, n, (cudaStream_t)stream));
}

static int check_segments(const uint32_t* ki, const void* vi, const uint32_t* ko, const void* vo,
                          int64_t n_total, const int64_t* offs, int64_t nseg, int vb) {
  int rc = check_kv(ki, vi, ko, vo, n_total, vb);
  if (rc) return rc;
  if (nseg < 0) return BCF_E_INVAL;
  if (n_total >= kMaxSweepN || nseg >= ((int64_t)1 << 31)) return BCF_E_UNSUPPORTED;
  if (nseg > 0 && (!offs || (reinterpret_cast<uintptr_t>(offs) & 7u))) return BCF_E_INVAL;
  if (n_total > 0 && nseg == 0) return BCF_E_INVAL;
  if (n_total > 0) {
    if (!disjoint(ki, (size_t)n_total * 4, ko, (size_t)n_total * 4)) return BCF_E_INVAL;
    if (vb && !disjoint(vi, (size_t)n_total * vb, vo, (size_t)n_total * vb)) return BCF_E_INVAL;
  }
  return BCF_OK;
}

int bcf_segmented_sort_workspace_size(int64_t n_total, int64_t nseg, int val_bytes, int key_bits,
                                      size_t* bytes) {
  if (!bytes || n_total < 0 || nseg < 0 || !valid_vb(val_bytes) || key_bits < 1 || key_bits > 32)
    return BCF_E_INVAL;
  if (n_total >= kMaxSweepN || nseg >= ((int64_t)1 << 31)) return BCF_E_UNSUPPORTED;
  *bytes = bcf::seg_layout(n_total, nseg, val_bytes, bcf::plan_passes(key_bits).passes, true).total;
  return BCF_OK;
}

int bcf_segmented_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n_total, const int64_t* offs, int64_t nseg,
                       int val_bytes, int key_bits, void* ws, size_t ws_bytes,
                       bcf_stream_t stream) {
  int rc = check_segments(keys_in, vals_in, keys_out, vals_out, n_total, offs, nseg, val_bytes);
  if (rc) return rc;
  if (key_bits < 1 || key_bits > 32) return BCF_E_INVAL;
  if (nseg == 0) return BCF_OK;
  const bcf::PassPlan pl = bcf::plan_passes(key_bits);
  const bcf::SegLayout L = bcf::seg_layout(n_total, nseg, val_bytes, pl.passes, true);
  if (!ws || !aligned16(ws)) return BCF_E_INVAL;
  if (ws_bytes < L.total) return BCF_E_WORKSPACE;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::segmented_sort(keys_in, vals_in, keys_out, vals_out, n_total, offs, nseg,
                                     val_bytes, pl, static_cast<unsigned char*>(ws), L,
                                     (cudaStream_t)stream));
}

int bcf_segmented_partition_workspace_size(int64_t n_total, int64_t nseg, int val_bytes,
                                           size_t* bytes) {
  if (!bytes || n_total < 0 || nseg < 0 || !valid_vb(val_bytes)) return BCF_E_INVAL;
  if (n_total >= kMaxSweepN || nseg >= ((int64_t)1 << 31)) return BCF_E_UNSUPPORTED;
  *bytes = bcf::seg_layout(n_total, nseg, val_bytes, 1, false).total;
  return BCF_OK;
}

int bcf_segmented_partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                            void* vals_out, int64_t n_total, const int64_t* offs,
                            const int32_t* w_per_seg, int64_t nseg, int val_bytes, int flags,
                            void* ws, size_t ws_bytes, bcf_stream_t stream) {
  int rc = check_segments(keys_in, vals_in, keys_out, vals_out, n_total, offs, nseg, val_bytes);
  if (rc) return rc;
  if (nseg > 0 && (!w_per_seg || (reinterpret_cast<uintptr_t>(w_per_seg) & 3u))) return BCF_E_INVAL;
  if (nseg == 0) return BCF_OK;
  const bcf::SegLayout L = bcf::seg_layout(n_total, nseg, val_bytes, 1, false);
  if (!ws || !aligned16(ws)) return BCF_E_INVAL;
  if (ws_bytes < L.total) return BCF_E_WORKSPACE;
  if (!device_ready()) return BCF_E_CUDA;
  return cuda_rc(bcf::segmented_partition(keys_in, vals_in, keys_out, vals_out, n_total, offs, w_per_seg,
                                          nseg, val_bytes, (flags & BCF_ASSUME_BALANCED) != 0,
                                          static_cast<unsigned char*>(ws), L, (cudaStream_t)stream));
}

// ------------------------------------------------------------------ tuning
int bcf_tune_num_configs(void) { return bcf::kNumSweepConfigs; }

int bcf_tune_config_info(int config, int* threads, int* keys_per_thread) {
  if (config < 0 || config >= bcf::kNumSweepConfigs || !threads || !keys_per_thread) return BCF_E_INVAL;
  *threads = bcf::kSweepCfgThreads[config];
  *keys_per_thread = bcf::kSweepCfgIPT[config];
  return BCF_OK;
}

int bcf_tune_config_form(int config) {
  if (config < 0 || config >= bcf::kNumSweepConfigs) return BCF_E_INVAL;
  return bcf::cfg_form(config);
}

static_assert(bcf::kOpSegmentedSort == BCF_OP_SEGMENTED_SORT && bcf::kTuneOps == BCF_OP_SEGMENTED_SORT + 1,
              "tuning operations of the header and the table");

int bcf_tune_set(int op, int log2_n, int config) {
  return bcf::tune_set(op, log2_n, config) == 0 ? BCF_OK : BCF_E_INVAL;
}

int bcf_tune_get(int op, int64_t n, int* config) {
  if (op < BCF_OP_SORT || op > BCF_OP_SEGMENTED_SORT || n < 0 || !config) return BCF_E_INVAL;
  *config = bcf::tuned_config(op, n);
  return BCF_OK;
}

// Tuning cache file: a text header line, then one line per explicit entry:
// "<device name>/<SMs>sm \t op \t log2_n \t config".  Entries of other devices are
// kept when this device's entries are rewritten.
static bool tune_device_key(std::string* key) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
  *key = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "sm";
  return true;
}

static const char kTuneHeader[] = "bcf-tune 1";

int bcf_tune_save(const char* path) {
  if (!path) return BCF_E_INVAL;
  std::string key;
  if (!tune_device_key(&key)) return BCF_E_CUDA;
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(path, "r")) {
    char line[512];
    bool first = true;
    while (std::fgets(line, sizeof line, f)) {
      std::string l(line);
      if (first) {
        first = false;
        if (l.rfind(kTuneHeader, 0) == 0) continue;
      }
      if (l.rfind(key + "\t", 0) != 0 && !l.empty() && l != "\n") keep.push_back(l);
    }
    std::fclose(f);
  }
  FILE* f = std::fopen(path, "w");
  if (!f) return BCF_E_INVAL;
  std::fprintf(f, "%s\n", kTuneHeader);
  for (const std::string& l : keep) std::fputs(l.c_str(), f);
  for (int op = 0; op < bcf::kTuneOps; ++op)
    for (int b = 0; b < 64; ++b) {
      const int c = bcf::tune_entry(op, b);
      if (c >= 0) std::fprintf(f, "%s\t%d\t%d\t%d\n", key.c_str(), op, b, c);
    }
  return std::fclose(f) == 0 ? BCF_OK : BCF_E_INVAL;
}

int bcf_tune_load(const char* path, int* applied) {
  if (!path) return BCF_E_INVAL;
  if (applied) *applied = 0;
  std::string key;
  if (!tune_device_key(&key)) return BCF_E_CUDA;
  FILE* f = std::fopen(path, "r");
  if (!f) return BCF_E_INVAL;
  char line[512];
  int count = 0;
  bool ok = std::fgets(line, sizeof line, f) && std::string(line).rfind(kTuneHeader, 0) == 0;
  while (ok && std::fgets(line, sizeof line, f)) {
    std::string l(line);
    if (l.rfind(key + "\t", 0) != 0) continue;
    int op = -1, b = -1, c = -2;
    if (std::sscanf(l.c_str() + key.size() + 1, "%d\t%d\t%d", &op, &b, &c) != 3 || bcf::tune_set(op, b, c) != 0) {
      ok = false;
      break;
    }
    ++count;
  }
  std::fclose(f);
  if (applied) *applied = count;
  return ok ? BCF_OK : BCF_E_INVAL;
}

int bcf_debug_lookback(int silent_tile, unsigned spin_limit) {
  if (silent_tile >= 0 && spin_limit == 0) return BCF_E_INVAL;
  bcf::debug_lookback(silent_tile, spin_limit);
  return BCF_OK;
}

}  // extern "C"
