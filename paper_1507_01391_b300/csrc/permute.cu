// permute.cu -- the permutation problem (Sec. 1): dst[pi[i]] = src[i], its inverse
// direction (gather) and the optional bijectivity check.
//
// Global scatter: every thread reads four consecutive items of src and pi with
// 128-bit loads and issues four scattered 4- or 8-byte stores.  Scattered stores
// only reach HBM efficiently when L2 can hold every partially written line until
// all of it has arrived, so key-value permutations run as two passes (keys, then
// payloads) whose outputs each fit the 126 MB L2; the fused one-pass form, whose
// 2 x 64 MB output at n = 2^24 does not fit, is kept for comparison.
#include "common.cuh"
#include "internal.h"

namespace bcf {

template <int KB>
struct Elem;
template <>
struct Elem<4> {
  using T = uint32_t;
  using V4 = uint4;
};
template <>
struct Elem<8> {
  using T = unsigned long long;
  using V4 = ulonglong2;  // two elements per 16-byte load
};

// Indices local to rows of row_len items (row_len 0: one row) -> global indices
// of items i, i+1, ...; an index outside its row becomes n (rejected by callers).
template <int C>
__device__ __forceinline__ void local_to_global(uint32_t (&d)[C], int64_t i, int64_t n, int64_t row_len) {
  if (row_len <= 0) return;
  int64_t row0 = (i / row_len) * row_len;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    if (i + c >= row0 + row_len) row0 += row_len;
    const int64_t g = (int64_t)d[c] < row_len ? row0 + d[c] : n;
    d[c] = (uint32_t)(g < n ? g : n);
  }
}

__device__ __forceinline__ bool claim(uint32_t* seen, uint32_t d) {
  const uint32_t bit = 1u << (d & 31);
  return (atomicOr(seen + (d >> 5), bit) & bit) == 0;
}

#ifndef BCF_PERMUTE_HINTS
#define BCF_PERMUTE_HINTS 1   // L2 policy: streaming inputs evict first, scattered outputs evict last
#endif
#ifndef BCF_PERMUTE_VEC
#define BCF_PERMUTE_VEC 4     // items per thread per step (4 or 8)
#endif

// L2 eviction policies.  The scattered stores fill each output sector piece by
// piece; keeping those lines (evict_last) while the streaming reads go first
// lets most sectors complete in L2 before they are written to HBM.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint4 ld_stream_v4(const void* p, uint64_t pol) {
#if BCF_PERMUTE_HINTS
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
#else
  (void)pol;
  return __ldcs(reinterpret_cast<const uint4*>(p));
#endif
}

template <typename T>
__device__ __forceinline__ void st_keep(T* p, T v, uint64_t pol) {
#if BCF_PERMUTE_HINTS
  if constexpr (sizeof(T) == 4)
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"((uint32_t)v), "l"(pol) : "memory");
  else
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"((unsigned long long)v), "l"(pol)
                 : "memory");
#else
  (void)pol;
  *p = v;
#endif
}

template <typename T>
__device__ __forceinline__ void load4(const T* p, int64_t i, T (&out)[4], uint64_t pol) {
  if constexpr (sizeof(T) == 4) {
    const uint4 v = ld_stream_v4(p + i, pol);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else {
    const uint4 a = ld_stream_v4(p + i, pol);
    const uint4 b = ld_stream_v4(p + i + 2, pol);
    out[0] = ((unsigned long long)a.y << 32) | a.x;
    out[1] = ((unsigned long long)a.w << 32) | a.z;
    out[2] = ((unsigned long long)b.y << 32) | b.x;
    out[3] = ((unsigned long long)b.w << 32) | b.z;
  }
}

// KB: key/element bytes (4 or 8).  VB: payload bytes (0, 4 or 8).
template <int KB, int VB>
__global__ void __launch_bounds__(256) k_permute(const void* __restrict__ src_k,
                                                  const void* __restrict__ src_v,
                                                  void* __restrict__ dst_k,
                                                  void* __restrict__ dst_v,
                                                  const uint32_t* __restrict__ pi, int64_t n,
                                                  int64_t row_len, uint32_t* seen,
                                                  unsigned* status) {
  using KT = typename Elem<KB>::T;
  using VT = typename ValT<VB>::type;
  const KT* sk = reinterpret_cast<const KT*>(src_k);
  KT* dk = reinterpret_cast<KT*>(dst_k);
  const VT* sv = reinterpret_cast<const VT*>(src_v);
  VT* dv = reinterpret_cast<VT*>(dst_v);
  const uint64_t keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
  constexpr int V = BCF_PERMUTE_VEC;
  const int64_t nvec = n / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
    const int64_t i0 = v * V;
    uint32_t d[V];
    KT k[V];
    VT val[V];
#pragma unroll
    for (int h = 0; h < V; h += 4) {  // issue every load of the step before any store
      const uint4 p4 = ld_stream_v4(pi + i0 + h, stream);
      d[h] = p4.x; d[h + 1] = p4.y; d[h + 2] = p4.z; d[h + 3] = p4.w;
      KT kk[4];
      load4(sk, i0 + h, kk, stream);
#pragma unroll
      for (int c = 0; c < 4; ++c) k[h + c] = kk[c];
      if (VB) {
        VT vv[4];
        load4(sv, i0 + h, vv, stream);
#pragma unroll
        for (int c = 0; c < 4; ++c) val[h + c] = vv[c];
      }
    }
    local_to_global(d, i0, n, row_len);
#pragma unroll
    for (int c = 0; c < V; ++c) {
      bool ok = (int64_t)d[c] < n;
      if (ok && seen) ok = claim(seen, d[c]);
      if (!ok) {
        set_status(status, DEV_BAD_PERM);
        continue;
      }
      st_keep(dk + d[c], k[c], keep);
      if (VB) st_keep(dv + d[c], val[c], keep);
    }
  }
  for (int64_t i = nvec * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t d1[1] = {pi[i]};
    local_to_global(d1, i, n, row_len);
    const uint32_t d = d1[0];
    bool ok = (int64_t)d < n;
    if (ok && seen) ok = claim(seen, d);
    if (!ok) {
      set_status(status, DEV_BAD_PERM);
      continue;
    }
    dk[d] = sk[i];
    if (VB) dv[d] = sv[i];
  }
}

template <int EB>
__global__ void __launch_bounds__(256) k_gather(const void* __restrict__ src,
                                                 void* __restrict__ dst,
                                                 const uint32_t* __restrict__ idx, int64_t n,
                                                 int64_t n_src, int64_t row_len, unsigned* status) {
  using T = typename Elem<EB>::T;
  const T* s = reinterpret_cast<const T*>(src);
  T* d = reinterpret_cast<T*>(dst);
  const int64_t nvec = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
    const int64_t i = v * 4;
    const uint4 p4 = __ldcs(reinterpret_cast<const uint4*>(idx + i));
    uint32_t q[4] = {p4.x, p4.y, p4.z, p4.w};
    local_to_global(q, i, n_src, row_len);
    T out[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if ((int64_t)q[c] < n_src) {
        out[c] = s[q[c]];
      } else {
        out[c] = T(0);
        set_status(status, DEV_BAD_PERM);
      }
    }
    if constexpr (EB == 4) {
      __stcs(reinterpret_cast<uint4*>(d + i), make_uint4(out[0], out[1], out[2], out[3]));
    } else {
      __stcs(reinterpret_cast<ulonglong2*>(d + i), make_ulonglong2(out[0], out[1]));
      __stcs(reinterpret_cast<ulonglong2*>(d + i + 2), make_ulonglong2(out[2], out[3]));
    }
  }
  for (int64_t i = nvec * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t q1[1] = {idx[i]};
    local_to_global(q1, i, n_src, row_len);
    const uint32_t q = q1[0];
    if ((int64_t)q < n_src) {
      d[i] = s[q];
    } else {
      d[i] = T(0);
      set_status(status, DEV_BAD_PERM);
    }
  }
}

static int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static unsigned grid_for(int64_t n) {
  const int64_t want = (n / BCF_PERMUTE_VEC + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;  // 8 resident blocks of 256 per SM
  int64_t g = want < cap ? want : cap;
  return (unsigned)(g > 0 ? g : 1);
}

template <int KB>
static cudaError_t permute_kb(const void* sk, const void* sv, void* dk, void* dv,
                              const uint32_t* pi, int64_t n, int64_t row_len, int vb,
                              uint32_t* seen, cudaStream_t s) {
  const unsigned g = grid_for(n);
  unsigned* st = status_word();
  switch (vb) {
    case 0: k_permute<KB, 0><<<g, 256, 0, s>>>(sk, sv, dk, dv, pi, n, row_len, seen, st); break;
    case 4: k_permute<KB, 4><<<g, 256, 0, s>>>(sk, sv, dk, dv, pi, n, row_len, seen, st); break;
    case 8: k_permute<KB, 8><<<g, 256, 0, s>>>(sk, sv, dk, dv, pi, n, row_len, seen, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t permute(const void* src_k, const void* src_v, void* dst_k, void* dst_v,
                    const uint32_t* pi, int64_t n, int64_t row_len, int kbytes, int vbytes,
                    uint32_t* seen_bitmap, bool fused, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (seen_bitmap && (fused || !vbytes)) {
    cudaError_t e = cudaMemsetAsync(seen_bitmap, 0, (size_t)((n + 31) / 32) * 4, s);
    if (e != cudaSuccess) return e;
  }
  if (!fused && vbytes) {
    // Keys, then payloads: each pass scatters into one output array, whose
    // partially written lines then stay in L2 until they are complete.
    cudaError_t e = permute(src_k, nullptr, dst_k, nullptr, pi, n, row_len, kbytes, 0, seen_bitmap,
                            true, s);
    if (e != cudaSuccess) return e;
    return permute(src_v, nullptr, dst_v, nullptr, pi, n, row_len, vbytes, 0, nullptr, true, s);
  }
  if (kbytes == 4) return permute_kb<4>(src_k, src_v, dst_k, dst_v, pi, n, row_len, vbytes, seen_bitmap, s);
  if (kbytes == 8) return permute_kb<8>(src_k, src_v, dst_k, dst_v, pi, n, row_len, vbytes, seen_bitmap, s);
  return cudaErrorInvalidValue;
}

cudaError_t gather(const void* src, void* dst, const uint32_t* idx, int64_t n, int64_t n_src,
                   int64_t row_len, int eb, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const unsigned g = grid_for(n);
  if (eb == 4) k_gather<4><<<g, 256, 0, s>>>(src, dst, idx, n, n_src, row_len, status_word());
  else if (eb == 8) k_gather<8><<<g, 256, 0, s>>>(src, dst, idx, n, n_src, row_len, status_word());
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace bcf
