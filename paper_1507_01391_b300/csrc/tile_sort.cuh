// tile_sort.cuh -- Lemma 1 ("short and wide" sort, Sec. 2) on one shared-memory tile.
//
// A tile of up to 4096 keys is the paper's w x m matrix with w = 16 rows and
// m = 256 columns (w*w <= m, the condition of Lemma 1).  Items are 64-bit
// (key << 32 | position in the tile): all distinct, so sorting them sorts the keys
// stably.  Item (r, c) sits at index c*16 + r of a u64 array, so row r always lives
// in the bank pair {2r, 2r+1}.  A 64-bit shared access is served per half-warp;
// in every half-warp the 16 lanes work on the 16 different rows, so every access
// below touches 16 distinct bank pairs: no bank conflicts (the CAC of Sec. 1).
//
// Schedule (Lemma 1): twice { sort rows alternating (row 0 ascending); convert
// row-major -> column-major; sort rows ascending; convert column-major ->
// row-major }, then sort rows ascending.  A final row -> column-major conversion
// puts sorted position t at index t, ready for a linear write-out.
//
// Row sort: the 16 threads of a row's team (one lane in each half-warp of the 8
// warps) each sort 16 consecutive items of the row in registers with Batcher's
// odd-even merge sorting network (63 comparators), then four merge-path rounds
// merge runs of 16 -> 256 inside the row's own banks.  A row sorted descending is
// sorted ascending on its complemented items (complemented when loaded, restored
// by the last merge round), so every comparison runs one way.  Conversions move
// one item per row per half-warp phase along a diagonal, so the 16 lanes of a
// phase read 16 different rows as well.  The first four conversions are done by
// the loads of the row sort that follows each: a thread reads its 16 items of the
// converted matrix straight from the unconverted one, in an order that keeps the
// lanes of a phase on 16 different rows.  After a row -> column-major conversion
// those 16 items are every 16th item of one sorted row, so they need no network.
#pragma once

#include "common.cuh"
#include "trace.cuh"

namespace bcf {

constexpr int kL1Threads = 256;   // 8 warps = 16 half-warps = 16 team members per row
constexpr int kL1Rows = 16;       // w
constexpr int kL1Cols = 256;      // m
constexpr int kL1Tile = kL1Rows * kL1Cols;
constexpr int kL1PerThread = kL1Cols / 16;  // items of a row per team member
constexpr size_t kL1SmemBytes = 2ull * kL1Tile * 8;

__device__ __forceinline__ void cas_u64(unsigned long long& a, unsigned long long& b) {
  const bool swap = a > b;
  const unsigned long long x = swap ? b : a, y = swap ? a : b;
  a = x;
  b = y;
}

// Ascending sort of 16 registers by Batcher's odd-even merge sort (Batcher 1968):
// for merge widths p = 1, 2, 4, 8 and strides k = p, p/2, ..., 1, compare
// elements i + j and i + j + k when both lie in the same block of 2p; 63
// comparators.  p and k are template arguments so that every loop unrolls and
// every register index is a constant: the 16 items stay in registers.
template <int P, int K>
__device__ __forceinline__ void oem_merge16(unsigned long long (&v)[16]) {
#pragma unroll
  for (int j = K % P; j + K < 16; j += 2 * K)
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i + j + K < 16 && (i + j) / (2 * P) == (i + j + K) / (2 * P)) cas_u64(v[i + j], v[i + j + K]);
  if constexpr (K > 1) oem_merge16<P, K / 2>(v);
}
template <int P = 1>
__device__ __forceinline__ void sort16(unsigned long long (&v)[16]) {
  oem_merge16<P, P>(v);
  if constexpr (2 * P < 16) sort16<2 * P>(v);
}

// One merge round of a row sort: runs [2bL, 2bL+L) and [2bL+L, 2bL+2L) of row r
// of src are merged into dst; team member t writes merged positions [16t, 16t+16)
// of its block, found by a merge-path search.  LAST: the items are restored from
// their complements (flip) as they are written.
template <int L, bool LAST>
__device__ __forceinline__ void l1_merge_round(const unsigned long long* src, unsigned long long* dst, int r,
                                               int t, unsigned long long flip) {
  const int o0 = t * 16;
  const int base = (o0 / (2 * L)) * (2 * L);
  const int d = o0 - base;
  const unsigned long long* A = src + (size_t)base * kL1Rows + r;
  const unsigned long long* B = src + (size_t)(base + L) * kL1Rows + r;
  int lo = d > L ? d - L : 0, hi = d < L ? d : L;
  while (lo < hi) {  // smallest i whose A[i] comes after B[d-1-i]
    const int mid = (lo + hi) >> 1;
    BCF_TR(&A[mid * kL1Rows], 8, 0, TS_L1_ROW_LD);
    BCF_TR(&B[(d - 1 - mid) * kL1Rows], 8, 0, TS_L1_ROW_LD);
    const unsigned long long a = A[mid * kL1Rows], b = B[(d - 1 - mid) * kL1Rows];
    if (a < b) lo = mid + 1;
    else hi = mid;
  }
  int i = lo, j = d - lo;
  unsigned long long* out = dst + (size_t)(base + d) * kL1Rows + r;
#pragma unroll 4
  for (int s = 0; s < 16; ++s) {
    if (i < L) BCF_TR(&A[i * kL1Rows], 8, 0, TS_L1_ROW_LD);
    if (j < L) BCF_TR(&B[j * kL1Rows], 8, 0, TS_L1_ROW_LD);
    const unsigned long long a = i < L ? A[i * kL1Rows] : 0ull;
    const unsigned long long b = j < L ? B[j * kL1Rows] : 0ull;
    const bool take_a = (j >= L) || (i < L && a < b);
    BCF_TR(&out[s * kL1Rows], 8, 1, TS_L1_ROW_ST);
    out[s * kL1Rows] = LAST ? ((take_a ? a : b) ^ flip) : (take_a ? a : b);
    i += take_a;
    j += !take_a;
  }
  BCF_SYNC();
}

// Where a row sort takes its items from.
enum L1Load {
  kL1Own,       // the rows of S
  kL1FromRows,  // row -> column-major conversion of src, whose rows are sorted alternating (row 0 ascending)
  kL1FromCols,  // column -> row-major conversion of src
};

// Sort every row (ascending, or alternating when alt: row 0 ascending) of S, or of
// the conversion of src (LOAD), into S.  Uses D as the merge buffer; the sorted
// rows end in S.  With a conversion, src is D or unused, never S.
template <int LOAD>
__device__ __forceinline__ void l1_sort_rows(const unsigned long long* src, unsigned long long* S,
                                             unsigned long long* D, bool alt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane & 15;                    // row
  const int t = (r + warp * 2 + (lane >> 4)) & 15;  // team member: 16 different ones in a half-warp
  const bool up = !(alt && (r & 1));
  const unsigned long long flip = up ? 0ull : ~0ull;  // descending rows sort complemented items
  unsigned long long v[16];
  if constexpr (LOAD == kL1FromRows) {
    // Position 16t + i of row r is src(t, 16i + r); src's row t is sorted ascending
    // for even t and descending for odd t, so read in that order the 16 items are
    // sorted.  The lanes of a half-warp read 16 different rows t.  (alt is false.)
    const int i0 = (t & 1) ? 15 : 0, di = (t & 1) ? -1 : 1;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int i = i0 + di * k;
      BCF_TR(&src[(i * 16 + r) * kL1Rows + t], 8, 0, TS_L1_CONVERT);
      v[k] = src[(i * 16 + r) * kL1Rows + t];
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if constexpr (LOAD == kL1FromCols) {
        // Position 16t + i of row r is src(i, 16r + t); lane r reads i = (k + r)
        // mod 16 in step k, so a half-warp's lanes read 16 different rows.  The
        // network sorts whatever order they arrive in.
        const int i = (k + r) & 15;
        BCF_TR(&src[(r * 16 + t) * kL1Rows + i], 8, 0, TS_L1_CONVERT);
        v[k] = src[(r * 16 + t) * kL1Rows + i] ^ flip;
      } else {
        BCF_TR(&S[(t * 16 + k) * kL1Rows + r], 8, 0, TS_L1_ROW_LD);
        v[k] = S[(t * 16 + k) * kL1Rows + r] ^ flip;
      }
    }
    sort16(v);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    BCF_TR(&S[(t * 16 + i) * kL1Rows + r], 8, 1, TS_L1_ROW_ST);
    S[(t * 16 + i) * kL1Rows + r] = v[i];
  }
  BCF_SYNC();
  // four merge rounds (runs of 16 -> 256), each specialised on its run length;
  // the last one restores the complemented rows, and the result is back in S
  static_assert(kL1Cols == 256 && kL1PerThread == 16, "runs of 16 merged four times fill a row");
  l1_merge_round<16, false>(S, D, r, t, flip);
  l1_merge_round<32, false>(D, S, r, t, flip);
  l1_merge_round<64, false>(S, D, r, t, flip);
  l1_merge_round<128, true>(D, S, r, t, flip);
}

// Row-major -> column-major: N(r, c) = M(c / 16, (c % 16) * 16 + r).
// Half-warp g (0..15), lane p writes row p at c = ((p + g) % 16) * 16 + j, reading
// row (p + g) % 16 of M: distinct rows within the phase.
__device__ __forceinline__ void l1_row_to_col(const unsigned long long* M, unsigned long long* N) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane & 15, g = warp * 2 + (lane >> 4);
  const int R = (p + g) & 15;
#pragma unroll 4
  for (int j = 0; j < 16; ++j) {
    const int c = R * 16 + j;
    BCF_TR(&M[(j * 16 + p) * kL1Rows + R], 8, 0, TS_L1_CONVERT);
    BCF_TR(&N[c * kL1Rows + p], 8, 1, TS_L1_CONVERT);
    N[c * kL1Rows + p] = M[(j * 16 + p) * kL1Rows + R];
  }
  BCF_SYNC();
}

// The Lemma 1 schedule on items already built in X; afterwards Y[t] holds the
// item of sorted position t.  Twice: sort rows alternating, convert to
// column-major, sort rows ascending, convert to row-major; then sort rows
// ascending and convert to column-major.  The first four conversions are fused
// into the row sorts after them.
__device__ __forceinline__ void lemma1_schedule(unsigned long long* X, unsigned long long* Y) {
  l1_sort_rows<kL1Own>(nullptr, X, Y, true);
#pragma unroll 1
  for (int rep = 0; rep < 2; ++rep) {
    l1_sort_rows<kL1FromRows>(X, Y, X, false);
    l1_sort_rows<kL1FromCols>(Y, X, Y, rep == 0);  // the second time: the final ascending sort
  }
  l1_row_to_col(X, Y);
}

// Sort one tile [start, start + len), len <= 4096, from keys_in/vals_in into
// keys_out/vals_out.  X and Y are two kL1Tile-item shared buffers.
template <int VB>
__device__ __forceinline__ void lemma1_tile(const uint32_t* __restrict__ keys_in,
                                            const void* __restrict__ vals_in,
                                            uint32_t* __restrict__ keys_out,
                                            void* __restrict__ vals_out, int64_t start, int len,
                                            unsigned long long* X, unsigned long long* Y) {
  using VT = typename ValT<VB>::type;
  // item (r, c) of the initial matrix = tile position q = c*16 + r
  for (int q = threadIdx.x; q < kL1Tile; q += kL1Threads) {
    const unsigned long long key = q < len ? (unsigned long long)keys_in[start + q] : 0xFFFFFFFFull;
    BCF_TR(&X[q], 8, 1, TS_L1_IO);
    X[q] = (key << 32) | (unsigned)q;  // padding sorts last (position >= len)
  }
  BCF_SYNC();
  lemma1_schedule(X, Y);  // Y[t] = item of sorted position t
  const VT* vin = reinterpret_cast<const VT*>(vals_in);
  VT* vout = reinterpret_cast<VT*>(vals_out);
  for (int t = threadIdx.x; t < len; t += kL1Threads) {
    BCF_TR(&Y[t], 8, 0, TS_L1_IO);
    const unsigned long long it = Y[t];
    keys_out[start + t] = (uint32_t)(it >> 32);
    if (VB) vout[start + t] = vin ? vin[start + (uint32_t)it] : VT(start + (uint32_t)it);
  }
  BCF_SYNC();
}

}  // namespace bcf
