// partition_l2.cu -- Lemma 2 (Sec. 2): 0-1 partition of w x m matrices with
// w = m^2, m = 32 (bcf_partition_lemma2).
//
// One block of 1024 threads holds one 1024 x 32 matrix (32,768 items) in shared
// memory; thread r is the processor of row r (the paper's bank r).  The steps are
// the proof's: balancing (two rounds of column-major square sorts, the second on
// squares made of every 32nd row), conversion from column-major to row-major,
// division into 128 sub-problems of 8 rows sorted directly, a sort of every
// column, and row-major sorts of the squares of 32 contiguous rows, then of the
// same decomposition shifted down by 16 rows.  Every sort is a stable 0-1 sort of
// the cells in the stated order, so the payload order is fully determined.
//
// Layout: payload (r, c) at c*1024 + (r & ~31) + ((r + r/32) mod 32).  A column
// read by the 32 rows of any square of either balancing round -- rows 32g + t or
// rows 32t + j, t = 0..31 -- touches 32 distinct banks.  The second balancing
// round writes its sorted squares straight to their places after the conversion
// (square j becomes column j), so the conversion costs no pass of its own, and
// sorts that would move nothing are skipped (see the steps below).  Labels live as
// one 32-bit mask per row (bit c = label of column c; rows rotated the same way);
// after each sort the new masks follow from the zero counts alone.
#include "common.cuh"
#include "internal.h"
#include "trace.cuh"

namespace bcf {
namespace {

constexpr int kL2M = 32;                       // columns: items per row
constexpr int kL2W = kL2M * kL2M;              // rows: w = m^2
constexpr int kL2Items = kL2W * kL2M;          // items per matrix
constexpr int kL2PayWords = kL2W * (kL2M + 1); // also holds the padded row-major write-out
constexpr size_t kL2Smem = (size_t)(kL2PayWords + kL2W + 2 * 32 * 32 + 32) * 4;

__device__ __forceinline__ int l2_addr(int r, int c) {
  return c * kL2W + (r & ~31) + ((r + (r >> 5)) & 31);
}

// Label mask of row r, with the same rotation inside each group of 32 rows, so
// that rows 32t + j (t = 0..31) also fall into distinct banks.
__device__ __forceinline__ int lm_idx(int r) { return (r & ~31) + ((r + (r >> 5)) & 31); }

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) { return __reduce_add_sync(0xffffffffu, x); }

// Mask of a row that holds `zeros` 0-items followed by 1-items.
__device__ __forceinline__ uint32_t ones_after(int zeros) {
  return zeros >= 32 ? 0u : (zeros <= 0 ? 0xffffffffu : (0xffffffffu << zeros));
}

// The warp's square (its lane j holds row row_of(j), all 32 columns, in pay[] and
// lab) sorted in column-major order: the 0-items, taken column by column and top
// to bottom, fill the square's first cells in that order, then the 1-items.  The
// square's cells have been read into registers before any of them is written.
template <typename RowOf>
__device__ __forceinline__ void square_colmajor(uint32_t* P, uint32_t* Lm, const uint32_t (&pay)[32],
                                                uint32_t lab, RowOf row_of, unsigned lt, int lane) {
  const uint32_t Z = (uint32_t)kL2W - warp_sum((uint32_t)__popc(lab));
  uint32_t zb = 0;  // 0-items in earlier columns
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const uint32_t bit = (lab >> c) & 1u;
    const uint32_t b = __ballot_sync(0xffffffffu, bit);
    const uint32_t x = __popc(b & lt);  // 1-items above in this column; lane - x 0-items
    const uint32_t rho = bit ? Z + (32u * c - zb) + x : zb + (uint32_t)lane - x;
    uint32_t* dst = &P[l2_addr(row_of((int)(rho & 31u)), (int)(rho >> 5))];
    BCF_TR(dst, 4, 1, TS_L2_SQUARE);
    *dst = pay[c];
    zb += 32u - __popc(b);
  }
  // Cell (j, c) of the sorted square holds a 0 iff 32c + j < Z.
  const int zc = (int)Z > lane ? ((int)Z - lane + 31) / 32 : 0;
  BCF_TR(&Lm[lm_idx(row_of(lane))], 4, 1, TS_L2_SQUARE);
  Lm[lm_idx(row_of(lane))] = ones_after(zc);
}

// Rows [row0, row0 + G) (lane j of the G-lane group holds row row0 + j) sorted in
// row-major order.
template <int G>
__device__ __forceinline__ void rows_rowmajor(uint32_t* P, uint32_t* Lm, const uint32_t (&pay)[32],
                                              uint32_t lab, int row0, int lane, uint32_t site) {
  const int j = lane & (G - 1);
  const uint32_t zr = 32u - __popc(lab);
  uint32_t incl = zr;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o, G);
    if (j >= o) incl += v;
  }
  const uint32_t zb = incl - zr;                                  // 0-items in earlier rows
  const uint32_t Z = __shfl_sync(0xffffffffu, incl, G - 1, G);    // 0-items in the group
  const uint32_t ob = 32u * j - zb;                               // 1-items in earlier rows
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const uint32_t bit = (lab >> c) & 1u;
    const uint32_t x = __popc(lab & ((1u << c) - 1u));  // 1-items left of c; c - x 0-items
    const uint32_t rho = bit ? Z + ob + x : zb + (uint32_t)c - x;
    uint32_t* dst = &P[l2_addr(row0 + (int)(rho >> 5), (int)(rho & 31u))];
    BCF_TR(dst, 4, 1, site);
    *dst = pay[c];
  }
  BCF_TR(&Lm[lm_idx(row0 + j)], 4, 1, site);
  Lm[lm_idx(row0 + j)] = ones_after((int)Z - 32 * j);
}

// True when every G-lane group of the warp holds rows of one label only (each
// lane passes its row's mask).  Sorting such a group moves nothing, so the warp
// may leave it as it is; the answer is the same in every lane.
template <int G>
__device__ __forceinline__ bool groups_uniform(uint32_t lab) {
  const unsigned z = __ballot_sync(0xffffffffu, lab == 0u);
  const unsigned o = __ballot_sync(0xffffffffu, lab == 0xffffffffu);
  const unsigned m = G == 32 ? 0xffffffffu : ((1u << (G & 31)) - 1u);
  bool all = true;
#pragma unroll
  for (int g = 0; g < 32; g += G) all &= ((z >> g) & m) == m || ((o >> g) & m) == m;
  return all;
}

__device__ __forceinline__ void load_pay(const uint32_t* P, int r, uint32_t (&pay)[32], uint32_t site) {
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    BCF_TR(&P[l2_addr(r, c)], 4, 0, site);
    pay[c] = P[l2_addr(r, c)];
  }
}

__device__ __forceinline__ uint32_t load_mask(const uint32_t* Lm, int r, uint32_t site) {
  BCF_TR(&Lm[lm_idx(r)], 4, 0, site);
  return Lm[lm_idx(r)];
}

__device__ __forceinline__ void load_row(const uint32_t* P, const uint32_t* Lm, int r, uint32_t (&pay)[32],
                                         uint32_t& lab, uint32_t site) {
  load_pay(P, r, pay, site);
  lab = load_mask(Lm, r, site);
}

__global__ void __launch_bounds__(1024, 1) k_partition_l2(const uint32_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ vals,
                                                          uint32_t* keys_out, uint32_t* vals_out,
                                                          int64_t tiles, unsigned* status) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* P = sm;                   // payloads
  uint32_t* Lm = P + kL2PayWords;     // label mask of each row
  uint32_t* zw = Lm + kL2W;           // column sort: zeros of warp g in column c at [g*32 + c]
  uint32_t* zpre = zw + 32 * 32;      // ... and zeros of earlier warps
  uint32_t* ztot = zpre + 32 * 32;    // ... and zeros of the whole column
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned lt = lanemask_lt();
  uint32_t pay[32];
  uint32_t lab;

  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t base = tile * kL2Items;
    // Input item c*w + r of the matrix sits in row r, column c (column-major
    // layout, Sec. 1): thread r reads its row, one coalesced column at a time.
    const uint32_t* kin = keys + base + t;
    lab = 0;
    uint32_t any = 0;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const uint32_t k = __ldcs(kin + c * kL2W);
      any |= k;
      lab |= (k != 0u ? 1u : 0u) << c;
    }
    if (any > 1u) set_status(status, DEV_BAD_KEY);
#pragma unroll
    for (int c = 0; c < 32; ++c) pay[c] = vals ? __ldcs(vals + base + c * kL2W + t) : (uint32_t)(base + c * kL2W + t);

    // While this matrix is sorted, L2 fetches the block's next one (32 KB pieces).
    if (t < 8 && tile + gridDim.x < tiles) {
      const int64_t nb = (tile + gridDim.x) * kL2Items + (int64_t)(t & 3) * (kL2Items / 4);
      if (t < 4) prefetch_l2_bulk(keys + nb, (unsigned)(kL2Items / 4 * sizeof(uint32_t)));
      else if (vals) prefetch_l2_bulk(vals + nb, (unsigned)(kL2Items / 4 * sizeof(uint32_t)));
    }

    // Balancing, round 0: squares of 32 contiguous rows (one per warp).
    square_colmajor(P, Lm, pay, lab, [&](int j) { return warp * 32 + j; }, lt, lane);
    BCF_SYNC();
    // Round 1: square j takes row j of each of the 32 round-0 squares, and is
    // sorted in column-major order; then the conversion refills the matrix read
    // column by column into rows.  The two are composed: the item at position rho
    // of square j's sorted order sits in row 32*(rho mod 32) + j, column rho/32
    // after the sort, and the conversion moves that cell to row rho, column j.
    // So square j becomes column j, top to bottom, and every item is written
    // once.  Squares overlap other squares' columns, hence the block barrier
    // between all reads and all writes.
    load_row(P, Lm, lane * 32 + warp, pay, lab, TS_L2_CONVERT);
    BCF_SYNC();
    {
      const uint32_t Z = (uint32_t)kL2W - warp_sum((uint32_t)__popc(lab));
      if (lane == 0) {
        BCF_TR(&ztot[warp], 4, 1, TS_L2_CONVERT);
        ztot[warp] = Z;  // zeros of square (now column) `warp`
      }
      uint32_t zb = 0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const uint32_t bit = (lab >> c) & 1u;
        const uint32_t b = __ballot_sync(0xffffffffu, bit);
        const uint32_t x = __popc(b & lt);
        const uint32_t rho = bit ? Z + (32u * c - zb) + x : zb + (uint32_t)lane - x;
        BCF_TR(&P[l2_addr((int)rho, warp)], 4, 1, TS_L2_CONVERT);
        P[l2_addr((int)rho, warp)] = pay[c];
        zb += 32u - __popc(b);
      }
    }
    BCF_SYNC();
    // Row t now holds a 1 in column j iff t >= (zeros of column j).
    {
      uint32_t m = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        BCF_TR(&ztot[j], 4, 0, TS_L2_CONVERT);
        m |= ((uint32_t)t >= ztot[j] ? 1u : 0u) << j;
      }
      BCF_TR(&Lm[lm_idx(t)], 4, 1, TS_L2_CONVERT);
      Lm[lm_idx(t)] = m;
    }

    // Divide: 128 sub-problems of 8 contiguous rows, each sorted row-major.  Only
    // the few that hold both labels move anything: a warp whose four are all
    // single-label leaves them in place.
    lab = load_mask(Lm, t, TS_L2_DIVIDE);
    if (!groups_uniform<8>(lab)) {
      load_pay(P, t, pay, TS_L2_DIVIDE);
      BCF_SYNCWARP();
      rows_rowmajor<8>(P, Lm, pay, lab, warp * 32 + (lane & ~7), lane, TS_L2_DIVIDE);
    }
    BCF_SYNC();

    // Column sorts: each column, top to bottom, stably 0s then 1s.  The row's
    // payloads are read after the counts (and before the barrier that precedes
    // any write).
    lab = load_mask(Lm, t, TS_L2_COLUMN);
    uint32_t myz = 0;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const uint32_t b = __ballot_sync(0xffffffffu, (lab >> c) & 1u);
      if (c == lane) myz = 32u - __popc(b);
    }
    BCF_TR(&zw[warp * 32 + lane], 4, 1, TS_L2_COLUMN);
    zw[warp * 32 + lane] = myz;
    BCF_SYNC();
    bool moves;  // does any item of this warp's rows change place?
    {
      uint32_t pre = 0, tot = 0;  // of column `lane`
#pragma unroll 4
      for (int g = 0; g < 32; ++g) {
        BCF_TR(&zw[g * 32 + lane], 4, 0, TS_L2_COLUMN);
        const uint32_t z = zw[g * 32 + lane];
        pre += g < warp ? z : 0u;
        tot += z;
      }
      BCF_TR(&zpre[warp * 32 + lane], 4, 1, TS_L2_COLUMN);
      zpre[warp * 32 + lane] = pre;
      if (warp == 0) {
        BCF_TR(&ztot[lane], 4, 1, TS_L2_COLUMN);
        ztot[lane] = tot;
      }
      // Rows of 0s with only 0s above them in every column, or rows of 1s with
      // only 1s from them down, already sit where the column sort puts them.
      moves = !(__all_sync(0xffffffffu, lab == 0u && pre == 32u * warp) ||
                __all_sync(0xffffffffu, lab == 0xffffffffu && tot == pre));
    }
    if (moves) load_pay(P, t, pay, TS_L2_COLUMN);
    BCF_SYNC();
    if (moves) {
      const uint32_t* vzp = zpre + warp * 32;
      const uint32_t* vzt = ztot;
      uint32_t nm = 0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const uint32_t bit = (lab >> c) & 1u;
        const uint32_t b = __ballot_sync(0xffffffffu, bit);
        BCF_TR(&vzp[c], 4, 0, TS_L2_COLUMN);
        BCF_TR(&vzt[c], 4, 0, TS_L2_COLUMN);
        const uint32_t zp = vzp[c], zt = vzt[c];
        const uint32_t x = __popc(b & lt);
        const uint32_t rho = bit ? zt + (32u * warp - zp) + x : zp + (uint32_t)lane - x;
        BCF_TR(&P[l2_addr((int)rho, c)], 4, 1, TS_L2_COLUMN);
        P[l2_addr((int)rho, c)] = pay[c];
        nm |= ((uint32_t)t >= zt ? 1u : 0u) << c;
      }
      BCF_TR(&Lm[lm_idx(t)], 4, 1, TS_L2_COLUMN);
      Lm[lm_idx(t)] = nm;
    }
    BCF_SYNC();

    // Squares of 32 contiguous rows sorted row-major, then the decomposition
    // shifted down by 16 rows.
    // Single-label squares (all but the one or two that hold the dirty rows) are
    // left in place.
    lab = load_mask(Lm, t, TS_L2_ROWS);
    if (!groups_uniform<32>(lab)) {
      load_pay(P, t, pay, TS_L2_ROWS);
      BCF_SYNCWARP();
      rows_rowmajor<32>(P, Lm, pay, lab, warp * 32, lane, TS_L2_ROWS);
    }
    BCF_SYNC();
    if (warp < 31) {
      const int r = warp * 32 + 16 + lane;
      lab = load_mask(Lm, r, TS_L2_SHIFTED);
      if (!groups_uniform<32>(lab)) {
        load_pay(P, r, pay, TS_L2_SHIFTED);
        BCF_SYNCWARP();
        rows_rowmajor<32>(P, Lm, pay, lab, warp * 32 + 16, lane, TS_L2_SHIFTED);
      }
    }
    BCF_SYNC();

    // Write-out in row-major order (output item r*m + c), staged through a
    // padded row-major copy so that both sides are conflict-free and coalesced.
    load_row(P, Lm, t, pay, lab, TS_L2_IO);
    BCF_SYNC();
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      BCF_TR(&P[t * 33 + c], 4, 1, TS_L2_IO);
      P[t * 33 + c] = pay[c];
    }
    BCF_SYNC();
    uint32_t* vo = vals_out + base;
    uint32_t* ko = keys_out + base;
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const int q = i * kL2W + t, r = q >> 5, c = q & 31;
      BCF_TR(&P[r * 33 + c], 4, 0, TS_L2_IO);
      __stcs(vo + q, P[r * 33 + c]);
      __stcs(ko + q, (load_mask(Lm, r, TS_L2_IO) >> c) & 1u);
    }
    BCF_SYNC();
  }
}

}  // namespace

cudaError_t partition_lemma2(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out, uint32_t* vals_out,
                             int64_t n, cudaStream_t s) {
  const int64_t tiles = n / kL2Items;
  if (tiles == 0) return cudaSuccess;
  static bool ready[64] = {};
  cudaError_t e = set_smem_once(k_partition_l2, (int)kL2Smem, ready);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(tiles, std::max(1, sm_count_cached()));
  k_partition_l2<<<(unsigned)grid, 1024, kL2Smem, s>>>(keys, vals, keys_out, vals_out, tiles, status_word());
  return cudaGetLastError();
}

BCF_TRACE_INSTALLER(partition_l2)

}  // namespace bcf
