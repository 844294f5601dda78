/*
 * bcf_oracle.h -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * Plain, slow, obviously-correct CPU definitions of what the bank-conflict-free
 * library computes (Afshani & Sitchinava, "Sorting and Permuting without Bank
 * Conflicts on GPUs", arXiv 1507.01391).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this code.  It shares no code,
 * header, table or helper with the CUDA library and does not include its header.
 *
 * Every function returns 0 on success and a negative code on an input that breaks
 * the stated precondition (the outputs are then left unspecified).
 */
#ifndef BCF_ORACLE_H
#define BCF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_OK 0
#define ORACLE_E_KEY (-1)        /* partition key outside [0, w) */
#define ORACLE_E_BALANCE (-2)    /* balanced partition with a bucket count != n/w */
#define ORACLE_E_PERM (-3)       /* permutation not a bijection / index out of range */
#define ORACLE_E_ARG (-4)        /* bad size or element width */
#define ORACLE_E_NOMEM (-5)

/* Sorting problem (Sec. 1, "Problems of interest"): ascending by key, stable. */
int oracle_sort_kv(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                   void* vals_out, int64_t n, int val_bytes);

/* Number of positions a stable ascending sort puts before element i. */
int64_t oracle_stable_rank(const uint32_t* keys, int64_t n, int64_t i);

/* Partition problem (Sec. 1; abstract): stable counting partition by label. */
int oracle_partition_kv(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                        void* vals_out, int64_t n, int64_t w, int balanced, int val_bytes);

/* Partition by splitters (pivot bucketing, Sec. 1): label of key k = number of
 * splitters s[t] <= k, then the stable counting partition by that label, moving
 * the keys themselves.  Splitters must be non-decreasing (ORACLE_E_ARG otherwise). */
int oracle_partition_splitters(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                               void* vals_out, int64_t n, const uint32_t* splitters,
                               int64_t nsplit, int balanced, int val_bytes);

/* Permutation problem (Sec. 1): out[pi[i]] = in[i] after a bijectivity check. */
int oracle_permute(const void* src, void* dst, const uint32_t* pi, int64_t n,
                   int elem_bytes);

/* Tile-local permutation: out[t*T + lpi[t*T+i]] = in[t*T+i]. */
int oracle_permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi,
                         int64_t n, int64_t tile);

/* dst[i] = src[idx[i]] -- the inverse direction of a scatter permutation. */
int oracle_gather(const void* src, void* dst, const uint32_t* idx, int64_t n,
                  int64_t n_src, int elem_bytes);

/* Per-segment versions over CSR offsets offs[0..nseg]. */
int oracle_segmented_sort_kv(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                             void* vals_out, const int64_t* offs, int64_t nseg,
                             int val_bytes);
int oracle_segmented_partition_kv(const uint32_t* keys, const void* vals,
                                  uint32_t* keys_out, void* vals_out,
                                  const int64_t* offs, const int32_t* w_per_seg,
                                  int64_t nseg, int balanced, int val_bytes);

/* Lemma 1 ("short and wide" sort, Sec. 2) on a w x m matrix stored row by row
 * (M[r*m + c]).  The individual steps are exported so a test can inspect the
 * matrix between them. */
void oracle_l1_sort_rows(uint32_t* M, int64_t w, int64_t m, int alternating);
void oracle_l1_row_to_col(uint32_t* M, int64_t w, int64_t m);
void oracle_l1_col_to_row(uint32_t* M, int64_t w, int64_t m);
int oracle_lemma1_sort(uint32_t* M, int64_t w, int64_t m);

/* Lemma 2 model (Sec. 2): 0-1 partition of a w x m matrix (labels in lab, 0 or 1;
 * payloads in pay; rows stored one after another), w = m or w = m*m, m a multiple
 * of 4.  stage 1..4 stops after balancing / convert-and-divide / column sorts /
 * shifted squares (4 = the whole algorithm).  The two step sorts are exported for
 * the pins: a column-major sort of the matrix made of rows[0..h), and a row-major
 * sort of rows [r0, r0 + h).  All sorts are stable 0-1 sorts. */
int oracle_lemma2_partition(uint32_t* lab, uint32_t* pay, int64_t w, int64_t m, int stage);
int oracle_l2_sort_colmajor(uint32_t* lab, uint32_t* pay, int64_t m, const int64_t* rows, int64_t h);
int oracle_l2_sort_rowmajor(uint32_t* lab, uint32_t* pay, int64_t m, int64_t r0, int64_t h);

/* The paper's bank model (Sec. 1, "Model of Computation") applied to a trace of
 * shared-memory accesses.  Record r: request id req[r] (records of one request
 * are contiguous), lane lane[r], byte address addr[r], access width width[r]
 * (4, 8 or 16 bytes).  Outputs: total hardware wavefronts, hardware conflicts
 * (wavefronts above one per phase), and conflicts under the strict model in
 * which two lanes may never touch the same bank in one request. */
/* Race check of a shared-memory trace (records of four uint32: request id,
 * thread | block << 16, byte address, width | kind << 8 | site << 16, kind 0 load,
 * 1 store, 2 atomic, 3 barrier).  Each warp's accesses are split by its barrier
 * records into segments; accesses of different threads of one block to one 4-byte
 * word in the same segment race when at least one is a store (atomics are not
 * checked).  *races receives the number of racing words, *words the number of
 * (block, segment, word) groups checked. */
int oracle_race_check(const uint32_t* rec, int64_t nrec, int64_t* races, int64_t* words);

int oracle_bank_count(const int64_t* req, const int32_t* lane, const uint32_t* addr,
                      const int32_t* width, int64_t nrec, int64_t* hw_wavefronts,
                      int64_t* hw_conflicts, int64_t* dmm_conflicts);

#ifdef __cplusplus
}
#endif
#endif
