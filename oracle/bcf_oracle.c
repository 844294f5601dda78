/*
 * bcf_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * Plain, slow, obviously-correct CPU definitions for the problems studied in
 * Afshani & Sitchinava, "Sorting and Permuting without Bank Conflicts on GPUs".
 * Every algorithm the paper gives reaches the exact sorted / partitioned /
 * permuted result (correctness of Lemma 1, Theorem 1 and the randomized
 * permutation of Sec. 3), so each oracle function is the plain definition written
 * out.  Only the Lemma 1 and Lemma 2 models and the bank model follow the paper's
 * steps (Lemma 2's 0-1 partition leaves the order of equal labels to its steps).
 *
 * No blocking, no fusion, no library sort: insertion sort and a bottom-up merge
 * sort, a counting partition, and a direct out[pi[i]] = in[i] loop.  Shares no
 * code with the CUDA library.  Only tests, the smoke check and the benchmark's
 * CPU legs load it.
 */
#include "bcf_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t key;
    uint32_t idx; /* original position: ties keep input order (stability) */
} kv_item;

/* Insertion sort of a[0..n) by key; equal keys keep their order because an item
 * only moves past strictly greater keys. */
static void insertion_sort_items(kv_item* a, int64_t n) {
    for (int64_t i = 1; i < n; ++i) {
        kv_item x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j].key > x.key) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = x;
    }
}

/* Bottom-up stable merge sort: runs of 32 are insertion-sorted, then runs are
 * merged pairwise, taking from the left run whenever keys are equal. */
static int merge_sort_items(kv_item* a, int64_t n) {
    const int64_t run = 32;
    for (int64_t lo = 0; lo < n; lo += run) {
        int64_t len = (n - lo < run) ? (n - lo) : run;
        insertion_sort_items(a + lo, len);
    }
    if (n <= run) return ORACLE_OK;
    kv_item* tmp = (kv_item*)malloc((size_t)n * sizeof(kv_item));
    if (!tmp) return ORACLE_E_NOMEM;
    kv_item* src = a;
    kv_item* dst = tmp;
    for (int64_t width = run; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = (lo + width < n) ? lo + width : n;
            int64_t hi = (lo + 2 * width < n) ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) {
                if (src[j].key < src[i].key) dst[k++] = src[j++];
                else dst[k++] = src[i++];
            }
            while (i < mid) dst[k++] = src[i++];
            while (j < hi) dst[k++] = src[j++];
        }
        kv_item* t = src;
        src = dst;
        dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(kv_item));
    free(tmp);
    return ORACLE_OK;
}

static int valid_val_bytes(int vb) { return vb == 0 || vb == 4 || vb == 8; }

/* Sorting problem (Sec. 1, "Problems of interest"): the output is the input in
 * ascending key order.  Payloads travel with their keys; equal keys keep their
 * input order, which makes the result unique. */
int oracle_sort_kv(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                   void* vals_out, int64_t n, int val_bytes) {
    if (n < 0 || n > (int64_t)0xFFFFFFFFLL || !valid_val_bytes(val_bytes))
        return ORACLE_E_ARG;
    if (n == 0) return ORACLE_OK;
    kv_item* a = (kv_item*)malloc((size_t)n * sizeof(kv_item));
    if (!a) return ORACLE_E_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        a[i].key = keys[i];
        a[i].idx = (uint32_t)i;
    }
    int rc = merge_sort_items(a, n);
    if (rc == ORACLE_OK) {
        for (int64_t r = 0; r < n; ++r) {
            keys_out[r] = a[r].key;
            if (val_bytes && vals && vals_out)
                memcpy((char*)vals_out + r * val_bytes,
                       (const char*)vals + (int64_t)a[r].idx * val_bytes, (size_t)val_bytes);
        }
    }
    free(a);
    return rc;
}

/* The position a stable ascending sort gives element i: the number of strictly
 * smaller keys plus the number of equal keys that come before it. */
int64_t oracle_stable_rank(const uint32_t* keys, int64_t n, int64_t i) {
    int64_t r = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (keys[j] < keys[i] || (keys[j] == keys[i] && j < i)) ++r;
    }
    return r;
}

/* Partition problem (Sec. 1 and the abstract): every item with label b goes to
 * bucket (row) b.  Counting sort: count each label, exclusive prefix of the
 * counts, then one forward pass that places items in input order (stable).
 * With `balanced`, the paper's precondition of exactly n/w copies of every
 * label is checked. */
int oracle_partition_kv(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                        void* vals_out, int64_t n, int64_t w, int balanced, int val_bytes) {
    if (n < 0 || w < 1 || !valid_val_bytes(val_bytes)) return ORACLE_E_ARG;
    if (balanced && (n % w) != 0) return ORACLE_E_BALANCE;
    int64_t* count = (int64_t*)calloc((size_t)w, sizeof(int64_t));
    if (!count) return ORACLE_E_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)keys[i] >= w) {
            free(count);
            return ORACLE_E_KEY;
        }
        count[keys[i]] += 1;
    }
    if (balanced) {
        for (int64_t b = 0; b < w; ++b) {
            if (count[b] != n / w) {
                free(count);
                return ORACLE_E_BALANCE;
            }
        }
    }
    /* exclusive prefix: next free slot of each bucket */
    int64_t run = 0;
    for (int64_t b = 0; b < w; ++b) {
        int64_t c = count[b];
        count[b] = run;
        run += c;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = count[keys[i]]++;
        keys_out[p] = keys[i];
        if (val_bytes && vals && vals_out)
            memcpy((char*)vals_out + p * val_bytes, (const char*)vals + i * val_bytes,
                   (size_t)val_bytes);
    }
    free(count);
    return ORACLE_OK;
}

/* Partition by splitters: each key's label is the count of splitters not above
 * it (a linear count, no search), then the same counting partition as above but
 * moving the original keys. */
int oracle_partition_splitters(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                               void* vals_out, int64_t n, const uint32_t* splitters,
                               int64_t nsplit, int balanced, int val_bytes) {
    if (n < 0 || nsplit < 0 || !valid_val_bytes(val_bytes)) return ORACLE_E_ARG;
    for (int64_t t = 1; t < nsplit; ++t)
        if (splitters[t - 1] > splitters[t]) return ORACLE_E_ARG;
    const int64_t w = nsplit + 1;
    if (balanced && (n % w) != 0) return ORACLE_E_BALANCE;
    uint32_t* label = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    int64_t* count = (int64_t*)calloc((size_t)w, sizeof(int64_t));
    if (!label || !count) {
        free(label);
        free(count);
        return ORACLE_E_NOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint32_t b = 0;
        for (int64_t t = 0; t < nsplit; ++t) b += splitters[t] <= keys[i];
        label[i] = b;
        count[b] += 1;
    }
    int rc = ORACLE_OK;
    if (balanced)
        for (int64_t b = 0; b < w; ++b)
            if (count[b] != n / w) rc = ORACLE_E_BALANCE;
    if (rc == ORACLE_OK) {
        int64_t run = 0;
        for (int64_t b = 0; b < w; ++b) {
            int64_t c = count[b];
            count[b] = run;
            run += c;
        }
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = count[label[i]]++;
            keys_out[p] = keys[i];
            if (val_bytes && vals && vals_out)
                memcpy((char*)vals_out + p * val_bytes, (const char*)vals + i * val_bytes,
                       (size_t)val_bytes);
        }
    }
    free(label);
    free(count);
    return rc;
}

/* Permutation problem (Sec. 1): the item at position i goes to position pi[i].
 * pi must be a bijection on [0, n); this is checked with a seen-table first. */
int oracle_permute(const void* src, void* dst, const uint32_t* pi, int64_t n,
                   int elem_bytes) {
    if (n < 0 || elem_bytes <= 0) return ORACLE_E_ARG;
    unsigned char* seen = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!seen) return ORACLE_E_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pi[i] >= n || seen[pi[i]]) {
            free(seen);
            return ORACLE_E_PERM;
        }
        seen[pi[i]] = 1;
    }
    free(seen);
    for (int64_t i = 0; i < n; ++i)
        memcpy((char*)dst + (int64_t)pi[i] * elem_bytes, (const char*)src + i * elem_bytes,
               (size_t)elem_bytes);
    return ORACLE_OK;
}

/* Tile-local permutation: tile t holds positions [t*T, min(n, (t+1)*T)); the item
 * at local position i goes to local position lpi[t*T + i] of the same tile. */
int oracle_permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi,
                         int64_t n, int64_t tile) {
    if (n < 0 || tile < 1 || tile > 65536) return ORACLE_E_ARG;
    unsigned char* seen = (unsigned char*)malloc((size_t)tile);
    if (!seen) return ORACLE_E_NOMEM;
    for (int64_t base = 0; base < n; base += tile) {
        int64_t len = (n - base < tile) ? (n - base) : tile;
        memset(seen, 0, (size_t)tile);
        for (int64_t i = 0; i < len; ++i) {
            int64_t d = lpi[base + i];
            if (d >= len || seen[d]) {
                free(seen);
                return ORACLE_E_PERM;
            }
            seen[d] = 1;
        }
        for (int64_t i = 0; i < len; ++i) dst[base + lpi[base + i]] = src[base + i];
    }
    free(seen);
    return ORACLE_OK;
}

/* dst[i] = src[idx[i]]. */
int oracle_gather(const void* src, void* dst, const uint32_t* idx, int64_t n,
                  int64_t n_src, int elem_bytes) {
    if (n < 0 || n_src < 0 || elem_bytes <= 0) return ORACLE_E_ARG;
    for (int64_t i = 0; i < n; ++i)
        if ((int64_t)idx[i] >= n_src) return ORACLE_E_PERM;
    for (int64_t i = 0; i < n; ++i)
        memcpy((char*)dst + i * elem_bytes, (const char*)src + (int64_t)idx[i] * elem_bytes,
               (size_t)elem_bytes);
    return ORACLE_OK;
}

static int valid_offsets(const int64_t* offs, int64_t nseg) {
    if (nseg < 0 || offs[0] != 0) return 0;
    for (int64_t s = 0; s < nseg; ++s)
        if (offs[s + 1] < offs[s]) return 0;
    return 1;
}

/* Segmented sort: each CSR segment [offs[s], offs[s+1]) is sorted on its own. */
int oracle_segmented_sort_kv(const uint32_t* keys, const void* vals, uint32_t* keys_out,
                             void* vals_out, const int64_t* offs, int64_t nseg,
                             int val_bytes) {
    if (!valid_offsets(offs, nseg) || !valid_val_bytes(val_bytes)) return ORACLE_E_ARG;
    for (int64_t s = 0; s < nseg; ++s) {
        int64_t lo = offs[s], len = offs[s + 1] - offs[s];
        const void* v = (val_bytes && vals) ? (const char*)vals + lo * val_bytes : NULL;
        void* vo = (val_bytes && vals_out) ? (char*)vals_out + lo * val_bytes : NULL;
        int rc = oracle_sort_kv(keys + lo, v, keys_out + lo, vo, len, val_bytes);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

/* Segmented partition: segment s is partitioned on its own with w_per_seg[s]
 * buckets. */
int oracle_segmented_partition_kv(const uint32_t* keys, const void* vals,
                                  uint32_t* keys_out, void* vals_out,
                                  const int64_t* offs, const int32_t* w_per_seg,
                                  int64_t nseg, int balanced, int val_bytes) {
    if (!valid_offsets(offs, nseg) || !valid_val_bytes(val_bytes)) return ORACLE_E_ARG;
    for (int64_t s = 0; s < nseg; ++s) {
        int64_t lo = offs[s], len = offs[s + 1] - offs[s];
        const void* v = (val_bytes && vals) ? (const char*)vals + lo * val_bytes : NULL;
        void* vo = (val_bytes && vals_out) ? (char*)vals_out + lo * val_bytes : NULL;
        int rc = oracle_partition_kv(keys + lo, v, keys_out + lo, vo, len, w_per_seg[s],
                                     balanced, val_bytes);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

/* ---- Lemma 1 model (Sec. 2): a w x m matrix, rows stored one after another ---- */

/* Step "sort rows": every row ascending, or (alternating) row 0 ascending, row 1
 * descending, and so on.  Insertion sort inside each row. */
void oracle_l1_sort_rows(uint32_t* M, int64_t w, int64_t m, int alternating) {
    for (int64_t r = 0; r < w; ++r) {
        uint32_t* row = M + r * m;
        int descending = alternating && (r % 2 == 1);
        for (int64_t i = 1; i < m; ++i) {
            uint32_t x = row[i];
            int64_t j = i - 1;
            while (j >= 0 && (descending ? row[j] < x : row[j] > x)) {
                row[j + 1] = row[j];
                --j;
            }
            row[j + 1] = x;
        }
    }
}

/* Step "row-major to column-major": read the matrix row by row and refill it
 * column by column (the first w items read form column 0). */
void oracle_l1_row_to_col(uint32_t* M, int64_t w, int64_t m) {
    int64_t n = w * m;
    uint32_t* seq = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!seq) return;
    memcpy(seq, M, (size_t)n * sizeof(uint32_t)); /* row-by-row reading order */
    for (int64_t c = 0; c < m; ++c)
        for (int64_t r = 0; r < w; ++r) M[r * m + c] = seq[c * w + r];
    free(seq);
}

/* Step "column-major to row-major": read the matrix column by column and refill
 * it row by row (the first m items read form row 0). */
void oracle_l1_col_to_row(uint32_t* M, int64_t w, int64_t m) {
    int64_t n = w * m;
    uint32_t* seq = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!seq) return;
    for (int64_t c = 0; c < m; ++c)
        for (int64_t r = 0; r < w; ++r) seq[c * w + r] = M[r * m + c];
    memcpy(M, seq, (size_t)n * sizeof(uint32_t));
    free(seq);
}

/* Lemma 1: twice { rows alternating; row->column-major; rows ascending;
 * column->row-major }, then rows ascending.  Valid when w*w <= m. */
int oracle_lemma1_sort(uint32_t* M, int64_t w, int64_t m) {
    if (w < 1 || m < 1) return ORACLE_E_ARG;
    for (int rep = 0; rep < 2; ++rep) {
        oracle_l1_sort_rows(M, w, m, 1);
        oracle_l1_row_to_col(M, w, m);
        oracle_l1_sort_rows(M, w, m, 0);
        oracle_l1_col_to_row(M, w, m);
    }
    oracle_l1_sort_rows(M, w, m, 0);
    return ORACLE_OK;
}

/* ---- Lemma 2 model (Sec. 2): 0-1 partition of a w x m matrix, w = m or m^2 ----
 *
 * lab holds the 0/1 labels and pay the payloads of the w x m matrix, rows stored
 * one after another (cell r*m + c).  Every "sort" of the proof is a 0-1 sort of
 * a sequence of cells; the proof does not say which of the equal items goes
 * where, so each one here is stable: the 0-items fill the first cells of the
 * sequence in the order they were met, then the 1-items. */

/* Stable 0-1 partition of the items in cells cell[0..s), taken in that order. */
static int l2_partition_cells(uint32_t* lab, uint32_t* pay, const int64_t* cell, int64_t s) {
    uint32_t* tl = (uint32_t*)malloc((size_t)s * sizeof(uint32_t));
    uint32_t* tp = (uint32_t*)malloc((size_t)s * sizeof(uint32_t));
    if (!tl || !tp) {
        free(tl);
        free(tp);
        return ORACLE_E_NOMEM;
    }
    int64_t o = 0;
    for (int label = 0; label <= 1; ++label)
        for (int64_t i = 0; i < s; ++i)
            if (lab[cell[i]] == (uint32_t)label) {
                tl[o] = lab[cell[i]];
                tp[o] = pay[cell[i]];
                ++o;
            }
    for (int64_t i = 0; i < s; ++i) {
        lab[cell[i]] = tl[i];
        pay[cell[i]] = tp[i];
    }
    free(tl);
    free(tp);
    return ORACLE_OK;
}

/* Sort the matrix made of rows rows[0..h) (all m columns) in column-major order:
 * its column 0 top to bottom, then column 1, and so on. */
int oracle_l2_sort_colmajor(uint32_t* lab, uint32_t* pay, int64_t m, const int64_t* rows, int64_t h) {
    int64_t* cell = (int64_t*)malloc((size_t)(h * m) * sizeof(int64_t));
    if (!cell) return ORACLE_E_NOMEM;
    for (int64_t c = 0; c < m; ++c)
        for (int64_t j = 0; j < h; ++j) cell[c * h + j] = rows[j] * m + c;
    int rc = l2_partition_cells(lab, pay, cell, h * m);
    free(cell);
    return rc;
}

/* Sort the contiguous rows [r0, r0 + h) in row-major order. */
int oracle_l2_sort_rowmajor(uint32_t* lab, uint32_t* pay, int64_t m, int64_t r0, int64_t h) {
    int64_t* cell = (int64_t*)malloc((size_t)(h * m) * sizeof(int64_t));
    if (!cell) return ORACLE_E_NOMEM;
    for (int64_t i = 0; i < h * m; ++i) cell[i] = r0 * m + i;
    int rc = l2_partition_cells(lab, pay, cell, h * m);
    free(cell);
    return rc;
}

/* Balancing on w = m^k rows: round i works on sub-matrices of m^i contiguous
 * rows, m of them to a group; square j of a group takes row j of each of the
 * group's sub-matrices, and every square is sorted in column-major order.  Round
 * 0 (sub-matrices of one row) therefore sorts squares of m contiguous rows. */
static int l2_balance(uint32_t* lab, uint32_t* pay, int64_t w, int64_t m) {
    int64_t* rows = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    if (!rows) return ORACLE_E_NOMEM;
    int rc = ORACLE_OK;
    for (int64_t sub = 1; sub < w && rc == ORACLE_OK; sub *= m) {
        int64_t group = sub * m;
        for (int64_t g = 0; g < w / group && rc == ORACLE_OK; ++g)
            for (int64_t j = 0; j < sub && rc == ORACLE_OK; ++j) {
                for (int64_t t = 0; t < m; ++t) rows[t] = g * group + t * sub + j;
                rc = oracle_l2_sort_colmajor(lab, pay, m, rows, m);
            }
    }
    free(rows);
    return rc;
}

/* Convert: read the w x m matrix column by column and refill it row by row. */
static int l2_col_to_row(uint32_t* a, int64_t w, int64_t m) {
    uint32_t* seq = (uint32_t*)malloc((size_t)(w * m) * sizeof(uint32_t));
    if (!seq) return ORACLE_E_NOMEM;
    for (int64_t c = 0; c < m; ++c)
        for (int64_t r = 0; r < w; ++r) seq[c * w + r] = a[r * m + c];
    memcpy(a, seq, (size_t)(w * m) * sizeof(uint32_t));
    free(seq);
    return ORACLE_OK;
}

/* Lemma 2's algorithm on a w x m matrix, w = m (sorted directly, row-major) or
 * w = m^2 (k = log_m w = 2, d = 2k dirty columns at most).  stage limits how
 * far it runs: 1 balancing; 2 then convert and divide into m*d sub-problems of
 * w/(m*d) <= m rows, each sorted directly in row-major order; 3 then every column
 * sorted (the column, read top to bottom, refilled row by row into a w/m x m
 * matrix that this function sorts, and read back); 4 (all) then the squares of m
 * contiguous rows sorted in row-major order, and again with the decomposition
 * shifted down by m/2 rows.  The w rows are the banks.  Labels must be 0 or 1. */
int oracle_lemma2_partition(uint32_t* lab, uint32_t* pay, int64_t w, int64_t m, int stage) {
    if (m < 4 || m % 4 != 0 || !(w == m || w == m * m) || stage < 1) return ORACLE_E_ARG;
    for (int64_t i = 0; i < w * m; ++i)
        if (lab[i] > 1) return ORACLE_E_KEY;
    if (w == m) return oracle_l2_sort_rowmajor(lab, pay, m, 0, w);
    int rc = l2_balance(lab, pay, w, m);
    if (rc != ORACLE_OK || stage < 2) return rc;
    if ((rc = l2_col_to_row(lab, w, m)) != ORACLE_OK) return rc;
    if ((rc = l2_col_to_row(pay, w, m)) != ORACLE_OK) return rc;
    const int64_t d = 4, chunk = w / (m * d);
    for (int64_t r0 = 0; r0 < w && rc == ORACLE_OK; r0 += chunk) rc = oracle_l2_sort_rowmajor(lab, pay, m, r0, chunk);
    if (rc != ORACLE_OK || stage < 3) return rc;
    uint32_t* cl = (uint32_t*)malloc((size_t)w * sizeof(uint32_t));
    uint32_t* cp = (uint32_t*)malloc((size_t)w * sizeof(uint32_t));
    if (!cl || !cp) rc = ORACLE_E_NOMEM;
    for (int64_t c = 0; c < m && rc == ORACLE_OK; ++c) {
        for (int64_t r = 0; r < w; ++r) {
            cl[r] = lab[r * m + c];
            cp[r] = pay[r * m + c];
        }
        rc = oracle_lemma2_partition(cl, cp, w / m, m, 4);
        for (int64_t r = 0; r < w && rc == ORACLE_OK; ++r) {
            lab[r * m + c] = cl[r];
            pay[r * m + c] = cp[r];
        }
    }
    free(cl);
    free(cp);
    if (rc != ORACLE_OK || stage < 4) return rc;
    for (int64_t r0 = 0; r0 + m <= w && rc == ORACLE_OK; r0 += m) rc = oracle_l2_sort_rowmajor(lab, pay, m, r0, m);
    for (int64_t r0 = m / 2; r0 + m <= w && rc == ORACLE_OK; r0 += m) rc = oracle_l2_sort_rowmajor(lab, pay, m, r0, m);
    return rc;
}

/* ---- Race check of a trace ----
 * Records of store kind 3 mark a block-wide barrier (one per warp), kind 4 a
 * warp-wide barrier (one per warp).  Two accesses to one word race when they come
 * from different threads of one block, at least one is a store (atomics are
 * ordered among themselves and never race), no block barrier lies between them
 * (the same block epoch of each warp), and they are not both in one warp with a
 * warp barrier between them (different warp epochs). */
typedef struct {
    uint32_t block, epoch, word, thread, sub;
    int store;
} race_entry;

static int race_cmp(const void* a, const void* b) {
    const race_entry* x = (const race_entry*)a;
    const race_entry* y = (const race_entry*)b;
    if (x->block != y->block) return x->block < y->block ? -1 : 1;
    if (x->epoch != y->epoch) return x->epoch < y->epoch ? -1 : 1;
    if (x->word != y->word) return x->word < y->word ? -1 : 1;
    return 0;
}

/* Whether accesses i and j of one group race. */
static int race_pair(const race_entry* i, const race_entry* j) {
    if (i->thread == j->thread || (!i->store && !j->store)) return 0;
    if ((i->thread >> 5) == (j->thread >> 5) && i->sub != j->sub) return 0;  /* warp barrier between */
    return 1;
}

int oracle_race_check(const uint32_t* rec, int64_t nrec, int64_t* races, int64_t* words) {
    if (nrec < 0 || !races || !words) return ORACLE_E_ARG;
    /* block and warp barriers seen so far by each (block, warp) */
    uint32_t* seen = (uint32_t*)calloc((size_t)65536 * 32, sizeof(uint32_t));
    uint32_t* wseen = (uint32_t*)calloc((size_t)65536 * 32, sizeof(uint32_t));
    int64_t cap = 0;
    for (int64_t r = 0; r < nrec; ++r) {
        const uint32_t kind = (rec[4 * r + 3] >> 8) & 0xFF, width = rec[4 * r + 3] & 0xFF;
        if (kind == 0 || kind == 1) cap += (width + 3) / 4;
    }
    race_entry* e = (race_entry*)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(race_entry));
    if (!seen || !wseen || !e) {
        free(seen);
        free(wseen);
        free(e);
        return ORACLE_E_NOMEM;
    }
    int64_t ne = 0;
    for (int64_t r = 0; r < nrec; ++r) {
        const uint32_t thread = rec[4 * r + 1] & 0xFFFF, block = rec[4 * r + 1] >> 16;
        const uint32_t kind = (rec[4 * r + 3] >> 8) & 0xFF, width = rec[4 * r + 3] & 0xFF;
        const size_t slot = (size_t)block * 32 + ((thread >> 5) & 31);
        if (kind == 3) {
            seen[slot] += 1;
            continue;
        }
        if (kind == 4) {
            wseen[slot] += 1;
            continue;
        }
        if (kind != 0 && kind != 1) continue;
        for (uint32_t q = 0; q < (width + 3) / 4; ++q) {
            e[ne].block = block;
            e[ne].epoch = seen[slot];
            e[ne].sub = wseen[slot];
            e[ne].word = rec[4 * r + 2] / 4 + q;
            e[ne].thread = thread;
            e[ne].store = (int)kind;
            ++ne;
        }
    }
    qsort(e, (size_t)ne, sizeof(race_entry), race_cmp);
    int64_t nr = 0, nw = 0;
    for (int64_t a = 0; a < ne;) {
        int64_t b = a;
        while (b < ne && race_cmp(&e[a], &e[b]) == 0) ++b;
        /* one group: the accesses of one word in one block epoch of one block */
        int race = 0;
        for (int64_t i = a; i < b && !race; ++i) {
            if (!e[i].store) continue;
            for (int64_t j = a; j < b && !race; ++j)
                if (j != i) race = race_pair(&e[i], &e[j]);
        }
        nr += race;
        ++nw;
        a = b;
    }
    free(seen);
    free(wseen);
    free(e);
    *races = nr;
    *words = nw;
    return ORACLE_OK;
}

/* ---- Bank model (Sec. 1, "Model of Computation") ----
 * Shared memory is w = 32 banks of 4-byte words; the word at byte address a is in
 * bank (a/4) mod 32.  Hardware rule: a request is split into phases by access
 * width (4 B: one phase of 32 lanes; 8 B: two phases of 16; 16 B: four of 8); in
 * a phase, the number of wavefronts is the largest number of DISTINCT words that
 * any one bank must deliver (lanes reading the same word share it).  Strict rule
 * (the paper's CAC): the largest number of distinct LANES that touch any one bank
 * in the request; conflicts are that number minus one. */
int oracle_bank_count(const int64_t* req, const int32_t* lane, const uint32_t* addr,
                      const int32_t* width, int64_t nrec, int64_t* hw_wavefronts,
                      int64_t* hw_conflicts, int64_t* dmm_conflicts) {
    int64_t wf_total = 0, hw_conf = 0, dmm_conf = 0;
    int64_t r0 = 0;
    while (r0 < nrec) {
        int64_t r1 = r0;
        while (r1 < nrec && req[r1] == req[r0]) ++r1;
        int wdt = width[r0];
        if (wdt != 4 && wdt != 8 && wdt != 16) return ORACLE_E_ARG;
        int words_per_lane = wdt / 4;
        int lanes_per_phase = 32 / words_per_lane;
        /* hardware rule, phase by phase */
        for (int ph = 0; ph < words_per_lane; ++ph) {
            uint32_t words[32][32]; /* distinct words seen per bank (at most 32) */
            int nwords[32];
            int active = 0;
            memset(nwords, 0, sizeof(nwords));
            for (int64_t r = r0; r < r1; ++r) {
                if (width[r] != wdt) return ORACLE_E_ARG;
                if (lane[r] / lanes_per_phase != ph) continue;
                active = 1;
                for (int k = 0; k < words_per_lane; ++k) {
                    uint32_t word = addr[r] / 4 + (uint32_t)k;
                    int bank = (int)(word % 32);
                    int dup = 0;
                    for (int q = 0; q < nwords[bank]; ++q)
                        if (words[bank][q] == word) dup = 1;
                    if (!dup && nwords[bank] < 32) words[bank][nwords[bank]++] = word;
                }
            }
            if (!active) continue;
            int wf = 0;
            for (int b = 0; b < 32; ++b)
                if (nwords[b] > wf) wf = nwords[b];
            wf_total += wf;
            hw_conf += wf - 1;
        }
        /* strict rule over the whole request */
        {
            uint32_t lane_mask[32];
            memset(lane_mask, 0, sizeof(lane_mask));
            for (int64_t r = r0; r < r1; ++r)
                for (int k = 0; k < words_per_lane; ++k) {
                    uint32_t word = addr[r] / 4 + (uint32_t)k;
                    lane_mask[word % 32] |= 1u << (lane[r] & 31);
                }
            int worst = 0;
            for (int b = 0; b < 32; ++b) {
                int c = __builtin_popcount(lane_mask[b]);
                if (c > worst) worst = c;
            }
            if (worst > 0) dmm_conf += worst - 1;
        }
        r0 = r1;
    }
    *hw_wavefronts = wf_total;
    *hw_conflicts = hw_conf;
    *dmm_conflicts = dmm_conf;
    return ORACLE_OK;
}
