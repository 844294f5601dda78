/*
 * bcf.h -- bank-conflict-free sort, permute and w-way partition on B300 (sm_103a).
 *
 * C ABI of libbcf.so.  The operations are the three problems of Afshani &
 * Sitchinava, "Sorting and Permuting without Bank Conflicts on GPUs" (Sec. 1,
 * "Problems of interest"): sorting, w-way partitioning (sorting an input that
 * holds labels in [0, w)) and permuting (sending the item at position i to
 * position pi[i]).  The paper's w processors over w banks are the 32 lanes of a
 * warp over the 32 four-byte shared-memory banks of an SM.
 *
 * Conventions shared by every entry point
 *  - Every data pointer is a DEVICE pointer owned by the caller.  Except where a
 *    function says otherwise, the library allocates and frees no device memory:
 *    scratch comes from a caller-provided workspace whose size the matching
 *    *_workspace_size() call returns.  Key, value, index and workspace pointers
 *    must be 16-byte aligned (cudaMalloc and torch allocations are); a misaligned
 *    pointer returns BCF_E_INVAL.
 *  - Calls are asynchronous on `stream` (NULL is the legacy default stream).  The
 *    return code reports argument errors and launch failures only.  Errors found
 *    by the GPU while it runs (a label >= w, an unbalanced partition, a pi that is
 *    not a bijection, a look-back wait that gave up) are recorded in a device
 *    status word that bcf_get_status() reads; outputs are then unspecified, but
 *    no kernel writes outside the caller's buffers and no kernel waits forever.
 *  - Keys are uint32.  Payload ("value") elements are 0, 4 or 8 bytes and are
 *    moved as raw bits (float NaN / -0.0 patterns survive).  Sizes are int64.
 *  - Index payload: for the sorts, vals_in == NULL with val_bytes == 4 means the
 *    payload of item i is i (its input position, counted from the start of the
 *    array), so vals_out receives the sorting permutation (an argsort).
 *  - Nothing here throws.  The only host state kept between calls is the tuning
 *    table (bcf_tune_*) and, per device, the SM count and each kernel's raised
 *    shared-memory limit (set on first use).
 */
#ifndef BCF_H
#define BCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared without pulling in the CUDA headers. */
typedef struct CUstream_st* bcf_stream_t;

/* ---- status codes ---- */
#define BCF_OK 0
#define BCF_E_INVAL 1          /* bad argument: null pointer, size, alignment, width */
#define BCF_E_WORKSPACE 2      /* workspace smaller than *_workspace_size() */
#define BCF_E_UNSUPPORTED 3    /* valid request outside what the library handles */
#define BCF_E_CUDA 4           /* a CUDA launch or copy failed */
#define BCF_E_TIMEOUT 5        /* device: a bounded inter-block wait gave up */
#define BCF_E_NOT_BALANCED 6   /* device: balanced partition saw a count != n/w */
#define BCF_E_BAD_PERM 7       /* device: pi not a bijection / index out of range */
#define BCF_E_BAD_KEY 8        /* device: partition label >= w */
/* (device-detected bad CSR offsets or per-segment widths report BCF_E_INVAL) */

/* ---- flags ---- */
#define BCF_ASSUME_BALANCED 0x1   /* partition: exactly n/w copies of each label */
#define BCF_CHECK_PERM 0x2        /* permute: verify pi is a bijection (needs ws) */
#define BCF_TILES_COLOURED 0x10   /* permute_tiles: randomized colouring schedule */
#define BCF_PARTITION_LEMMA1 0x20 /* partition: Lemma 1 tile schedule */
#define BCF_PERMUTE_FUSED 0x40    /* permute_kv: one pass for keys and payloads */
#define BCF_PERMUTE_BUCKETED 0x80 /* permute: two coalesced passes through ws */
#define BCF_TILES_SORTED_FINISH 0x100 /* permute_tiles, coloured: Sec. 3 finishing step */
#define BCF_PARTITION_DIRECT 0x200 /* partition, w <= 32: no shared-memory scatter */

/* Message for a status code (static string; never NULL). */
const char* bcf_status_string(int status);

/* Library version as 10000*major + 100*minor + patch. */
int bcf_version(void);

/* Synchronises `stream`, then reads and clears the device status word.  *out is
 * BCF_OK or the most severe device error recorded since the last call, in the
 * order BCF_E_TIMEOUT > BCF_E_INVAL > BCF_E_BAD_PERM > BCF_E_NOT_BALANCED >
 * BCF_E_BAD_KEY.  The
 * word is shared by all calls on the device; bad segment offsets or widths found
 * on the device report BCF_E_INVAL.  Returns BCF_E_CUDA if the sync or the read
 * fails. */
int bcf_get_status(bcf_stream_t stream, int* out);

/* ---------------------------------------------------------------------------
 * Sorting (Sec. 1; the paper sorts in O((n/w) log n) time, Lemma 1 and
 * Theorem 1).  Stable ascending sort of n (key, value) pairs by key.
 *  keys_in/vals_in   input, n keys and n values (vals_in NULL: no payload when
 *                    val_bytes is 0, index payload when it is 4)
 *  keys_out/vals_out output; may equal the inputs (in place); must not overlap
 *                    them otherwise
 *  val_bytes         0, 4 or 8
 *  key_bits          1..32; every key must be < 2^key_bits (fewer digit passes)
 *  ws, ws_bytes      workspace of at least bcf_sort_workspace_size() bytes
 * Method: least-significant-digit radix passes of at most 8 bits; each pass ranks
 * and scatters tiles in shared memory and finds each tile's global offsets (per-
 * tile counts and a scan, or for n <= 2^18 a bounded decoupled look-back).  A pass
 * whose digit is the same in every key moves nothing and is skipped; the device
 * decides this from the first pass's read of the keys, with no host round trip,
 * so the call stays capturable in a CUDA graph.  n must be < 2^30. */
int bcf_sort_workspace_size(int64_t n, int val_bytes, int key_bits, size_t* bytes);
int bcf_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
             void* vals_out, int64_t n, int val_bytes, int key_bits, void* ws,
             size_t ws_bytes, bcf_stream_t stream);
/* Digit passes that the last bcf_sort with this workspace ran (the others were
 * skipped: their digit is the same in every key).  n, val_bytes and key_bits are
 * those of that call; `stream` is its stream, which this synchronises before it
 * reads two words of ws.  BCF_E_CUDA if the read fails. */
int bcf_sort_passes_run(const void* ws, int64_t n, int val_bytes, int key_bits, int* passes,
                        bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * w-way partition (Sec. 1 and abstract; Corollary 1 and Theorem 1 solve it in
 * O(n/w) time).  Stable: item i with label keys_in[i] in [0, w) goes to the block
 * of its label, blocks in label order, input order kept inside a block.
 *  w        1..256 buckets
 *  flags    BCF_ASSUME_BALANCED: exactly n/w copies of every label, so block b
 *           starts at b*n/w without a counting pass; n % w != 0 -> BCF_E_INVAL,
 *           other counts -> device status BCF_E_NOT_BALANCED.
 *           BCF_PARTITION_LEMMA1: order each 4096-key tile with the Lemma 1
 *           schedule (Sec. 2) on (label, position) items -- row sorts inside
 *           their own banks, conflict-free row/column conversions -- instead of
 *           the rank-and-scatter sweep.  Same (stable) result, slower; its
 *           shared-memory schedule has no bank conflicts.
 *           BCF_PARTITION_DIRECT (w <= 32 only, else BCF_E_UNSUPPORTED; not with
 *           BCF_PARTITION_LEMMA1): every label is its own bank, so ranking keys
 *           per warp and finding their runs touches one word per label; each key
 *           is then stored from its registers straight to its global place
 *           instead of being scattered into label order in shared memory first.
 *           Same result, no bank conflicts in any shared access; its scattered
 *           global stores make it about 1.1x the default at 2^16-2^18 keys and
 *           slower beyond (it suits small partitions).
 *  A label >= w -> device status BCF_E_BAD_KEY.  In place allowed (uses ws).
 * n must be < 2^30. */
int bcf_partition_workspace_size(int64_t n, int w, int val_bytes, int flags, size_t* bytes);
int bcf_partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                  void* vals_out, int64_t n, int w, int val_bytes, int flags, void* ws,
                  size_t ws_bytes, bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Partition by splitters (the pivot bucketing of the sorting problem, Sec. 1: a
 * w-way partition whose labels come from w - 1 pivots): key k goes to bucket
 * b(k) = number of splitters s with s <= k, so bucket b holds the keys in
 * [s[b-1], s[b]).  Stable; keys (and payloads) move, labels are not stored.
 *  splitters  device array of nsplit uint32 values in non-decreasing order
 *             (equal splitters give empty buckets); 0 <= nsplit <= 255, w =
 *             nsplit + 1.  Descending neighbours set device status BCF_E_BAD_KEY
 *             (the output is then unspecified).
 *  flags      BCF_ASSUME_BALANCED: exactly n/w keys per bucket (n % w == 0,
 *             else BCF_E_INVAL; other counts -> BCF_E_NOT_BALANCED).
 *  ws         bcf_partition_splitters_workspace_size() bytes.  In place allowed.
 * n must be < 2^30. */
int bcf_partition_splitters_workspace_size(int64_t n, int nsplit, int val_bytes, int flags, size_t* bytes);
int bcf_partition_splitters(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                            void* vals_out, int64_t n, const uint32_t* splitters, int nsplit,
                            int val_bytes, int flags, void* ws, size_t ws_bytes, bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Permutation (Sec. 1): dst[pi[i]] = src[i] for i in [0, n).
 *  elem_bytes  4 or 8 (bcf_permute); src and dst must not overlap.
 *  row_len     0: pi holds global indices.  > 0: the arrays are rows of row_len
 *              items and pi[i] is local to the row of i (a batch of independent
 *              permutations): dst[row(i)*row_len + pi[i]] = src[i].
 *  flags       BCF_CHECK_PERM: also verify that pi is a bijection (device status
 *              BCF_E_BAD_PERM otherwise).
 *              BCF_PERMUTE_BUCKETED: instead of one scattered store per element
 *              (each costs an L2 sector operation), move the elements in two
 *              coalesced passes: group them by destination block into ws
 *              (blocks of 4096 to 53248 positions, as many as fill whole waves
 *              of one block per SM; tiles of 8192 elements, one global atomic
 *              claim per tile and block), then place each block in shared
 *              memory and write it out in order.  Same result.  Applies to 4-byte elements
 *              with payloads of 0 or 4 bytes and n <= 2^26; otherwise the
 *              one-pass scatter runs.  With a pi that is not a bijection the
 *              output is unspecified (nothing is written outside dst) and, when
 *              the device can tell, BCF_E_BAD_PERM is set.
 *  ws          bcf_permute_workspace_size(n, val_bytes, flags) bytes, 16-byte
 *              aligned (val_bytes 0 for bcf_permute); NULL when that size is 0.
 *              Caller-owned; contents need not be initialised.
 * An index outside its range is never written; it sets BCF_E_BAD_PERM. */
int bcf_permute_workspace_size(int64_t n, int val_bytes, int flags, size_t* bytes);
int bcf_permute(const void* src, void* dst, const uint32_t* pi, int64_t n, int64_t row_len,
                int elem_bytes, int flags, void* ws, size_t ws_bytes, bcf_stream_t stream);
/* Keys and values moved by one pi (val_bytes 0, 4 or 8).  By default the keys
 * and the payloads are scattered in two passes, each of whose outputs stays in
 * L2 while it fills; BCF_PERMUTE_FUSED scatters both in one pass;
 * BCF_PERMUTE_BUCKETED (which takes precedence) moves both through ws in two
 * coalesced passes. */
int bcf_permute_kv(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                   const uint32_t* pi, int64_t n, int64_t row_len, int val_bytes, int flags,
                   void* ws, size_t ws_bytes, bcf_stream_t stream);

/* Tile-local permutation (the paper's permutation problem on one shared-memory
 * matrix, Sec. 3): tile t covers [t*tile, min(n,(t+1)*tile)); the key at local
 * position i moves to local position lpi[t*tile + i].  tile in {1024, 2048, 4096}.
 * flags BCF_TILES_COLOURED selects the randomized colouring schedule of Sec. 3
 * (colour k = (j - h(i)) mod m; conflict-free sends; leftovers retried with a
 * fresh h, then sent one bank at a time), seeded by `seed`; otherwise a direct
 * scatter into shared memory.  With BCF_TILES_COLOURED, BCF_TILES_SORTED_FINISH
 * sends the leftovers as the finishing step of Sec. 3 does instead: sorted by
 * destination (bank, slot), packed into ceil(L/32) columns, and sent in three
 * conflict-free groups (labels whose bank is private to their row; each row's
 * first and last destination banks, the label of slot j in step j).  Results are
 * identical either way.  A local index outside the tile sets BCF_E_BAD_PERM and
 * is not written. */
int bcf_permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi, int64_t n,
                      int tile, int flags, uint64_t seed, bcf_stream_t stream);

/* Gather: dst[i] = src[idx[i]] for i in [0, n); idx[i] < n_src, else the element
 * is not read, dst[i] is 0 and BCF_E_BAD_PERM is set.  row_len > 0: idx[i] is
 * local to the row of i (rows of row_len items in both arrays).  The inverse
 * direction of bcf_permute (the backward pass of a permutation).  elem_bytes 4
 * or 8. */
int bcf_gather(const void* src, void* dst, const uint32_t* idx, int64_t n, int64_t n_src,
               int64_t row_len, int elem_bytes, bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Tile sort (Lemma 1, Sec. 2): each tile of `tile` consecutive keys (the last may
 * be shorter) is sorted on its own, stably, in shared memory, following the
 * Lemma 1 schedule on a 16 x 256 matrix (w*w <= m) -- rows sorted inside their
 * own banks, conflict-free row-major <-> column-major conversions between them.
 * tile must be 4096.  Out of place: outputs must not overlap the inputs. */
int bcf_sort_tiles(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                   void* vals_out, int64_t n, int tile, int val_bytes, bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Lemma 2 (Sec. 2): 0-1 partition of independent w x m matrices, m = 32 and
 * w = m^2 = 1024 rows (the processors, one bank each), 32768 items per matrix.
 * Matrix t holds items [32768 t, 32768 (t+1)); inside it, item k sits in row
 * k mod 1024, column k / 1024 (the column-major layout of Sec. 1).  The output of
 * matrix t is the partitioned matrix read row by row: its 0-labelled items, then
 * its 1-labelled ones.  The order among equal labels is the one Lemma 2's steps
 * produce (balancing, convert and divide, column sorts, shifted square sorts,
 * every sort a stable 0-1 sort of its cells); it is not the input order.
 *  keys_in   labels, 0 or 1 (another value sets BCF_E_BAD_KEY and counts as 1).
 *  vals_in   uint32 payloads, or NULL: item k carries its input position k.
 *  keys_out, vals_out  n entries each; in place allowed (every block reads its
 *            whole matrix before writing it).
 *  n         a multiple of 32768 (BCF_E_INVAL otherwise), below 2^32. */
int bcf_partition_lemma2(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                         uint32_t* vals_out, int64_t n, bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Segmented forms.  offs is a DEVICE array of nseg+1 int64 CSR offsets (offs[0]
 * = 0, nondecreasing, offs[nseg] = n_total).  Each segment is sorted (or
 * partitioned) on its own.  No host synchronisation and no allocation: the whole
 * call can be captured in a CUDA graph.  Segments of at most 4096 keys are
 * sorted whole in shared memory (Lemma 1 tile sort) by persistent blocks that
 * pull them from a queue; longer ones go through digit sweeps whose tiles cover
 * all long segments at once.  Offsets that break the rules set the device status
 * BCF_E_INVAL (the bad segments are skipped).  Out of place only: outputs must
 * not overlap the inputs.  n_total < 2^30. */
int bcf_segmented_sort_workspace_size(int64_t n_total, int64_t nseg, int val_bytes,
                                      int key_bits, size_t* bytes);
int bcf_segmented_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n_total, const int64_t* offs, int64_t nseg,
                       int val_bytes, int key_bits, void* ws, size_t ws_bytes,
                       bcf_stream_t stream);

/* Stable partition of every segment by its labels (the partition problem, Sec. 1,
 * per segment).  w_per_seg: DEVICE int32[nseg], each in 1..256 (else BCF_E_INVAL);
 * the labels of segment s must be < w_per_seg[s] (else the device status
 * BCF_E_BAD_KEY).  flags: BCF_ASSUME_BALANCED -- every label of segment s holds
 * len_s / w_per_seg[s] keys (else BCF_E_NOT_BALANCED).  Every segment, short or
 * long, goes through one label pass whose tiles cover all segments at once, in
 * the pass form the BCF_OP_SEGMENTED_SORT entry names. */
int bcf_segmented_partition_workspace_size(int64_t n_total, int64_t nseg, int val_bytes,
                                           size_t* bytes);
int bcf_segmented_partition(const uint32_t* keys_in, const void* vals_in,
                            uint32_t* keys_out, void* vals_out, int64_t n_total,
                            const int64_t* offs, const int32_t* w_per_seg, int64_t nseg,
                            int val_bytes, int flags, void* ws, size_t ws_bytes,
                            bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Tuning of the sort and partition passes (no counterpart in the paper).  Each
 * digit pass can run with one of bcf_tune_num_configs() configurations: a tile
 * shape (threads per block x keys per thread) and a pass form
 * (bcf_tune_config_form).  Single-launch configurations run every digit pass as
 * one kernel whose tiles find their global offsets by a decoupled look-back,
 * after one histogram read of the keys for all passes; the others run each pass
 * as per-tile digit counts, a scan and then the pass, either with the same pass
 * body or over shared-memory-staged tiles (the staged form runs one look-back
 * sweep launch per pass for n <= 2^18).  The library keeps a small host-side table, per operation and
 * per ceil(log2 n), of the configuration to use; an entry of -1 (the initial
 * state) applies a size rule measured on a B300 (staged sweeps of 2048-key tiles
 * up to n = 2^14, single-launch passes of 2048-key tiles up to 2^18, counts +
 * scan + the pass body of 4096-key tiles above).  The table is process-wide host state and is not synchronised:
 * set it before concurrent calls.  Workspace sizes already cover every
 * configuration.  paper_1507_01391_b300.tune measures the configurations on the
 * device and fills the table (with a text cache per device). */
#define BCF_OP_SORT 0
#define BCF_OP_PARTITION 1
/* Batched sort (bcf_segmented_sort, keyed by ceil(log2 n_total)): its plan cuts
 * the long segments into 4096-key tiles, so only the counts + scan
 * configurations of 256 x 16 apply (bcf_tune_set refuses the others with
 * BCF_E_INVAL); without an entry the long segments' passes use the pass body fed
 * scanned offsets (form 1).  The batched partition (bcf_segmented_partition)
 * takes its pass form from the same entry. */
#define BCF_OP_SEGMENTED_SORT 2
int bcf_tune_num_configs(void);
/* BCF_E_INVAL for an unknown configuration or a null output. */
int bcf_tune_config_info(int config, int* threads, int* keys_per_thread);
/* Pass form of a configuration: 0 single launch per pass (decoupled look-back),
 * 1 per-tile counts + scan + the same pass body, 2 counts + scan + the
 * shared-memory-staged sweep; BCF_E_INVAL for an unknown configuration. */
int bcf_tune_config_form(int config);
/* op in [BCF_OP_SORT, BCF_OP_SEGMENTED_SORT]; config in [-1, num_configs) (for
 * BCF_OP_SEGMENTED_SORT -1 or a 256 x 16 configuration of form 1 or 2); log2_n
 * in [0, 63].  BCF_E_INVAL otherwise. */
int bcf_tune_set(int op, int log2_n, int config);
/* The configuration a call of n keys would use now. */
int bcf_tune_get(int op, int64_t n, int* config);
/* Tuning cache (the library's only persistent state): bcf_tune_save writes the
 * explicit table entries of the current device (keyed "<device name>/<SMs>sm")
 * to the text file `path`, keeping other devices' entries already there;
 * bcf_tune_load applies the current device's entries from `path` (*applied, if
 * not NULL, receives how many).  Host-only; BCF_E_INVAL for an unreadable /
 * unwritable file or a malformed entry, BCF_E_CUDA if the device cannot be
 * queried. */
int bcf_tune_save(const char* path);
int bcf_tune_load(const char* path, int* applied);

/* ---------------------------------------------------------------------------
 * Partition without a workspace.  The paper has no counterpart: this is a
 * calling convention for users who cannot allocate device memory when they call
 * the library -- code running inside CUDA stream capture (cudaMalloc is not
 * allowed while a global-mode capture is active), plugins whose host framework
 * owns all device memory, and latency-critical loops that must never enter the
 * allocator.  Same operation and errors as bcf_partition with the default
 * staged-sweep tile configuration (256 threads x 16 keys, not the tuning table),
 * out of place only (outputs must not overlap the inputs; an overlap returns
 * BCF_E_INVAL), for n <= BCF_NOALLOC_MAX_N (larger n returns BCF_E_UNSUPPORTED).
 * flags: BCF_ASSUME_BALANCED only; any other flag (BCF_PARTITION_LEMMA1 among
 * them) returns BCF_E_UNSUPPORTED.
 * Scratch lives in a fixed device array of about 1 MiB inside libbcf.so, held on
 * every device that loads the library until the process exits; nothing is
 * allocated or freed.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls share the array: each call clears what must start at zero on its
 * stream, and calls whose work overlaps on the GPU (different streams with no
 * ordering between them) race on it. */
#define BCF_NOALLOC_MAX_N (1 << 22)
int bcf_partition_noalloc(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                          void* vals_out, int64_t n, int w, int val_bytes, int flags,
                          bcf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Testing aid for failure detection (no counterpart in the paper).  Inputs of at
 * most 2^18 keys run each sort / partition pass as one sweep launch in which a
 * tile waits, with a bounded number of polls, for the status words its
 * predecessors publish.  After bcf_debug_lookback(t, polls) with t >= 0, tile t of
 * those sweeps publishes nothing and every wait gives up after `polls` polls, so
 * the next call ends with device status BCF_E_TIMEOUT (its output is then
 * unspecified; nothing is written outside the output arrays) instead of hanging.
 * t < 0 restores normal operation.  Host state, not thread-safe; meant for tests.
 * Returns BCF_E_INVAL for polls == 0 with t >= 0. */
int bcf_debug_lookback(int silent_tile, unsigned spin_limit);

#ifdef __cplusplus
}
#endif
#endif /* BCF_H */
