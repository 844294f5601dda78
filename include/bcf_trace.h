/*
 * bcf_trace.h -- shared-memory access traces of the tile kernels.
 *
 * Exported only by the trace build of the library (libbcf_trace.so, the same
 * sources compiled with -DBCF_TRACE); the product library libbcf.so has none of
 * this.  While a trace is active, every instrumented shared-memory access of the
 * sweep, tile-permute and Lemma 1 tile-sort kernels appends one 16-byte record
 * per active lane to a caller buffer, so the accesses can be replayed through the
 * bank model of the paper (Sec. 1, "Model of Computation": w banks, at most one
 * access per bank per step) and its bank conflicts counted on the host.
 *
 * Buffer layout (device memory, 16-byte aligned, owned by the caller): a 64-bit
 * record counter, 8 bytes of padding, then records of four uint32:
 *   [0] request id  -- shared by the lanes of one warp-wide access
 *   [1] thread index in the block (lane = low 5 bits) | block index << 16
 *   [2] address     -- byte offset in the block's shared-memory window
 *   [3] width | store << 8 | site << 16   (store: 0 load, 1 store, 2 atomic,
 *                    3 block-wide barrier, 4 warp-wide barrier; width 4, 8 or 16
 *                    bytes, 0 for a barrier; site: the access site, see trace.cuh)
 * After every block-wide barrier of a traced kernel each warp appends one barrier
 * record (store 3), and after a warp-wide barrier the warp appends one (store 4),
 * so a replay can tell which accesses may race: those of different threads to one
 * word between the same two block barriers, one a store, unless both threads are
 * in one warp and a warp barrier lies between the two accesses.
 * The counter keeps counting past the buffer's capacity; records beyond it are
 * dropped.  One trace at a time per process; kernels of other calls that run while
 * it is active are traced too.
 */
#ifndef BCF_TRACE_H
#define BCF_TRACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Start tracing into buf (buf_bytes >= 32).  Synchronous.  BCF_E_INVAL for a null
 * or misaligned buffer, BCF_E_CUDA if the device cannot be reached. */
int bcf_trace_begin(void* buf, size_t buf_bytes);

/* Synchronise the device, stop tracing and report how many records the traced
 * kernels produced (possibly more than fit). */
int bcf_trace_end(uint64_t* records);

/* ---- Bank-conflict probes ----
 * Each probe kernel repeats one shared-memory access pattern of the Lemma 1 tile
 * sort (Sec. 2) on its 64 KB tile (16 x 256 64-bit items, item (r, c) at index
 * c*16 + r: row r in bank pair {2r, 2r+1}), optionally with global traffic issued
 * between its shared accesses, so that a profiler's bank-conflict counters can be
 * read per pattern.  All patterns are conflict-free in the bank model of Sec. 1;
 * the traced copy (traced != 0) records its accesses for the replay while a trace
 * is active, the untraced copy touches global memory only through the traffic
 * asked for and one checksum store per thread. */
#define BCF_PROBE_READOUT 0   /* 64-bit read of Y[t], t lane-contiguous (the write-out) */
#define BCF_PROBE_BUILD 1     /* 64-bit store of X[q], q lane-contiguous (building the items) */
#define BCF_PROBE_ROW_LD 2    /* row sort: 64-bit loads, half-warp lanes on the 16 rows */
#define BCF_PROBE_ROW_ST 3    /* row sort: 64-bit stores to the same cells */
#define BCF_PROBE_CONVERT 4   /* row-major -> column-major along a diagonal (load + store) */
#define BCF_PROBE_MERGE 5     /* merge-path search: any column of the lane's own row */
#define BCF_PROBE_READ32 6    /* 32-bit lane-contiguous reads */
#define BCF_PROBE_FROM_ROWS 7 /* row sort's load fused with a row -> column-major conversion */
#define BCF_PROBE_FROM_COLS 8 /* row sort's load fused with a column -> row-major conversion */
#define BCF_PROBE_PATTERNS 9
#define BCF_PROBE_NONE 0      /* no global traffic beside the pattern */
#define BCF_PROBE_GATHER 1    /* a 4-byte gather from the block's 16 KB of gin, cached in L1 */
#define BCF_PROBE_GATHER_L2 2 /* the same gather from L2 only */
#define BCF_PROBE_STORE 3     /* a lane-contiguous 4-byte store to gout */
#define BCF_PROBE_TRAFFICS 4

/* Launch probe `pattern` with global traffic `traffic` on `blocks` blocks of 256
 * threads (64 KB of dynamic shared memory each), `reps` rounds of 16 accesses per
 * thread, on `stream` (a cudaStream_t; NULL = the legacy default stream).  gin:
 * device, at least blocks*4096 uint32 (the gather source); gout: device, at least
 * blocks*(4096 + 256) uint32 (streaming stores, then one checksum per thread).
 * Asynchronous.  BCF_E_INVAL for an unknown pattern or traffic, a null pointer,
 * blocks outside [1, 65535] or reps < 1; BCF_E_CUDA if the launch fails. */
int bcf_trace_bank_probe(int pattern, int traffic, int traced, const uint32_t* gin, uint32_t* gout,
                         int blocks, int reps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BCF_TRACE_H */
