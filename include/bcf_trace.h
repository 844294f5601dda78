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
 *                    3 barrier; width 4, 8 or 16 bytes, 0 for a barrier; site:
 *                    the access site, see trace.cuh)
 * After every block-wide barrier of a traced kernel each warp appends one barrier
 * record (store 3), so a replay can tell which accesses may race: those of
 * different threads to one word between the same two barriers, one a store.
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

#ifdef __cplusplus
}
#endif
#endif /* BCF_TRACE_H */
