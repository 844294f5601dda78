// internal.h -- host-side interfaces between the C ABI (abi.cu) and the kernel
// translation units.  Not installed; the public interface is include/bcf.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <algorithm>
#include <stdint.h>

namespace bcf {

// Device status word of the current device (a module variable in abi.cu).
unsigned* status_word();

// Raise a kernel's dynamic shared-memory limit once per device; `done` is the
// caller's per-kernel flag array (one static array per kernel instance).
template <typename K>
inline cudaError_t set_smem_once(K kernel, int bytes, bool (&done)[64]) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (done[dev]) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- digit sweeps
// Tuning of the digit sweep (compile-time; the defaults are the shipped values).
#ifndef BCF_SWEEP_THREADS
#define BCF_SWEEP_THREADS 256
#endif
#ifndef BCF_SWEEP_IPT
#define BCF_SWEEP_IPT 16
#endif
#ifndef BCF_SWEEP_MINBLOCKS
#define BCF_SWEEP_MINBLOCKS 4
#endif
#ifndef BCF_LB_WINDOW
#define BCF_LB_WINDOW 8       // look-back status words read per round trip (multiple of 4)
#endif
#ifndef BCF_PEERS_MATCH
#define BCF_PEERS_MATCH 0     // 1: peers from __match_any_sync, 2: from one shared atomicOr of the
                              // lane bit per key, instead of per-bit ballots (both slower here)
#endif
constexpr int kSweepThreads = BCF_SWEEP_THREADS;
constexpr int kSweepIPT = BCF_SWEEP_IPT;
constexpr int kSweepTile = kSweepThreads * kSweepIPT;  // keys per tile (default configuration)
constexpr int kLookbackWindow = BCF_LB_WINDOW;
static_assert(kLookbackWindow % 4 == 0, "count rows are read and written as 16-byte vectors");

// Configurations of the sort / partition passes that the tuner picks from: a pass
// form and a tile shape (threads per block x keys per thread).
//   0..3   single launch per pass: the digit pass of onesweep.cuh finds its tiles'
//          global offsets by a decoupled look-back (after one histogram read);
//   4..7   the same pass body fed precomputed offsets: per-tile digit counts, a
//          scan, then the pass (reduce-then-scan, no inter-block waits);
//   8..11  reduce-then-scan with the shared-memory-staged digit sweep of
//          sweep.cuh (one look-back sweep launch per pass up to kSmallSweepN).
constexpr int kNumOneConfigs = 4;
constexpr int kNumSweepConfigs = 12;
constexpr int kSweepCfgThreads[kNumSweepConfigs] = {256, 256, 512, 384, 256, 256, 512, 384,
                                                     kSweepThreads, 256, 512, 256};
constexpr int kSweepCfgIPT[kNumSweepConfigs] = {16, 8, 12, 16, 16, 8, 12, 16, kSweepIPT, 4, 16, 8};
// Blocks per SM the onesweep.cuh pass body is compiled for (registers), by shape.
constexpr int kOneCfgMinBlocks[2 * kNumOneConfigs] = {3, 4, 2, 2, 3, 4, 2, 2};
constexpr int kRtsCfg0 = 2 * kNumOneConfigs;  // first configuration of the sweep.cuh passes
// Pass form of a configuration: 0 look-back, 1 offsets + onesweep body, 2 staged sweep.
inline int cfg_form(int cfg) { return cfg < kNumOneConfigs ? 0 : (cfg < kRtsCfg0 ? 1 : 2); }
inline bool cfg_is_onesweep(int cfg) { return cfg >= 0 && cfg < kRtsCfg0; }  // onesweep.cuh body
// Tuning table operations: flat sort, flat partition, batched (segmented) sort.
constexpr int kOpSegmentedSort = 2;
constexpr int kTuneOps = 3;
// The batched sort's plan cuts segments into tiles of kSweepTile keys, so its
// passes take the counts + scan forms of that tile shape only.
inline bool cfg_segment_capable(int cfg) {
  return cfg >= kNumOneConfigs && cfg < kNumSweepConfigs && kSweepCfgThreads[cfg] * kSweepCfgIPT[cfg] == kSweepTile;
}
// Splitter partition: the search's prefix table covers the keys' top 12 bits.
constexpr int kSplitPrefixBits = 12;
constexpr int kSplitPrefixes = 1 << kSplitPrefixBits;
constexpr int kMinSweepTile = 1024;  // smallest tile of any configuration (sizes workspaces)
constexpr int kOneMinTile = 2048;    // smallest tile of the onesweep.cuh configurations
// Inputs up to this size run each sweep.cuh digit pass as one look-back sweep
// launch (fewer launches); larger ones use tile counts + scan + sweep.
constexpr int64_t kSmallSweepN = (int64_t)1 << 18;
inline int sweep_cfg_tile(int cfg) { return kSweepCfgThreads[cfg] * kSweepCfgIPT[cfg]; }

// Tuning table (host state): configuration used by a sort (op 0) or partition
// (op 1) of n keys.  Entries of -1 fall back to a size rule.
int tuned_config(int op, int64_t n);
int tune_set(int op, int log2_n, int cfg);
int tune_entry(int op, int log2_n);  // explicit table entry, -1 if none

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
  size_t hist = 0, counters = 0, lookback = 0, digit_base = 0, status = 0;
  // single-launch passes: two look-back status regions of os_words words each
  // (tile-major, one row of `radix` words per tile), used by alternate passes
  size_t os_status = 0, os_words = 0;
  size_t labels = 0;       // splitter partition: one bucket byte per key
  size_t split_table = 0;  // splitter partition: prefix table of the splitter search
  size_t total = 0;
  int64_t tiles = 0;
  int64_t lb_stride = 0;  // look-back status words per digit (tiles rounded up to 8)
  int radix = 256;
};
// Workspace carve-up; the per-(digit, tile) count buffer is sized for tiles of
// `tile` keys (kMinSweepTile fits every configuration).  `onesweep`: room for the
// look-back status regions of the single-launch configurations.
SweepLayout sweep_layout(int64_t n, int val_bytes, int passes, int radix, bool need_tmp,
                         int tile = kMinSweepTile, bool onesweep = true);

// Three words of a sort's workspace, in the zeroed counter block: which key bits
// vary (OR of the keys, OR of their complements), then the mask of passes that ran.
inline uint32_t* sort_vary_words(unsigned char* ws, const SweepLayout& L) {
  return reinterpret_cast<uint32_t*>(ws + L.counters) + 5;
}
// Passes the last sort in ws ran; syncs the stream.  Returns a cudaError_t value.
int sort_passes_run(const unsigned char* ws, const SweepLayout& L, const PassPlan& plan, cudaStream_t s,
                    int* out);

// Radix sort launch sequence (see bcf_sort in include/bcf.h).
// `cfg` is a sweep configuration whose tiles fit the layout's count buffer.
cudaError_t radix_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n, int val_bytes, const PassPlan& plan,
                       unsigned char* ws, const SweepLayout& L, cudaStream_t s, int cfg = 0);

// Single-pass stable partition by label (see bcf_partition).
cudaError_t partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                      void* vals_out, int64_t n, int w, int val_bytes, bool balanced,
                      unsigned char* ws, const SweepLayout& L, cudaStream_t s, int cfg = 0,
                      bool direct = false);

// Partition with the Lemma 1 tile schedule (BCF_PARTITION_LEMMA1); same layout.
cudaError_t partition_lemma1(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                             void* vals_out, int64_t n, int w, int val_bytes, bool balanced,
                             unsigned char* ws, const SweepLayout& L, cudaStream_t s);

// ---------------------------------------------------------------- permutations
cudaError_t permute(const void* src_k, const void* src_v, void* dst_k, void* dst_v,
                    const uint32_t* pi, int64_t n, int64_t row_len, int kbytes, int vbytes,
                    uint32_t* seen_bitmap, bool fused, cudaStream_t s);
// w-way partition by w - 1 ascending splitters (radix.cu).
cudaError_t partition_splitters(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                                void* vals_out, int64_t n, const uint32_t* splitters, int nsplit, int vb,
                                bool balanced, unsigned char* ws, const SweepLayout& L, cudaStream_t s);
// Testing aid for the bounded look-back waits (radix.cu).
void debug_lookback(int silent_tile, unsigned spin_limit);
// Two-pass bucketed permutation (permute_bucketed.cu).
bool permute_bucketed_supported(int64_t n, int kb, int vb);
size_t permute_bucketed_workspace(int64_t n, int vb);
cudaError_t permute_bucketed(const uint32_t* sk, const uint32_t* sv, uint32_t* dk, uint32_t* dv,
                             const uint32_t* pi, int64_t n, int64_t row_len, int vb, bool check,
                             unsigned char* ws, cudaStream_t s);
cudaError_t gather(const void* src, void* dst, const uint32_t* idx, int64_t n, int64_t n_src,
                   int64_t row_len, int elem_bytes, cudaStream_t s);
cudaError_t permute_tiles(const uint32_t* src, uint32_t* dst, const uint16_t* lpi, int64_t n,
                          int tile, bool coloured, bool sorted_finish, uint64_t seed, cudaStream_t s);

// ---------------------------------------------------------------- segments
struct SegLayout {
  int small_max = 0;        // segments of 1..small_max keys take the small path
  int64_t slots_cap = 0;    // capacity for long segments
  int64_t tiles_cap = 0;    // capacity for sweep tiles of long segments
  int64_t lb_stride = 0;    // look-back status words per digit
  int passes = 0;
  size_t keys_tmp = 0, vals_tmp = 0, small_ids = 0, seg_slot = 0, seg_tile0 = 0, slot_seg = 0;
  size_t tiny_ids = 0, bin_first = 0;  // tiny segments packed several to a tile
  size_t tile_seg = 0, seg_base = 0, ctr = 0, lookback = 0;
  size_t zero_begin = 0, zero_bytes = 0, total = 0;
};
SegLayout seg_layout(int64_t n_total, int64_t nseg, int val_bytes, int passes, bool sort);

cudaError_t segmented_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                           void* vals_out, int64_t n_total, const int64_t* offs, int64_t nseg,
                           int val_bytes, const PassPlan& plan, unsigned char* ws,
                           const SegLayout& L, cudaStream_t s);
cudaError_t segmented_partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                                void* vals_out, int64_t n_total, const int64_t* offs,
                                const int32_t* w_per_seg, int64_t nseg, int val_bytes,
                                bool balanced, unsigned char* ws, const SegLayout& L,
                                cudaStream_t s);
cudaError_t sort_tiles(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n, int val_bytes, cudaStream_t s);

// Lemma 2's 0-1 partition of independent 1024 x 32 matrices (n a multiple of 32768).
cudaError_t partition_lemma2(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out, uint32_t* vals_out,
                             int64_t n, cudaStream_t s);
// Number of SMs of the current device (cached per device).
int sm_count_cached();

}  // namespace bcf
