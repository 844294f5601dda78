// radix.cu -- host launch sequences of the LSD radix sort and the w-way partition
// (the sweep kernel itself is in sweep.cuh).
#include "common.cuh"
#include "internal.h"
#include "onesweep.cuh"
#include "sweep.cuh"

namespace bcf {

// ------------------------------------------------------------- host side
// Passes of 8-bit digits from the least significant end: digit q is key byte q.
// A key width that is not a multiple of 8 leaves the top pass with fewer varying
// bits (keys are below 2^key_bits, so the byte's upper bits are zero); the digit
// stays a whole byte, which the pass body takes with one byte permute.
PassPlan plan_passes(int key_bits) {
  PassPlan pl;
  pl.passes = (key_bits + 7) / 8;
  for (int q = 0; q < pl.passes; ++q) {
    pl.shift[q] = 8 * q;
    pl.nbits[q] = 8;
  }
  return pl;
}

// ------------------------------------------------------------- tuning table
namespace {
int8_t g_tune[kTuneOps][64];  // [op][log2 n]: configuration, -1 = size rule
bool g_tune_init = false;

void tune_init() {
  if (g_tune_init) return;
  for (int op = 0; op < kTuneOps; ++op)
    for (int b = 0; b < 64; ++b) g_tune[op][b] = -1;
  g_tune_init = true;
}

int ilog2_ceil(int64_t n) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < n) ++b;
  return b;
}
}  // namespace

int tuned_config(int op, int64_t n) {
  tune_init();
  const int b = ilog2_ceil(n);
  const int cfg = (op >= 0 && op < kTuneOps) ? g_tune[op][b] : -1;
  if (cfg >= 0 && cfg < kNumSweepConfigs) return cfg;
  // Batched sorts: the long segments' passes with the pass body fed scanned
  // offsets (measured faster than the staged sweep on the 10,000-segment batch).
  if (op == kOpSegmentedSort) return kNumOneConfigs;
  // Size rule (measured on a B300 by the tuner, sorts and balanced 256-way
  // partitions alike): up to 2^14 keys the staged look-back sweep of 2048-key
  // tiles; up to 2^18 single-launch passes of 2048-key tiles (fewest launches);
  // above, counts + scan + the pass body of 4096-key tiles.
  if (n <= ((int64_t)1 << 14)) return kRtsCfg0 + 3;
  if (n <= ((int64_t)1 << 18)) return 1;
  return kNumOneConfigs;
}

int tune_set(int op, int log2_n, int cfg) {
  tune_init();
  if (op < 0 || op >= kTuneOps || log2_n < 0 || log2_n >= 64 || cfg < -1 || cfg >= kNumSweepConfigs) return -1;
  if (op == kOpSegmentedSort && cfg >= 0 && !cfg_segment_capable(cfg)) return -1;
  g_tune[op][log2_n] = (int8_t)cfg;
  return 0;
}

int tune_entry(int op, int log2_n) {
  tune_init();
  if (op < 0 || op >= kTuneOps || log2_n < 0 || log2_n >= 64) return -1;
  return g_tune[op][log2_n];
}

SweepLayout sweep_layout(int64_t n, int val_bytes, int passes, int radix, bool need_tmp, int tile,
                         bool onesweep) {
  SweepLayout L;
  L.radix = radix;
  L.tiles = (n + tile - 1) / tile;
  L.lb_stride = (L.tiles + kLookbackWindow) / kLookbackWindow * kLookbackWindow;  // > tiles
  size_t off = 0;
  if (need_tmp) {
    L.keys_tmp = off;
    off = align_up(off + (size_t)n * 4);
    L.vals_tmp = off;
    off = align_up(off + (size_t)n * val_bytes);
  }
  L.digit_base = off;  // small inputs: global digit starts from k_histogram
  off = align_up(off + 4 * 256 * 4);
  L.zero_begin = off;
  L.hist = off;  // per-pass digit totals
  off = align_up(off + 4 * 256 * 4);
  L.counters = off;  // small inputs: tile tickets per pass + histogram done flag
  off = align_up(off + 8 * 4);
  L.status = off;  // small inputs: look-back status words, one region per pass
  if (n <= kSmallSweepN) off = align_up(off + (size_t)(passes > 0 ? passes : 1) * L.lb_stride * radix * 4);
  L.zero_bytes = off - L.zero_begin;
  L.lookback = off;  // per-(digit, tile) counts, scanned in place into run starts
  off = align_up(off + (size_t)L.lb_stride * radix * 4);
  if (onesweep) {  // look-back status of the single-launch passes, two regions
    L.os_status = off;
    L.os_words = (size_t)((n + kOneMinTile - 1) / kOneMinTile) * radix;
    off = align_up(off + 2 * L.os_words * 4);
  }
  L.total = off;
  return L;
}

// One digit pass, reduce-then-scan: tile counts -> run starts -> sweep, with
// tiles of THREADS x IPT keys.
template <int BITS, int THREADS, int IPT>
static cudaError_t pass_t(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                          int64_t n, int vb, int shift, int nbits, int w, bool balanced,
                          uint32_t* totals, uint32_t* offsets, cudaStream_t s, const PassSel& sel) {
  constexpr int RADIX = 1 << BITS;
  constexpr int T = THREADS * IPT;
  SweepLayout L;  // this configuration's tile count and status stride
  L.tiles = (n + T - 1) / T;
  L.lb_stride = (L.tiles + kLookbackWindow) / kLookbackWindow * kLookbackWindow;  // > tiles
  CountParams cp{};
  cp.keys = src_k;
  cp.n = n;
  cp.shift = shift;
  cp.nbits = nbits;
  cp.label_bits = w > 0 ? BITS : 0;
  cp.counts = offsets;
  cp.stride = L.lb_stride;
  cp.totals = totals;
  cp.sel = sel;
  const int64_t count_blocks = (L.tiles + kCountTilesPerBlock - 1) / kCountTilesPerBlock;
  k_tile_counts<BITS, T><<<(unsigned)count_blocks, 256, 0, s>>>(cp, L.tiles);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  launch_scan_offsets(RADIX, offsets, L.tiles, L.lb_stride, totals, balanced ? 1 : 0, n, w > 0 ? w : 1,
                      status_word(), s, sel);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  SweepParams sp{};
  sp.keys_in = src_k;
  sp.vals_in = src_v;
  sp.keys_out = dst_k;
  sp.vals_out = dst_v;
  sp.n = n;
  sp.shift = shift;
  sp.nbits = nbits;
  sp.w = w;
  sp.balanced = balanced ? 1 : 0;
  sp.lb_stride = L.lb_stride;
  sp.tile_offsets = offsets;
  sp.status = status_word();
  sp.sel = sel;
  return sweep_dispatch<BITS, THREADS, IPT>(sp, L.tiles, vb, s);
}

template <int BITS>
static cudaError_t pass(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                       int64_t n, int vb, int shift, int nbits, int w, bool balanced,
                       uint32_t* totals, uint32_t* offsets, cudaStream_t s, int cfg,
                       const PassSel& sel = PassSel{}) {
  switch (cfg) {
#define BCF_PASS(C)                                                                                  \
  case C:                                                                                            \
    return pass_t<BITS, kSweepCfgThreads[C], kSweepCfgIPT[C]>(src_k, src_v, dst_k, dst_v, n, vb, shift, \
                                                              nbits, w, balanced, totals, offsets, s, sel);
    BCF_PASS(8)
    BCF_PASS(9)
    BCF_PASS(10)
    BCF_PASS(11)
#undef BCF_PASS
  }
  return cudaErrorInvalidValue;
}

// Testing aid (bcf_debug_lookback): the look-back sweeps leave one tile silent and
// give up waiting after a short poll count.
namespace {
int g_silent_tile1 = 0;
unsigned g_spin_limit = 0;
}  // namespace
void debug_lookback(int silent_tile, unsigned spin_limit) {
  g_silent_tile1 = silent_tile >= 0 ? silent_tile + 1 : 0;
  g_spin_limit = silent_tile >= 0 ? spin_limit : 0;
}

// Small inputs: one sweep launch per pass with a decoupled look-back over at most
// kSmallSweepN / kMinSweepTile tiles, after one histogram read for all passes
// (skipped for balanced partitions, whose digit starts are closed-form).
template <int BITS, int THREADS, int IPT>
static cudaError_t lookback_pass_t(const uint32_t* src_k, const void* src_v, uint32_t* dst_k,
                                   void* dst_v, int64_t n, int vb, int shift, int w, bool balanced,
                                   const uint32_t* digit_base, uint32_t* status, uint32_t* ticket,
                                   cudaStream_t s, const PassSel& sel) {
  constexpr int T = THREADS * IPT;
  const int64_t tiles = (n + T - 1) / T;
  SweepParams sp{};
  sp.keys_in = src_k;
  sp.vals_in = src_v;
  sp.keys_out = dst_k;
  sp.vals_out = dst_v;
  sp.n = n;
  sp.shift = shift;
  sp.nbits = BITS;
  sp.w = w;
  sp.balanced = balanced ? 1 : 0;
  sp.digit_base = digit_base;
  sp.lookback = status;
  sp.lb_stride = (tiles + kLookbackWindow) / kLookbackWindow * kLookbackWindow;
  sp.ticket = ticket;
  sp.status = status_word();
  sp.spin_limit = g_spin_limit;
  sp.silent_tile1 = g_silent_tile1;
  sp.sel = sel;
  return sweep_dispatch<BITS, THREADS, IPT>(sp, tiles, vb, s);
}

template <int BITS>
static cudaError_t lookback_pass(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                                 int64_t n, int vb, int shift, int w, bool balanced,
                                 const uint32_t* digit_base, uint32_t* status, uint32_t* ticket,
                                 cudaStream_t s, int cfg, const PassSel& sel = PassSel{}) {
  switch (cfg) {
#define BCF_LBP(C)                                                                                     \
  case C:                                                                                              \
    return lookback_pass_t<BITS, kSweepCfgThreads[C], kSweepCfgIPT[C]>(src_k, src_v, dst_k, dst_v, n, vb, \
                                                                       shift, w, balanced, digit_base,   \
                                                                       status, ticket, s, sel);
    BCF_LBP(8)
    BCF_LBP(9)
    BCF_LBP(10)
    BCF_LBP(11)
#undef BCF_LBP
  }
  return cudaErrorInvalidValue;
}

static cudaError_t small_histogram(const uint32_t* keys, int64_t n, int passes, const int* shift,
                                   int label_bits, unsigned char* ws, const SweepLayout& L, cudaStream_t s,
                                   uint32_t* vary = nullptr) {
  HistParams hp{};
  hp.vary = vary;
  hp.keys = keys;
  hp.n = n;
  hp.passes = passes;
  for (int q = 0; q < 4; ++q) {
    hp.shift[q] = q < passes ? shift[q] : 0;
    hp.nbits[q] = 8;
  }
  hp.label_bits = label_bits;
  hp.hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  hp.digit_base = reinterpret_cast<uint32_t*>(ws + L.digit_base);
  hp.done = reinterpret_cast<uint32_t*>(ws + L.counters) + 4;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n / 4 + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 2));
  k_histogram<256><<<grid, 256, 0, s>>>(hp);
  return cudaGetLastError();
}

// ------------------------------------------------------------- single-launch passes
// One digit pass of configuration cfg (0..kNumOneConfigs-1): a launch of
// k_onesweep over ceil(n / tile) blocks.
template <int BITS, int THREADS, int IPT, int MINB>
static cudaError_t onesweep_pass_t(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                                   int64_t n, int vb, int shift, int w, bool balanced,
                                   const uint32_t* digit_base, uint32_t* status, uint32_t* zero_next,
                                   uint32_t* ticket, cudaStream_t s, const PassSel& sel,
                                   uint32_t* totals = nullptr, uint32_t* offsets = nullptr,
                                   bool direct = false) {
  constexpr int T = THREADS * IPT;
  OneSweepParams op{};
  op.direct = direct ? 1 : 0;
  if (offsets) {  // reduce-then-scan: per-tile counts and their scan first
    constexpr int RADIX = 1 << BITS;
    const int64_t tiles = (n + T - 1) / T;
    const int64_t stride = (tiles + kLookbackWindow) / kLookbackWindow * kLookbackWindow;  // > tiles
    CountParams cp{};
    cp.keys = src_k;
    cp.n = n;
    cp.shift = shift;
    cp.nbits = BITS;
    cp.label_bits = w > 0 ? BITS : 0;
    cp.counts = offsets;
    cp.stride = stride;
    cp.totals = totals;
    cp.sel = sel;
    const int64_t count_blocks = (tiles + kCountTilesPerBlock - 1) / kCountTilesPerBlock;
    k_tile_counts<BITS, T><<<(unsigned)count_blocks, 256, 0, s>>>(cp, tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launch_scan_offsets(RADIX, offsets, tiles, stride, totals, balanced ? 1 : 0, n, w > 0 ? w : 1,
                        status_word(), s, sel);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    op.tile_offsets = offsets;
    op.offs_stride = stride;
  }
  op.keys_in = src_k;
  op.vals_in = src_v;
  op.keys_out = dst_k;
  op.vals_out = dst_v;
  op.n = n;
  op.shift = shift;
  op.w = w;
  op.balanced = balanced ? 1 : 0;
  op.digit_base = digit_base;
  op.status = status;
  op.zero_next = zero_next;
  op.ticket = ticket;
  op.err = status_word();
  op.spin_limit = g_spin_limit;
  op.silent_tile1 = g_silent_tile1;
  op.sel = sel;
  return onesweep_dispatch<BITS, THREADS, IPT, MINB>(op, (n + T - 1) / T, vb, s);
}

// Configurations 0..3: look-back passes; 4..7: the same shapes fed by counts +
// scan (totals and offsets given).
template <int BITS>
static cudaError_t onesweep_pass(const uint32_t* src_k, const void* src_v, uint32_t* dst_k, void* dst_v,
                                 int64_t n, int vb, int shift, int w, bool balanced, const uint32_t* digit_base,
                                 uint32_t* status, uint32_t* zero_next, uint32_t* ticket, cudaStream_t s,
                                 int cfg, const PassSel& sel = PassSel{}, uint32_t* totals = nullptr,
                                 uint32_t* offsets = nullptr, bool direct = false) {
  const bool rts = cfg >= kNumOneConfigs;
  switch (cfg % kNumOneConfigs) {
#define BCF_OSP(C)                                                                                         \
  case C:                                                                                                  \
    return onesweep_pass_t<BITS, kSweepCfgThreads[C], kSweepCfgIPT[C], kOneCfgMinBlocks[C]>(             \
        src_k, src_v, dst_k, dst_v, n, vb, shift, w, balanced, digit_base, status, zero_next, ticket, s, sel, \
        rts ? totals : nullptr, rts ? offsets : nullptr, direct);
    BCF_OSP(0)
    BCF_OSP(1)
    BCF_OSP(2)
    BCF_OSP(3)
#undef BCF_OSP
  }
  return cudaErrorInvalidValue;
}

// Look-back rows (tiles) of a single-launch configuration.
static inline int64_t os_rows(int64_t n, int cfg) {
  const int64_t t = sweep_cfg_tile(cfg);
  return (n + t - 1) / t;
}

// One read of the keys counts the digits of every pass (8-bit digits at `shift`),
// turns the counts into exclusive digit starts (L.digit_base) and clears the
// first pass's look-back status region.
static cudaError_t onesweep_histogram(const uint32_t* keys, int64_t n, int passes, const int* shift,
                                      unsigned char* ws, const SweepLayout& L, cudaStream_t s,
                                      uint32_t* vary, int cfg) {
  OneHistParams hp{};
  hp.keys = keys;
  hp.n = n;
  hp.passes = passes;
  for (int q = 0; q < 4; ++q) hp.shift[q] = q < passes ? shift[q] : 0;
  hp.hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  hp.digit_base = reinterpret_cast<uint32_t*>(ws + L.digit_base);
  hp.done = reinterpret_cast<uint32_t*>(ws + L.counters) + 4;
  hp.vary = vary;
  hp.zero = reinterpret_cast<uint32_t*>(ws + L.os_status);
  hp.zero_words = os_rows(n, cfg) * L.radix;  // the rows configuration cfg uses
  bool bytes = true;  // digits are whole key bytes from byte 0 up
  for (int q = 0; q < passes; ++q) bytes &= shift[q] == 8 * q;
  static bool attr_b[64] = {false}, attr_g[64] = {false};
  const int smem = (int)onesweep_hist_smem(4);
  cudaError_t e = bytes ? set_smem_once(k_onesweep_hist<true>, smem, attr_b)
                        : set_smem_once(k_onesweep_hist<false>, smem, attr_g);
  if (e != cudaSuccess) return e;
  const int64_t per_block = (int64_t)kHistThreads * 4 * kHistUnroll;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, sm_count_cached()));
  if (bytes) k_onesweep_hist<true><<<grid, kHistThreads, onesweep_hist_smem(passes), s>>>(hp);
  else k_onesweep_hist<false><<<grid, kHistThreads, onesweep_hist_smem(passes), s>>>(hp);
  return cudaGetLastError();
}

static inline uint32_t* os_region(unsigned char* ws, const SweepLayout& L, int q) {
  return reinterpret_cast<uint32_t*>(ws + L.os_status) + (size_t)(q & 1) * L.os_words;
}

// In-place sorts only.  An odd number of passes that ran leaves the result in the
// temporary: copy it home.  With no pass run the keys are already in place, and
// only a position payload (no payload input) remains to be written.
__global__ void __launch_bounds__(256) k_pass_copy(PassSel sel, int64_t n, int vb) {
  const int k = __popc(passes_run_mask(sel, vary_bits(sel)));
  const bool from_tmp = (k & 1) != 0;
  const bool iota = k == 0 && vb == 4 && sel.v_in == nullptr;
  if (!from_tmp && !iota) return;
  const uint32_t* sk = from_tmp ? sel.k_tmp : nullptr;
  const unsigned char* sv = from_tmp ? static_cast<const unsigned char*>(sel.v_tmp) : nullptr;
  unsigned char* dv = static_cast<unsigned char*>(sel.v_out);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = n / 4;  // groups of four elements: 16-byte keys, 16 or 32 bytes of payload
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += stride) {
    if (sk) reinterpret_cast<uint4*>(sel.k_out)[g] = reinterpret_cast<const uint4*>(sk)[g];
    if (vb == 0) continue;
    if (iota) {
      const uint32_t i = (uint32_t)(g * 4);
      reinterpret_cast<uint4*>(dv)[g] = make_uint4(i, i + 1, i + 2, i + 3);
    } else if (sv) {
      for (int h = 0; h < vb / 4; ++h)
        reinterpret_cast<uint4*>(dv)[g * (vb / 4) + h] = reinterpret_cast<const uint4*>(sv)[g * (vb / 4) + h];
    }
  }
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (sk) sel.k_out[i] = sk[i];
    if (vb == 4 && iota) reinterpret_cast<uint32_t*>(dv)[i] = (uint32_t)i;
    else if (vb == 4 && sv) reinterpret_cast<uint32_t*>(dv)[i] = reinterpret_cast<const uint32_t*>(sv)[i];
    else if (vb == 8 && sv)
      reinterpret_cast<unsigned long long*>(dv)[i] = reinterpret_cast<const unsigned long long*>(sv)[i];
  }
}

cudaError_t radix_sort(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                       void* vals_out, int64_t n, int vb, const PassPlan& plan,
                       unsigned char* ws, const SweepLayout& L, cudaStream_t s, int cfg) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* kt = reinterpret_cast<uint32_t*>(ws + L.keys_tmp);
  void* vt = vb ? (void*)(ws + L.vals_tmp) : nullptr;
  const int P = plan.passes;
  // Which passes run, and the buffers of each, are settled on the device (PassSel).
  PassSel sel;
  sel.vary = sort_vary_words(ws, L);
  sel.ran = sort_vary_words(ws, L) + 2;
  sel.passes = P;
  sel.in_place = keys_in == keys_out;
  for (int q = 0; q < P; ++q) sel.shift[q] = plan.shift[q];
  sel.k_in = keys_in;
  sel.v_in = vals_in;
  sel.k_out = keys_out;
  sel.v_out = vals_out;
  sel.k_tmp = kt;
  sel.v_tmp = vt;
  const bool one = cfg_is_onesweep(cfg);
  const bool small = !one && n <= kSmallSweepN;
  if (cfg_form(cfg) == 0 && (e = onesweep_histogram(keys_in, n, P, plan.shift, ws, L, s, sel.vary, cfg)) != cudaSuccess)
    return e;
  if (small && (e = small_histogram(keys_in, n, P, plan.shift, 0, ws, L, s, sel.vary)) != cudaSuccess) return e;
  uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(ws + L.lookback);
  // The buffers passed down are those of the case in which every pass runs (the
  // kernels switch only when the device finds a skipped pass before theirs).
  const bool odd_in_place = sel.in_place && (P % 2 == 1);
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  for (int q = 0; q < P; ++q) {
    sel.q = q;
    const bool to_out = odd_in_place ? (q % 2 == 1) : (((P - 1 - q) % 2) == 0);
    uint32_t* dk = to_out ? keys_out : kt;
    void* dv = to_out ? vals_out : vt;
    if (one) {
      e = onesweep_pass<8>(src_k, src_v, dk, dv, n, vb, plan.shift[q], 0, false,
                           reinterpret_cast<uint32_t*>(ws + L.digit_base) + q * 256, os_region(ws, L, q),
                           q + 1 < P ? os_region(ws, L, q + 1) : nullptr,
                           reinterpret_cast<uint32_t*>(ws + L.counters) + q, s, cfg, sel, totals + q * 256, offsets);
    } else if (small) {
      e = lookback_pass<8>(src_k, src_v, dk, dv, n, vb, plan.shift[q], 0, false,
                           reinterpret_cast<uint32_t*>(ws + L.digit_base) + q * 256,
                           reinterpret_cast<uint32_t*>(ws + L.status) + (size_t)q * L.lb_stride * 256,
                           reinterpret_cast<uint32_t*>(ws + L.counters) + q, s, cfg, sel);
    } else {
      e = pass<8>(src_k, src_v, dk, dv, n, vb, plan.shift[q], plan.nbits[q], 0, false, totals + q * 256,
                  offsets, s, cfg, sel);
    }
    if (e != cudaSuccess) return e;
    src_k = dk;
    src_v = dv;
  }
  if (!sel.in_place) return cudaSuccess;  // out of place the last pass that runs writes the output
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n / 4 + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  k_pass_copy<<<grid, 256, 0, s>>>(sel, n, vb);
  return cudaGetLastError();
}

int sort_passes_run(const unsigned char* ws, const SweepLayout& L, const PassPlan& plan, cudaStream_t s,
                    int* out) {
  uint32_t ran = 0;
  cudaError_t e = cudaMemcpyAsync(&ran, sort_vary_words(const_cast<unsigned char*>(ws), L) + 2, sizeof ran,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return (int)e;
  int k = 0;
  for (int q = 0; q < plan.passes; ++q) k += (ran >> q) & 1u;
  *out = k;
  return 0;
}

cudaError_t partition(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                      void* vals_out, int64_t n, int w, int vb, bool balanced,
                      unsigned char* ws, const SweepLayout& L, cudaStream_t s, int cfg, bool direct) {
  if (n == 0) return cudaSuccess;
  // The direct write-out exists in the pass body only (a partition by at most 32
  // labels): take its single-launch or counts + scan form of the same size class.
  if (direct && !cfg_is_onesweep(cfg)) cfg = n <= kSmallSweepN ? 1 : kNumOneConfigs;
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(ws + L.lookback);
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  if (keys_in == keys_out) {  // in place: sweep from a copy of the input
    uint32_t* kt = reinterpret_cast<uint32_t*>(ws + L.keys_tmp);
    if ((e = cudaMemcpyAsync(kt, keys_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    src_k = kt;
    if (vb && vals_in) {
      void* vt = ws + L.vals_tmp;
      if ((e = cudaMemcpyAsync(vt, vals_in, (size_t)n * vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
      src_v = vt;
    }
  }
  if (cfg_is_onesweep(cfg)) {
    // Look-back form: balanced partitions have closed-form label starts and only
    // the status region to clear; otherwise one histogram read gives the label
    // starts and clears it.  Offsets form: counts + scan (which checks balance).
    const int zero = 0;
    if (cfg_form(cfg) == 0) {
      if (balanced) e = cudaMemsetAsync(ws + L.os_status, 0, (size_t)os_rows(n, cfg) * L.radix * 4, s);
      else e = onesweep_histogram(src_k, n, 1, &zero, ws, L, s, nullptr, cfg);
      if (e != cudaSuccess) return e;
    }
    uint32_t* base = reinterpret_cast<uint32_t*>(ws + L.digit_base);
    uint32_t* ticket = reinterpret_cast<uint32_t*>(ws + L.counters);
    if (L.radix == 32)  // at most 32 labels: each label its own bank
      return onesweep_pass<5>(src_k, src_v, keys_out, vals_out, n, vb, 0, w, balanced, base, os_region(ws, L, 0),
                              nullptr, ticket, s, cfg, PassSel{}, totals, offsets, direct);
    return onesweep_pass<8>(src_k, src_v, keys_out, vals_out, n, vb, 0, w, balanced, base, os_region(ws, L, 0),
                            nullptr, ticket, s, cfg, PassSel{}, totals, offsets);
  }
  if (n <= kSmallSweepN) {
    const int bits = L.radix == 32 ? 5 : 8;
    const int zero = 0;
    if (!balanced && (e = small_histogram(src_k, n, 1, &zero, bits, ws, L, s)) != cudaSuccess) return e;
    uint32_t* base = reinterpret_cast<uint32_t*>(ws + L.digit_base);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.status);
    uint32_t* ticket = reinterpret_cast<uint32_t*>(ws + L.counters);
    if (bits == 5)
      return lookback_pass<5>(src_k, src_v, keys_out, vals_out, n, vb, 0, w, balanced, base, status, ticket, s, cfg);
    return lookback_pass<8>(src_k, src_v, keys_out, vals_out, n, vb, 0, w, balanced, base, status, ticket, s, cfg);
  }
  if (L.radix == 32)
    return pass<5>(src_k, src_v, keys_out, vals_out, n, vb, 0, 5, w, balanced, totals, offsets, s, cfg);
  return pass<8>(src_k, src_v, keys_out, vals_out, n, vb, 0, 8, w, balanced, totals, offsets, s, cfg);
}

// w-way partition by w - 1 splitters (sample-sort bucketing): one reduce-then-scan
// pass whose digit is the number of splitters <= key, default tile configuration.
// The prefix table of split_bucket (one block of 256 threads), built from the
// ascending splitters: the window (first splitter, shift), the counts of splitters
// per prefix, then their exclusive scan.  The entries are followed by the window's
// two words.  A descending pair of splitters is flagged in the status word (the
// prefixes are clamped, so such a table stays in bounds).
__global__ void __launch_bounds__(256) k_split_table(const uint32_t* __restrict__ spl, int nsplit,
                                                     uint16_t* __restrict__ table, unsigned* status) {
  constexpr int PER = kSplitPrefixes / 256;
  __shared__ uint32_t cnt[kSplitPrefixes];
  __shared__ uint32_t scratch[32];
  const int tid = threadIdx.x;
  const uint32_t base = nsplit ? spl[0] : 0u;
  const uint32_t range = nsplit ? spl[nsplit - 1] - base : 0u;
  const uint32_t sh = (uint32_t)max(0, (32 - __clz(range)) - kSplitPrefixBits);  // range >> sh < 2^12
  for (int i = tid; i < kSplitPrefixes; i += 256) cnt[i] = 0;
  BCF_SYNC();
  for (int i = tid; i < nsplit; i += 256) {
    const uint32_t v = spl[i];
    atomicAdd(&cnt[min((v - base) >> sh, (uint32_t)(kSplitPrefixes - 1))], 1u);
    if (i > 0 && spl[i - 1] > v) set_status(status, DEV_BAD_KEY);
  }
  BCF_SYNC();
  uint32_t c[PER], sum = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    c[j] = cnt[tid * PER + j];
    sum += c[j];
  }
  uint32_t total;
  uint32_t lo = block_excl_scan<256>(sum, scratch, &total);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    table[tid * PER + j] = (uint16_t)(lo | ((lo + c[j]) << 8));  // nsplit <= 255: both fit a byte
    lo += c[j];
  }
  if (tid == 0) {
    reinterpret_cast<uint32_t*>(table + kSplitPrefixes)[0] = base;
    reinterpret_cast<uint32_t*>(table + kSplitPrefixes)[1] = sh;
  }
}

cudaError_t partition_splitters(const uint32_t* keys_in, const void* vals_in, uint32_t* keys_out,
                                void* vals_out, int64_t n, const uint32_t* splitters, int nsplit, int vb,
                                bool balanced, unsigned char* ws, const SweepLayout& L, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  constexpr int THREADS = kSweepCfgThreads[kRtsCfg0], IPT = kSweepCfgIPT[kRtsCfg0], T = THREADS * IPT;
  cudaError_t e = cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(ws + L.lookback);
  const uint32_t* src_k = keys_in;
  const void* src_v = vals_in;
  if (keys_in == keys_out) {  // in place: sweep from a copy of the input
    uint32_t* kt = reinterpret_cast<uint32_t*>(ws + L.keys_tmp);
    if ((e = cudaMemcpyAsync(kt, keys_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    src_k = kt;
    if (vb && vals_in) {
      void* vt = ws + L.vals_tmp;
      if ((e = cudaMemcpyAsync(vt, vals_in, (size_t)n * vb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
      src_v = vt;
    }
  }
  const int64_t tiles = (n + T - 1) / T;
  const int64_t stride = (tiles + kLookbackWindow) / kLookbackWindow * kLookbackWindow;  // > tiles
  CountParams cp{};
  cp.keys = src_k;
  cp.n = n;
  cp.counts = offsets;
  cp.stride = stride;
  cp.totals = totals;
  cp.splitters = splitters;
  cp.nsplit = nsplit;
  cp.split_table = reinterpret_cast<const uint16_t*>(ws + L.split_table);
  cp.labels = ws + L.labels;
  k_split_table<<<1, 256, 0, s>>>(splitters, nsplit, reinterpret_cast<uint16_t*>(ws + L.split_table), status_word());
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t count_blocks = (tiles + kCountTilesPerBlock - 1) / kCountTilesPerBlock;
  k_tile_counts<8, T, true><<<(unsigned)count_blocks, 256, 0, s>>>(cp, tiles);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  launch_scan_offsets(256, offsets, tiles, stride, totals, balanced ? 1 : 0, n, nsplit + 1, status_word(), s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  SweepParams sp{};
  sp.keys_in = src_k;
  sp.vals_in = src_v;
  sp.keys_out = keys_out;
  sp.vals_out = vals_out;
  sp.n = n;
  sp.nbits = 8;
  sp.balanced = balanced ? 1 : 0;
  sp.lb_stride = stride;
  sp.tile_offsets = offsets;
  sp.status = status_word();
  sp.labels = ws + L.labels;
  return sweep_dispatch<8, THREADS, IPT, true>(sp, tiles, vb, s);
}

BCF_TRACE_INSTALLER(radix)

}  // namespace bcf
