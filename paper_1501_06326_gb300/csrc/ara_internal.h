// Internal interface between the C-ABI host code (ara_abi.cu) and the
// kernels (ara_kernels.cu, ara_select.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ara_device_math.cuh"

namespace ara {

// --------------------------------------------------------------- load time
// Validation flags written by the check kernels (bitwise OR).
enum : uint32_t {
  kBadOffsets = 1u,    // offsets[0] != 0 or offsets decrease
  kBadEventId = 2u,    // id outside [0, catalogue)
  kBadOrder = 4u,      // ELT event ids not strictly increasing
  kBadValue = 8u,      // negative / non-finite mean, sigma or exposure
  kBadExposure = 16u,  // exposure <= mean for a record with mean > 0 and sigma > 0
  kLongTrial = 32u,    // a trial with 2^22 or more events
  kHasCorrelated = 64u,  // not an error: an ELT holds a record with sigma_C > 0
};

// A record's Beta shapes in FP64 and ln B(a, b), computed once when the
// record is prepared (the table builds read them on every node).
struct __align__(16) BetaShape {
  double a, b, lnB, pad;
};

cudaError_t launch_check_offsets(const int64_t* off, int64_t n_trials, int64_t n_events, uint32_t* flags,
                                 cudaStream_t s);
cudaError_t launch_check_ids(const int32_t* ids, int64_t n, int32_t catalogue, uint32_t* flags, cudaStream_t s);
// Copies n ids from pinned host memory that kernels can read at the same
// address (src) into device memory (dst) on a few SMs, checking each against
// [0, catalogue) as it passes: the copy engine stays free for other streams.
cudaError_t launch_upload_ids(const int32_t* src, int32_t* dst, int64_t n, int32_t catalogue, uint32_t* flags,
                              cudaStream_t s);

// Prepare the Pair records of one ELT from (mean, sigma, exposure) in FP64:
// Beta shapes, x0/y0, C, I_{1/2}(a, b), kind.  Also checks order and values
// and reduces the largest event id into *max_event and the largest loss a
// record can produce (max(exposure, mean) over records with a loss, as FP32
// bits) into *max_loss (both atomicMax; max_loss may be null).
cudaError_t launch_prepare_records(const int32_t* events, const float* mean, const float* sigma,
                                   const float* exposure, int64_t n, Pair* out, BetaShape* shapes, uint32_t* flags,
                                   int32_t* max_event, uint32_t* max_loss, cudaStream_t s,
                                   const float* sigma_c = nullptr, float2* weights = nullptr);

// Quantile tables of prepared records, built in FP64: kTabNodes float4 per
// record in `tab`; then, for the first fine_table_cap(n) records (in record
// order) whose coarse table fails its check, kTabFineStride float4 per slot in
// `tabf`.  Sets each record's table-exact and fine bits.  `work` holds
// build_tables_work_words(n) words; on return work[n] is the number of
// candidates for fine tables (min(work[n], cap) slots are used).
size_t build_tables_work_words(int64_t n);
uint32_t fine_table_cap(int64_t n);
cudaError_t launch_build_tables(Pair* recs, const BetaShape* shapes, int64_t n, float4* tab, float4* tabf,
                                uint32_t* work, cudaStream_t s, int* n_launch);
// The two halves of launch_build_tables: coarse tables of n records (need[rec]
// = 1 marks a candidate for a fine table; one launch may span several ELTs),
// then the fine tables of one ELT (`work`: build_tables_work_words(n) words).
cudaError_t launch_build_coarse(Pair* recs, const BetaShape* shapes, int64_t n, float4* tab, uint32_t* need,
                                cudaStream_t s);
cudaError_t launch_build_fine(Pair* recs, const BetaShape* shapes, int64_t n, const uint32_t* need, float4* tabf,
                              uint32_t* work, cudaStream_t s, int* n_launch);
// Fine tables of several ELTs in one launch: job i covers records
// [rec_begin, rec_begin + n) whose candidates were scanned into `slot` (n + 1
// words), and owns fine slots [slot_begin, slot_begin + cap) of `tabf`.  `jobs`
// is a device array, ordered by slot_begin.
struct FineJob {
  int64_t rec_begin, n;
  const uint32_t* slot;
  int64_t slot_begin;
  uint32_t cap, pad;
};
cudaError_t launch_build_fine_jobs(Pair* recs, const BetaShape* shapes, const FineJob* jobs, int n_jobs,
                                   int64_t total_slots, float4* tabf, cudaStream_t s);

// Check kernels (device functions of the hot path on given inputs).
cudaError_t launch_debug_uniforms(uint32_t seed_lo, uint32_t seed_hi, int64_t n, const int64_t* trials,
                                  const int32_t* ks, const int32_t* elts, float* out, cudaStream_t s);
cudaError_t launch_debug_losses(const Pair* recs, const float4* tab, const float4* tabf, const float* z, int64_t n,
                                int newton_only, float* out, int32_t* iters, cudaStream_t s);

// --------------------------------------------------------------- scan
// Exclusive prefix sum of n uint32 values; out[n] receives the total.
// `tmp` must hold scan_tmp_words(n) words.
size_t scan_tmp_words(int64_t n);
cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s,
                               int* n_launch = nullptr);

// --------------------------------------------------------------- layer index
constexpr int kMaxIndexElts = 64;  // ELT positions of one index (a layer, or the union of a batch of layers)

struct LayerEltRefs {
  int32_t n_elts;
  const int32_t* events[kMaxIndexElts];  // sorted event ids of the ELT at position p
  const Pair* recs[kMaxIndexElts];       // prepared records (meta carries the record index)
  const float2* wts[kMaxIndexElts];      // per record (w_I, w_C) of a correlated sigma
  int64_t rec_begin[kMaxIndexElts + 1];  // prefix sums of record counts over positions
};

struct LayerIndex {
  uint32_t* bits;        // [n_words] membership bitmap over the catalogue
  uint32_t* word_cnt;    // [n_words + 1] scratch: popcounts, then exclusive scan
  uint32_t* word_pairs;  // [n_words + 1] scratch: pairs per word, then exclusive scan
  uint2* rankdir;        // [n_words] {bits, base}: base = pairs before the word, or (1 << 31) | slots
                         // before the word when the word holds an event with several ELT records
  unsigned long long* mask;  // [n_recs] per slot: bitmask of layer positions
  uint32_t* slot_cnt;    // [n_recs + 1] scratch -> slot_start
  Pair* pairs;           // [n_recs]
  PairHot* hot;          // [n_recs] the table-path part of each pair
  float2* pw;            // [n_recs] (w_I, w_C) of each pair's record (pairs of kind kKindBetaC)
  int32_t* pev;          // [n_recs] each pair's event id (the per-event output reads it)
  uint32_t* scan_tmp;
  int64_t n_words;
  int64_t n_recs;
};

cudaError_t build_layer_index(const LayerEltRefs& refs, LayerIndex& ix, cudaStream_t s, int* n_launch);

// --------------------------------------------------------------- main kernels
// The layer runs as two kernels over tiles of kWarpTrials consecutive trials:
//   k_gather  streams the YET, filters the events, resolves the hits and writes
//             one 8-byte record per hit event into the tile's region of an
//             event buffer (the region of a tile starts at its first event);
//   k_losses  reads the records of a tile and computes the pair losses, event
//             losses, trial sums and year losses.
constexpr int kGatherThreads = 1024;  // 32 warps per CTA, one CTA per SM
constexpr int kLossThreads = 256;
constexpr int kLossBlocksPerSm = 3;  // 24 warps per SM at up to 85 registers: no spills in the loss loop
// Hit-event record written by k_gather: x = (trial in tile << 28) |
// ((ELT pairs - 1) << 22) | event index in the trial; y = first pair.
constexpr uint32_t kRecTrialShift = 28;
constexpr uint32_t kRecCntShift = 22;
constexpr uint32_t kRecCntMask = 63u;
constexpr uint32_t kRecKMask = (1u << 22) - 1u;
constexpr int kWarpTrials = 8;        // trials per tile (< 32)
constexpr int kMaxTrialEvents = 1 << 22;

struct GatherParams {
  const int64_t* off;
  const int32_t* ids;
  int64_t t_begin, t_end, n_tiles;
  int64_t e0;  // off[t_begin]: the event buffer is indexed from here
  const uint2* rankdir;
  int64_t n_words;
  const uint32_t* slot_start;
  int32_t filt_words;  // filter words: at least n_words / 2, else a power of two
  uint2* ev_buf;
  uint32_t* tile_cnt;
  unsigned long long* queue;  // tile counter
};

struct LossParams {
  const int64_t* off;
  int64_t t_begin, t_end, n_tiles;
  int64_t e0;
  const uint2* ev_buf;
  const uint32_t* tile_cnt;
  const Pair* pairs;
  const PairHot* hot;
  const float2* pw;
  int32_t n_elts;
  int32_t elt_id[32];
  const float4* tab[32];   // coarse quantile tables of the layer's ELTs (by position)
  const float4* tabf[32];  // fine quantile tables
  float t_ret[32], t_lim[32], t_share[32];
  float occ_r, occ_l;  // occurrence terms in FP32 (the loss arithmetic)
  double agg_r, agg_l;
  uint32_t seed_lo, seed_hi;
  uint32_t rk[20];  // Philox round keys of the seed: (seed_lo + r W0, seed_hi + r W1), r = 0..9
  int32_t primary_only;
  int32_t newton_only;
  double* ylt;
  double* def_acc;  // per trial: deferred occurrence losses of trials still pending at their tile's end
  int64_t* diag_hits;
  uint64_t* diag_hash;
  float* occ;  // per-event output: [event buffer entries] each hit event's O_k, beside its record (or NULL)
  unsigned long long* counters;  // [0] tile queue, [1] pairs, [2] non-converged, [3] Halley events
};

// Batched layers (one pass for several layers over the union of their ELTs):
// k_gather as above over the union's index, then k_losses_batch.
constexpr int kBatchLayers = 32;  // ARA_MAX_BATCH_LAYERS
constexpr int kBatchThreads = 128;
constexpr int kBatchBlocksPerSm = 4;

struct BatchParams {
  const int64_t* off;
  int64_t t_begin, t_end, n_tiles;
  int64_t e0;
  const uint2* ev_buf;
  const uint32_t* tile_cnt;
  const Pair* pairs;
  const PairHot* hot;
  const float2* pw;
  int32_t n_elts;  // union positions
  int32_t n_layers;
  int32_t elt_id[kMaxIndexElts];
  const float4* tab[kMaxIndexElts];
  const float4* tabf[kMaxIndexElts];
  float t_ret[kMaxIndexElts], t_lim[kMaxIndexElts], t_share[kMaxIndexElts];
  unsigned long long layers_of[kMaxIndexElts];  // per union position: bitmask of the layers holding it
  float occ_r[kBatchLayers], occ_l[kBatchLayers];
  double agg_r[kBatchLayers], agg_l[kBatchLayers];
  float scale[kBatchLayers];           // fixed point: a layer's occurrence loss O counts as round(O * scale)
                                       // units, scale = 2^e with -126 <= e <= 127 (an FP32 power of two)
  double inv_scale[kBatchLayers];      // 1 / scale
  uint32_t rk[20];                     // Philox round keys of the seed
  int32_t primary_only;
  int32_t newton_only;
  double* ylt_l[kBatchLayers];         // layer l's year losses of trials [t_begin, layer_t_end[l]) (indexed from t_begin)
  unsigned long long* counters;        // [0] tile queue, [1] pairs, [2] non-converged, [3] ring overflow (0)
  int64_t layer_t_end[kBatchLayers];   // layer l's trials end here (<= t_end): later trials get no losses, no output
};

// The losses kernel's work items; all three add the same fixed-point numbers,
// so they give the same results.
enum BatchItem : int {
  kItemTile = 0,   // one warp per tile of kWarpTrials trials, a lane per record
  kItemTrial = 1,  // one warp per trial of a tile, a lane per record
  kItemDense = 2,  // one warp per tile, a lane per pair (records streamed through per-warp rings)
};
cudaError_t launch_losses_batch(const BatchParams& p, int item, int grid, cudaStream_t s);
// CTAs of the dense kernel that one SM holds for n_layers layers (0 on error).
int losses_dense_blocks_per_sm(int n_layers);

size_t gather_smem_bytes(int filt_words);
int gather_filter_words(int64_t n_words, int max_smem);
cudaError_t launch_gather(const GatherParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_losses(const LossParams& p, int grid, cudaStream_t s);

// Per-event output: from the records of each tile and their occurrence losses
// O_k (k_losses with LossParams::occ), each trial's in-order running sum S_k,
// A_k = aggregate terms of S_k and inc_k = A_k - A_{k-1}, written as one row
// per hit event at row_base[tile] + its place in the tile (rows at or beyond
// `cap` are not written); max_occ[t] = the trial's largest O_k (the caller
// zeroes it first: trials without rows keep 0).
struct EventRowsParams {
  const int64_t* off;
  int64_t t_begin, t_end, n_tiles, e0;
  const uint2* ev_buf;
  const float* occ;
  const uint32_t* tile_cnt;
  const uint32_t* row_base;  // [n_tiles + 1] exclusive scan of tile_cnt
  const int32_t* pair_event;  // [pairs] each pair's event id (a record's event: that of its first pair)
  double agg_r, agg_l;
  int64_t cap;
  int64_t* row_trial;   // each of the five may be NULL
  int32_t* row_k;
  int32_t* row_event;
  double* row_occ;
  double* row_inc;
  double* max_occ;      // [t_end - t_begin] or NULL
};
// One wave of resident blocks over num_sms SMs.
cudaError_t launch_event_rows(const EventRowsParams& q, int num_sms, cudaStream_t s);
constexpr int kEventRowsThreads = 256;

// --------------------------------------------------------------- PML / TVaR / sort
// Scratch sizes in bytes for n year losses.
// Scratch of the five-launch select (a select state alone, sizeof the
// state, runs the ten-launch select).
size_t select_scratch_bytes(int64_t n);
// pml/tvar: n_rp device doubles each; rps: host array.
cudaError_t pml_tvar_device(const double* ylt, int64_t n, const double* rps_host, int32_t n_rp, double* pml,
                            double* tvar, void* scratch, size_t scratch_bytes, cudaStream_t s, int* n_launch);
size_t sort_scratch_bytes(int64_t n);
// vals/trials[i] = ylt[order[i]], trial_offset + order[i] for i < m_valid;
// (-inf, -1) for m_valid <= i < m.
cudaError_t top_gather_device(const double* ylt, const int64_t* order, int64_t m_valid, int64_t m, int64_t trial_offset,
                              double* vals, int64_t* trials, cudaStream_t s);
cudaError_t sort_desc_device(const double* ylt, int64_t n, int64_t* order, void* scratch, cudaStream_t s,
                             int* n_launch);

}  // namespace ara
