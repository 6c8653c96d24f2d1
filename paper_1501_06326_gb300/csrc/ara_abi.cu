// C-ABI host side of the ARA engine: context, device residency of the YET and
// the ELT pool, validation, per-layer index build and kernel orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/ara.h"
#include "ara_batch.h"

namespace {

// The YET index keeps each event's occurrence offsets at every 2^kYetGridShift trials (the serving
// chunk: 262,144 trials measured better than 131,072 on the serving workload, p99 18.6 against 35.8 ms
// at 3,200 requests/s and 7.0e12 against 6.6e12 evals/s at saturation; 65,536 far worse). An indexed
// pass runs in slices of 2^k trials, k >= kYetGridShift, the largest whose sums (8 bytes per layer and
// trial) fit kIdxSliceBytes, about half of L2: the sums' atomic adds then stay in L2 while the
// occurrences stream through it (16 layers: 2^19 trials; measured on batched-16, 6.2 ms a pass against
// 8.1 ms in one slice and 6.6 ms at 2^18).
constexpr int kYetGridShift = 18;
// The index is built by buckets per (event, grid cell) while no bucket holds more occurrences than this
// (each bucket is sorted by one thread), else by the radix sort.
constexpr uint32_t kYetBucketSortMax = 2048;
constexpr int64_t kIdxSliceBytes = int64_t{64} << 20;
int idx_slice_shift(int n_layers) {
  int k = kYetGridShift;
  while (k < 40 && (int64_t{8} * n_layers << (k + 1)) <= kIdxSliceBytes) ++k;
  return k;
}
// 64-bit words holding an indexed pass's slice queues (one 32-bit word per slice)
int64_t idx_queue_words(int64_t t_begin, int64_t t_end, int n_layers) {
  return (ara::indexed_slices(t_begin, t_end, idx_slice_shift(n_layers)) + 1) / 2;
}

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Elt {
  DevBuf events;  // int32 [n] (+ padding)
  DevBuf recs;    // ara::Pair [n]
  DevBuf tab;     // float4 [n * kTabNodes] coarse quantile tables
  DevBuf tabf;    // float4 [n_fine * kTabFineStride] fine quantile tables
  DevBuf wts;     // float2 [n] (w_I, w_C) per record, when the ELT holds correlated records
  bool correlated = false;
  int64_t n = 0;
  int64_t n_fine = 0;
  float max_loss = 0.0f;  // largest loss a record can produce (max(exposure, mean))
  int32_t max_event = -1;
  ara_elt_terms terms{0.0f, INFINITY, 1.0f};
};

// A request of the serving loop (ara_submit).
struct ServeReq {
  std::vector<int32_t> elt_ids;
  ara_layer layer{};  // elt_ids points into the vector above
  uint64_t seed = 0;
  int64_t t_end = 0;
  std::vector<double> rps, pml, tvar;
  bool done = false;
  int status = ARA_OK;
  // once admitted: its year losses in the serving arena, its result slot, its chunk cursor
  size_t ylt_off = 0, ylt_bytes = 0;
  int32_t slot = -1;
  int64_t next_chunk = 0, n_chunks = 0;
};

// A launched serving round: the event recorded after its work and the
// requests whose results it completes.
struct ServeRound {
  cudaEvent_t ev = nullptr;
  std::vector<int64_t> finishing;
};

}  // namespace

struct ara_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t used = 0;
  std::string err;
  // YET
  DevBuf yet_off, yet_ids;
  std::vector<int64_t> h_off;
  int64_t n_trials = 0;
  int64_t max_trial_events = 0;
  int64_t n_events = 0;
  int32_t catalogue = 0;
  bool yet_loaded = false;
  // YET upload in flight (ara_load_yet_async): copied and checked on copy_stream;
  // the first call that uses the YET waits for yet_ready and reads the flags
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t yet_ready = nullptr;
  DevBuf yet_flags;                  // uint32 check flags of the upload
  uint32_t* h_yet_flags = nullptr;   // pinned copy of them
  bool yet_pending = false;
  const char* yet_who = "ara_load_yet";
  int64_t p_trials = 0, p_events = 0, p_longest = 0;
  int32_t p_catalogue = 0;
  // ELT pool
  std::map<int32_t, Elt> pool;
  // per-layer index (grown on demand)
  DevBuf bits, word_cnt, word_pairs, rankdir, mask, slot_cnt, pairs, pairs_hot, pairs_w, pairs_ev, scan_tmp;
  DevBuf ev_buf, tile_cnt;  // hit-event records of the layer kernels
  // event-major index of the YET (ara_build_yet_index) and the indexed passes' buffers
  DevBuf yix_occ, yix_grid;
  bool yix_ready = false;
  bool yix_sorted = false;  // built by the radix sort (a bucket was too large)
  float yix_build_ms = 0.0f;
  DevBuf u_flags, u_scan, u_event, u_first, idx_acc;
  DevBuf def_acc;           // per-trial FP64 sums of deferred occurrence losses
  DevBuf elt_stage, elt_recs_stage, elt_tab_stage, elt_flags;  // ELT load staging (grow-only)
  DevBuf elt_tabf_stage, elt_work;
  // misc scratch
  DevBuf flags;     // uint32 flags + int32 max event
  DevBuf counters;  // 4 x u64
  DevBuf ylt_tmp;   // device YLT when the caller's output is on the host
  DevBuf diag_tmp;  // device diagnostics when the caller's outputs are on the host
  DevBuf ev_occ;     // per-event output: O_k beside each event buffer record (float)
  DevBuf row_base;   //   rows before each tile (exclusive scan of tile_cnt) and its scan scratch
  DevBuf evr_stage;  //   rows and max_occ staged on the device for host arrays
  DevBuf sel;       // select / sort scratch
  DevBuf in_tmp;    // staging of host inputs for pml/sort
  DevBuf out_tmp;   // small device outputs
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  ara_stats stats{};
  // timing accumulators: event pairs recorded around launch groups since the last reset
  struct Timed {
    int kind;  // 0 gather kernel, 1 index build, 2 pml/tvar, 3 losses kernel
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Timed> timed;
  int64_t launches = 0;
  int num_sms = 0;
  int max_smem = 0;
  bool no_timing = false;   // serving passes record no timing events
  // the batched losses kernel's configuration per batch shape, chosen by measurement (ARA_AUTOTUNE)
  std::map<std::vector<int64_t>, std::pair<int, int>> tune_cache;  // shape -> (work item, blocks per SM)
  int32_t last_item = 0, last_blocks = 0, last_tuned = 0;
  int32_t force_item = ARA_BATCH_AUTO, force_blocks = 0;  // ara_set_batch_config
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  // serving (continuous batching)
  std::deque<int64_t> serve_queue;      // submitted, not yet admitted, in arrival order
  std::vector<int64_t> serve_active;    // admitted and not finished, in admission order
  std::map<int64_t, ServeReq> serve_reqs;
  std::deque<ServeRound> serve_rounds;  // launched and not retired, in launch order
  std::vector<cudaEvent_t> serve_ev_free;
  int64_t next_ticket = 1;
  bool serve_ready = false;
  DevBuf serve_arena;                   // year losses of the admitted requests
  std::map<size_t, size_t> arena_free;  // free blocks of the arena: offset -> bytes
  DevBuf serve_out;                     // device result slots (PML, TVaR)
  DevBuf serve_sel;                     // select scratch of the requests' PML/TVaR
  cudaStream_t serve_side = nullptr;    // the requests' PML/TVaR and result copies, beside the passes
  cudaEvent_t serve_join = nullptr;     // the passes' stream up to a point, for the side stream to wait on
  double* serve_host = nullptr;         // pinned host result slots
  std::vector<int32_t> serve_slots_free;
  int64_t serve_rounds_launched = 0, serve_passes = 0, serve_finished = 0;
};

namespace {

// Two events for one timed launch group (reused after a reset).
bool timed_pair(ara_ctx* c, int kind, cudaEvent_t* a, cudaEvent_t* b) {
  if (c->no_timing) {
    *a = *b = nullptr;
    return true;
  }
  const size_t need = 2 * (c->timed.size() + 1);
  while (c->ev_pool.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    c->ev_pool.push_back(e);
  }
  *a = c->ev_pool[need - 2];
  *b = c->ev_pool[need - 1];
  c->timed.push_back({kind, *a, *b});
  return true;
}

// Records a timing event (a null event, from a pass without timing, is skipped).
cudaError_t record_ev(cudaEvent_t e, cudaStream_t s) { return e ? cudaEventRecord(e, s) : cudaSuccess; }

int fail(ara_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define ARA_CUDA(c, call)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail((c), ARA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void release(ara_ctx* c, DevBuf& b) {
  if (b.ptr) {
    cudaFree(b.ptr);
    c->used -= b.bytes;
  }
  b.ptr = nullptr;
  b.bytes = 0;
}

// Make b hold at least `bytes` (contents are not preserved).
int reserve(ara_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return ARA_OK;
  const size_t old = b.bytes;
  release(c, b);
  if (c->budget && c->used + bytes > c->budget)
    return fail(c, ARA_ENOMEM, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu in use, %zu released)",
                bytes, c->used, c->budget, old);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, ARA_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  b.ptr = p;
  b.bytes = bytes;
  c->used += bytes;
  return ARA_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Small parameter arrays to the host: a plain copy from host memory (no
// device synchronisation), cudaMemcpy from device memory.
cudaError_t copy_params_to_host(void* dst, const void* src, size_t bytes) {
  if (!is_device_ptr(src)) {
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
  }
  return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
}

// Pinned (or registered) host memory that kernels can read at the same address.
bool is_mapped_host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

cudaMemcpyKind kind_to_device(const void* src) {
  return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

int bind(ara_ctx* c) {
  if (!c) return ARA_EINVAL;
  ARA_CUDA(c, cudaSetDevice(c->device));
  return ARA_OK;
}

}  // namespace

extern "C" {

int ara_create(ara_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return ARA_EINVAL;
  *out = nullptr;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) {
    cudaGetLastError();
    return ARA_ECUDA;
  }
  if (device < 0 || device >= n_dev) return ARA_EINVAL;
  ara_ctx* c = new ara_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return ARA_ECUDA;
  }
  for (auto& e : c->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      ara_destroy(c);
      return ARA_ECUDA;
    }
  }
  if (reserve(c, c->flags, 64) != ARA_OK || reserve(c, c->counters, 64) != ARA_OK) {
    ara_destroy(c);
    return ARA_ENOMEM;
  }
  *out = c;
  return ARA_OK;
}

int ara_set_stream(ara_ctx* c, void* cuda_stream) {
  int rc = bind(c);
  if (rc) return rc;
  ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return ARA_OK;
}

}  // extern "C"

namespace {

// Waits for the YET upload in flight, if any, and makes it the loaded YET when
// its checks passed.
int yet_finish(ara_ctx* c) {
  if (!c->yet_pending) return ARA_OK;
  c->yet_pending = false;
  ARA_CUDA(c, cudaEventSynchronize(c->yet_ready));
  const uint32_t f = *c->h_yet_flags;
  if (f & ara::kBadOffsets) return fail(c, ARA_EINVAL, "%s: offsets are not non-decreasing", c->yet_who);
  if (f & ara::kLongTrial) return fail(c, ARA_EINVAL, "%s: a trial has 2^22 or more events", c->yet_who);
  if (f & ara::kBadEventId)
    return fail(c, ARA_EINVAL, "%s: an event id lies outside [0, %d)", c->yet_who, c->p_catalogue);
  c->n_trials = c->p_trials;
  c->n_events = c->p_events;
  c->max_trial_events = c->p_longest;
  c->catalogue = c->p_catalogue;
  c->yet_loaded = true;
  return ARA_OK;
}

// Starts loading a YET: the offsets are read on the host during the call; the
// offsets and ids are copied to the device and checked on copy_stream, which
// runs beside later work on the context's stream until yet_finish.
int yet_begin(ara_ctx* c, int64_t n_trials, const int64_t* offsets, const int32_t* event_ids,
              int32_t catalogue_size, const char* who) {
  int rc = bind(c);
  if (rc) return rc;
  if (n_trials < 1 || !offsets || catalogue_size < 1)
    return fail(c, ARA_EINVAL, "%s: need n_trials >= 1, offsets and catalogue_size >= 1", who);
  if (!c->serve_queue.empty() || !c->serve_active.empty() || !c->serve_rounds.empty())
    return fail(c, ARA_EINVAL, "%s: served requests are queued or running on the loaded YET", who);
  // the serving workspace and arena follow the YET's size
  c->serve_ready = false;
  release(c, c->serve_arena);
  // an upload still in flight is replaced: wait for it, whatever its checks say
  if (c->yet_pending) {
    c->yet_pending = false;
    ARA_CUDA(c, cudaEventSynchronize(c->yet_ready));
  }
  c->yet_loaded = false;
  c->yix_ready = false;  // the index belongs to the YET being replaced
  release(c, c->yix_occ);
  release(c, c->yix_grid);
  if (!c->copy_stream) {
    ARA_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    ARA_CUDA(c, cudaEventCreateWithFlags(&c->yet_ready, cudaEventDisableTiming));
    ARA_CUDA(c, cudaMallocHost(&c->h_yet_flags, sizeof(uint32_t)));
    if ((rc = reserve(c, c->yet_flags, 16))) return rc;
  }
  // the work before the call may still read the old YET
  ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  // the sizes first; the host copy of all offsets is taken while the upload runs
  int64_t first = 0, n_events = 0;
  ARA_CUDA(c, copy_params_to_host(&first, offsets, sizeof(int64_t)));
  ARA_CUDA(c, copy_params_to_host(&n_events, offsets + n_trials, sizeof(int64_t)));
  if (first != 0 || n_events < 0) return fail(c, ARA_EINVAL, "%s: offsets[0] must be 0 and offsets[n] >= 0", who);
  if (n_events > 0 && !event_ids) return fail(c, ARA_EINVAL, "%s: event_ids is NULL", who);
  if ((rc = reserve(c, c->yet_off, sizeof(int64_t) * (n_trials + 1)))) return rc;
  // ids: padded by 4 entries so that 16-byte loads near the end stay inside the buffer
  if ((rc = reserve(c, c->yet_ids, sizeof(int32_t) * (n_events + 4)))) return rc;
  cudaStream_t cs = c->copy_stream;
  uint32_t* flags = static_cast<uint32_t*>(c->yet_flags.ptr);
  ARA_CUDA(c, cudaMemsetAsync(flags, 0, sizeof(uint32_t), cs));
  ARA_CUDA(c, cudaMemcpyAsync(c->yet_off.ptr, offsets, sizeof(int64_t) * (n_trials + 1), kind_to_device(offsets), cs));
  ARA_CUDA(c, cudaMemsetAsync(static_cast<int32_t*>(c->yet_ids.ptr) + n_events, 0, sizeof(int32_t) * 4, cs));
  ARA_CUDA(c, ara::launch_check_offsets(static_cast<const int64_t*>(c->yet_off.ptr), n_trials, n_events, flags, cs));
  int32_t* d_ids = static_cast<int32_t*>(c->yet_ids.ptr);
  if (n_events > 0 && is_mapped_host_ptr(event_ids)) {
    // pinned host ids: a kernel reads them over the host link and checks them on
    // the way, so that the copy engine serves the other streams' copies meanwhile
    ARA_CUDA(c, ara::launch_upload_ids(event_ids, d_ids, n_events, catalogue_size, flags, cs));
  } else if (n_events > 0) {
    ARA_CUDA(c, cudaMemcpyAsync(d_ids, event_ids, sizeof(int32_t) * n_events, kind_to_device(event_ids), cs));
    ARA_CUDA(c, ara::launch_check_ids(d_ids, n_events, catalogue_size, flags, cs));
  }
  c->launches += 1 + (n_events > 0 ? 1 : 0);
  ARA_CUDA(c, cudaMemcpyAsync(c->h_yet_flags, flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs));
  ARA_CUDA(c, cudaEventRecord(c->yet_ready, cs));
  // offsets: keep a host copy (sizes and ranges are planned on the host); on an
  // error the upload just started is waited for, so that nothing is left in flight
  c->h_off.resize(static_cast<size_t>(n_trials) + 1);
  const cudaError_t he = copy_params_to_host(c->h_off.data(), offsets, sizeof(int64_t) * (n_trials + 1));
  if (he != cudaSuccess) {
    cudaEventSynchronize(c->yet_ready);
    return fail(c, ARA_ECUDA, "%s: copy of the offsets: %s", who, cudaGetErrorString(he));
  }
  int64_t longest = 0;  // bounds a trial's sum in the batched layers' fixed point
  for (int64_t t = 0; t < n_trials; ++t) longest = std::max(longest, c->h_off[t + 1] - c->h_off[t]);
  c->p_trials = n_trials;
  c->p_events = n_events;
  c->p_longest = longest;
  c->p_catalogue = catalogue_size;
  c->yet_who = who;
  c->yet_pending = true;
  return ARA_OK;
}

}  // namespace

extern "C" {

int ara_load_yet(ara_ctx* c, int64_t n_trials, const int64_t* offsets, const int32_t* event_ids,
                 int32_t catalogue_size) {
  const int rc = yet_begin(c, n_trials, offsets, event_ids, catalogue_size, "ara_load_yet");
  return rc ? rc : yet_finish(c);
}

int ara_load_yet_async(ara_ctx* c, int64_t n_trials, const int64_t* offsets, const int32_t* event_ids,
                       int32_t catalogue_size) {
  return yet_begin(c, n_trials, offsets, event_ids, catalogue_size, "ara_load_yet_async");
}

int ara_finish_yet(ara_ctx* c) {
  const int rc = bind(c);
  return rc ? rc : yet_finish(c);
}

// ara_load_elts and ara_load_xelts; sigma_c == NULL: no correlated part.
static int load_elts_impl(ara_ctx* c, const char* who, int32_t n_elts, const int32_t* elt_ids,
                          const int64_t* rec_offsets, const int32_t* event_ids, const float* mean, const float* sigma,
                          const float* sigma_c, const float* exposure, const ara_elt_terms* terms) {
  int rc = bind(c);
  if (rc) return rc;
  if (n_elts < 1 || !elt_ids || !rec_offsets) return fail(c, ARA_EINVAL, "%s: bad arguments", who);
  std::vector<int32_t> ids(n_elts);
  std::vector<int64_t> offs(static_cast<size_t>(n_elts) + 1);
  std::vector<ara_elt_terms> tm(n_elts, ara_elt_terms{0.0f, INFINITY, 1.0f});
  ARA_CUDA(c, copy_params_to_host(ids.data(), elt_ids, sizeof(int32_t) * n_elts));
  ARA_CUDA(c, copy_params_to_host(offs.data(), rec_offsets, sizeof(int64_t) * (n_elts + 1)));
  if (terms) ARA_CUDA(c, copy_params_to_host(tm.data(), terms, sizeof(ara_elt_terms) * n_elts));
  if (offs[0] != 0) return fail(c, ARA_EINVAL, "%s: rec_offsets[0] must be 0", who);
  for (int32_t i = 0; i < n_elts; ++i) {
    if (ids[i] < 0) return fail(c, ARA_EINVAL, "%s: pool id %d is negative", who, ids[i]);
    if (offs[i + 1] < offs[i]) return fail(c, ARA_EINVAL, "%s: rec_offsets decrease at %d", who, i);
    if (offs[i + 1] - offs[i] >= static_cast<int64_t>(ara::kMaxEltRecords))
      return fail(c, ARA_EINVAL, "%s: ELT %d has %lld records (at most %u)", who, ids[i],
                  (long long)(offs[i + 1] - offs[i]), ara::kMaxEltRecords - 1);
    const ara_elt_terms& t = tm[i];
    if (!(t.retention >= 0.0f) || !(t.limit >= 0.0f) || !(t.share >= 0.0f) || std::isnan(t.limit) ||
        !std::isfinite(t.retention) || !std::isfinite(t.share))
      return fail(c, ARA_EINVAL, "%s: ELT %d has invalid financial terms", who, ids[i]);
    for (int32_t j = 0; j < i; ++j)
      if (ids[j] == ids[i]) return fail(c, ARA_EINVAL, "%s: pool id %d appears twice", who, ids[i]);
    for (int64_t tk : c->serve_active) {
      const std::vector<int32_t>& used = c->serve_reqs[tk].elt_ids;
      if (std::find(used.begin(), used.end(), ids[i]) != used.end())
        return fail(c, ARA_EINVAL, "%s: ELT %d is used by a served request that has not finished", who, ids[i]);
    }
  }
  const int64_t R = offs[n_elts];
  if (R > 0 && (!event_ids || !mean || !sigma || !exposure))
    return fail(c, ARA_EINVAL, "%s: record arrays are NULL", who);
  // ---- stage: inputs, prepared records and tables of all ELTs (grow-only context buffers)
  std::vector<int64_t> fine_off(static_cast<size_t>(n_elts) + 1, 0), work_off(static_cast<size_t>(n_elts) + 1, 0);
  for (int32_t i = 0; i < n_elts; ++i) {
    const int64_t n = offs[i + 1] - offs[i];
    fine_off[i + 1] = fine_off[i] + ara::fine_table_cap(n);
    work_off[i + 1] = work_off[i] + static_cast<int64_t>(ara::build_tables_work_words(n));
  }
  const size_t in_bytes =
      static_cast<size_t>(R) * (sizeof(int32_t) + 4 * sizeof(float) + sizeof(ara::BetaShape) + sizeof(float2)) + 64;
  if ((rc = reserve(c, c->elt_stage, in_bytes)) ||
      (rc = reserve(c, c->elt_recs_stage, sizeof(ara::Pair) * (R + 1))) ||
      (rc = reserve(c, c->elt_tab_stage, sizeof(float4) * ara::kTabNodes * (R + 1))) ||
      (rc = reserve(c, c->elt_tabf_stage, sizeof(float4) * ara::kTabFineStride * (fine_off[n_elts] + 1))) ||
      (rc = reserve(c, c->elt_work, sizeof(uint32_t) * (work_off[n_elts] + R + 8) +
                                        sizeof(ara::FineJob) * static_cast<size_t>(n_elts))) ||
      (rc = reserve(c, c->elt_flags, sizeof(uint32_t) * 4 * n_elts)))
    return rc;
  int32_t* d_ev = static_cast<int32_t*>(c->elt_stage.ptr);
  float* d_mu = reinterpret_cast<float*>(d_ev + R);
  float* d_sg = d_mu + R;
  float* d_ex = d_sg + R;
  float* d_sc = d_ex + R;
  ara::BetaShape* d_shapes =
      reinterpret_cast<ara::BetaShape*>((reinterpret_cast<uintptr_t>(d_sc + R) + 15) & ~uintptr_t(15));
  float2* d_w = reinterpret_cast<float2*>(d_shapes + R);
  ara::Pair* d_recs = static_cast<ara::Pair*>(c->elt_recs_stage.ptr);
  float4* d_tab = static_cast<float4*>(c->elt_tab_stage.ptr);
  float4* d_tabf = static_cast<float4*>(c->elt_tabf_stage.ptr);
  uint32_t* d_work = static_cast<uint32_t*>(c->elt_work.ptr);
  uint32_t* d_need = d_work + work_off[n_elts];  // [R] fine-table candidates, all ELTs
  uint32_t* d_flags = static_cast<uint32_t*>(c->elt_flags.ptr);
  if (R > 0) {
    ARA_CUDA(c, cudaMemcpyAsync(d_ev, event_ids, sizeof(int32_t) * R, kind_to_device(event_ids), c->stream));
    ARA_CUDA(c, cudaMemcpyAsync(d_mu, mean, sizeof(float) * R, kind_to_device(mean), c->stream));
    ARA_CUDA(c, cudaMemcpyAsync(d_sg, sigma, sizeof(float) * R, kind_to_device(sigma), c->stream));
    ARA_CUDA(c, cudaMemcpyAsync(d_ex, exposure, sizeof(float) * R, kind_to_device(exposure), c->stream));
    if (sigma_c) ARA_CUDA(c, cudaMemcpyAsync(d_sc, sigma_c, sizeof(float) * R, kind_to_device(sigma_c), c->stream));
  }
  // per ELT: flags word, the largest event id (0xFFFFFFFF = none), candidates for fine
  // tables, the largest loss (FP32 bits)
  std::vector<uint32_t> init(4 * static_cast<size_t>(n_elts));
  for (int32_t i = 0; i < n_elts; ++i) {
    init[4 * i] = 0u;
    init[4 * i + 1] = 0xFFFFFFFFu;
    init[4 * i + 2] = 0u;
    init[4 * i + 3] = 0u;
  }
  ARA_CUDA(c, cudaMemcpyAsync(d_flags, init.data(), sizeof(uint32_t) * init.size(), cudaMemcpyHostToDevice, c->stream));
  for (int32_t i = 0; i < n_elts; ++i) {
    const int64_t o = offs[i], n = offs[i + 1] - offs[i];
    uint32_t* f = d_flags + 4 * i;
    ARA_CUDA(c, ara::launch_prepare_records(d_ev + o, d_mu + o, d_sg + o, d_ex + o, n, d_recs + o, d_shapes + o, f,
                                            reinterpret_cast<int32_t*>(f + 1), f + 3, c->stream,
                                            sigma_c ? d_sc + o : nullptr, sigma_c ? d_w + o : nullptr));
    c->launches += 1;
  }
  // coarse tables of every record in one launch, then each ELT's fine tables
  ARA_CUDA(c, ara::launch_build_coarse(d_recs, d_shapes, R, d_tab, d_need, c->stream));
  c->launches += (R > 0) ? 1 : 0;
  std::vector<ara::FineJob> jobs;
  for (int32_t i = 0; i < n_elts; ++i) {
    const int64_t o = offs[i], n = offs[i + 1] - offs[i];
    if (n == 0) continue;
    int launched = 0;
    uint32_t* w = d_work + work_off[i];
    ARA_CUDA(c, ara::scan_exclusive_u32(d_need + o, w, n, w + n + 1, c->stream, &launched));
    ARA_CUDA(c, cudaMemcpyAsync(d_flags + 4 * i + 2, w + n, sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream));
    c->launches += launched;
    jobs.push_back(ara::FineJob{o, n, w, fine_off[i], ara::fine_table_cap(n), 0});
  }
  if (!jobs.empty()) {
    // fine tables of every ELT in one launch (the job list is staged after the need flags)
    ara::FineJob* d_jobs = reinterpret_cast<ara::FineJob*>(
        (reinterpret_cast<uintptr_t>(d_need + R) + 15) & ~uintptr_t(15));
    ARA_CUDA(c, cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(ara::FineJob) * jobs.size(), cudaMemcpyHostToDevice,
                                c->stream));
    ARA_CUDA(c, ara::launch_build_fine_jobs(d_recs, d_shapes, d_jobs, static_cast<int>(jobs.size()),
                                            fine_off[n_elts], d_tabf, c->stream));
    c->launches += 1;
  }
  std::vector<uint32_t> hf(4 * static_cast<size_t>(n_elts));
  ARA_CUDA(c, cudaMemcpyAsync(hf.data(), d_flags, sizeof(uint32_t) * hf.size(), cudaMemcpyDeviceToHost, c->stream));
  ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int32_t i = 0; i < n_elts; ++i) {
    const uint32_t f = hf[4 * i];
    const char* why = nullptr;
    if (f & ara::kBadOrder) why = "event ids are not strictly increasing";
    else if (f & ara::kBadEventId) why = "an event id is negative";
    else if (f & ara::kBadValue) why = "a mean, sigma, sigma_c or exposure is negative or not finite";
    else if (f & ara::kBadExposure) why = "a record with mean > 0 and sigma > 0 has exposure <= mean";
    if (why) return fail(c, ARA_EINVAL, "%s: ELT %d: %s", who, ids[i], why);
  }
  // ---- commit: each ELT keeps (or grows) its own buffers; the pool only changes once all checks passed
  for (int32_t i = 0; i < n_elts; ++i) {
    const int64_t o = offs[i], n = offs[i + 1] - offs[i];
    const int64_t n_fine = std::min<int64_t>(hf[4 * i + 2], ara::fine_table_cap(n));
    const bool corr = (hf[4 * i] & ara::kHasCorrelated) != 0u;
    Elt& el = c->pool[ids[i]];
    if ((rc = reserve(c, el.events, sizeof(int32_t) * (n + 4))) ||
        (rc = reserve(c, el.recs, sizeof(ara::Pair) * (n > 0 ? n : 1))) ||
        (rc = reserve(c, el.tab, sizeof(float4) * ara::kTabNodes * (n > 0 ? n : 1))) ||
        (rc = reserve(c, el.tabf, sizeof(float4) * ara::kTabFineStride * (n_fine > 0 ? n_fine : 1))) ||
        (corr && (rc = reserve(c, el.wts, sizeof(float2) * n)))) {
      release(c, el.events);
      release(c, el.recs);
      release(c, el.tab);
      release(c, el.tabf);
      release(c, el.wts);
      c->pool.erase(ids[i]);
      return rc;
    }
    if (!corr) release(c, el.wts);
    el.correlated = corr;
    el.n = n;
    el.n_fine = n_fine;
    el.terms = tm[i];
    el.max_event = static_cast<int32_t>(hf[4 * i + 1]);
    std::memcpy(&el.max_loss, &hf[4 * i + 3], sizeof(float));
    if (n > 0) {
      ARA_CUDA(c, cudaMemcpyAsync(el.events.ptr, d_ev + o, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
      ARA_CUDA(c, cudaMemcpyAsync(el.recs.ptr, d_recs + o, sizeof(ara::Pair) * n, cudaMemcpyDeviceToDevice, c->stream));
      ARA_CUDA(c, cudaMemcpyAsync(el.tab.ptr, d_tab + o * ara::kTabNodes, sizeof(float4) * ara::kTabNodes * n,
                                  cudaMemcpyDeviceToDevice, c->stream));
      if (corr)
        ARA_CUDA(c, cudaMemcpyAsync(el.wts.ptr, d_w + o, sizeof(float2) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (n_fine > 0) {
      ARA_CUDA(c, cudaMemcpyAsync(el.tabf.ptr, d_tabf + fine_off[i] * ara::kTabFineStride,
                                  sizeof(float4) * ara::kTabFineStride * n_fine, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  return ARA_OK;
}

int ara_load_elts(ara_ctx* c, int32_t n_elts, const int32_t* elt_ids, const int64_t* rec_offsets,
                  const int32_t* event_ids, const float* mean, const float* sigma, const float* exposure,
                  const ara_elt_terms* terms) {
  return load_elts_impl(c, "ara_load_elts", n_elts, elt_ids, rec_offsets, event_ids, mean, sigma, nullptr, exposure,
                        terms);
}

int ara_load_xelts(ara_ctx* c, int32_t n_elts, const int32_t* elt_ids, const int64_t* rec_offsets,
                   const int32_t* event_ids, const float* mean, const float* sigma_i, const float* sigma_c,
                   const float* exposure, const ara_elt_terms* terms) {
  int rc = bind(c);
  if (rc) return rc;
  if (!sigma_c && n_elts >= 1 && rec_offsets) {
    int64_t R = 0;
    ARA_CUDA(c, copy_params_to_host(&R, rec_offsets + n_elts, sizeof(int64_t)));
    if (R > 0) return fail(c, ARA_EINVAL, "ara_load_xelts: sigma_c is NULL");
  }
  return load_elts_impl(c, "ara_load_xelts", n_elts, elt_ids, rec_offsets, event_ids, mean, sigma_i, sigma_c,
                        exposure, terms);
}

// ---------------------------------------------------------------- layer passes
// What a pass over a trial range needs before its losses kernel: the index of
// the ELTs it covers (a layer, or the union of a batch) and the gather launch.
struct PassPlan {
  ara::LayerEltRefs refs{};
  ara::LayerIndex ix{};
  ara::GatherParams g{};
  int64_t n_out = 0, n_tiles = 0, e0 = 0;
  int grid = 0;
  size_t smem = 0;
  int filt_words = 0;
};

static int check_trial_range(ara_ctx* c, int64_t t0, int64_t t1, const char* who) {
  const int rc = yet_finish(c);
  if (rc) return rc;
  if (!c->yet_loaded) return fail(c, ARA_ENOTLOADED, "%s: no YET loaded", who);
  if (t0 < 0 || t1 > c->n_trials || t0 >= t1)
    return fail(c, ARA_EINVAL, "%s: trial range [%lld, %lld) outside [0, %lld)", who, (long long)t0, (long long)t1,
                (long long)c->n_trials);
  return ARA_OK;
}

// A layer's ELT list (1..ARA_MAX_LAYER_ELTS distinct ids) and terms; `ids`
// receives the ids in canonical (ascending) order, so that no result depends
// on the order in which the caller lists a layer's ELTs.
static int check_layer(ara_ctx* c, const ara_layer* L, const char* who, std::vector<int32_t>* ids) {
  if (L->n_elts < 1 || L->n_elts > ARA_MAX_LAYER_ELTS || !L->elt_ids)
    return fail(c, ARA_EINVAL, "%s: a layer needs 1..%d ELTs", who, ARA_MAX_LAYER_ELTS);
  if (!(L->occ_retention >= 0.0) || !(L->agg_retention >= 0.0) || !(L->occ_limit >= 0.0) ||
      !(L->agg_limit >= 0.0) || !std::isfinite(L->occ_retention) || !std::isfinite(L->agg_retention))
    return fail(c, ARA_EINVAL, "%s: retentions must be finite and >= 0, limits >= 0", who);
  ids->assign(L->elt_ids, L->elt_ids + L->n_elts);
  std::sort(ids->begin(), ids->end());
  for (size_t i = 1; i < ids->size(); ++i)
    if ((*ids)[i] == (*ids)[i - 1]) return fail(c, ARA_EINVAL, "%s: pool id %d repeated in a layer", who, (*ids)[i]);
  return ARA_OK;
}

// The ELT word of a pair's Philox counter: its pool id, or the word every
// ELT of an occurrence shares under ARA_SHARED_Z.
static int32_t philox_elt_word(int32_t pool_id, uint32_t flags) {
  return (flags & ARA_SHARED_Z) ? static_cast<int32_t>(0xFFFFFFFEu) : pool_id;
}

// Index buffers for the ELTs `ids` (ascending pool ids, at most
// kMaxIndexElts) and the gather over [t0, t1).
static int plan_pass(ara_ctx* c, const std::vector<int32_t>& ids, int64_t t0, int64_t t1, const char* who,
                     PassPlan* pl) {
  int rc;
  pl->refs = ara::LayerEltRefs{};
  pl->refs.n_elts = static_cast<int32_t>(ids.size());
  pl->refs.rec_begin[0] = 0;
  bool any_corr = false;
  for (size_t i = 0; i < ids.size(); ++i) {
    auto it = c->pool.find(ids[i]);
    if (it == c->pool.end()) return fail(c, ARA_ENOTLOADED, "%s: ELT %d is not loaded", who, ids[i]);
    const Elt& el = it->second;
    if (el.max_event >= c->catalogue)
      return fail(c, ARA_EINVAL, "%s: ELT %d holds event id %d outside the catalogue of %d", who, ids[i],
                  el.max_event, c->catalogue);
    pl->refs.events[i] = static_cast<const int32_t*>(el.events.ptr);
    pl->refs.recs[i] = static_cast<const ara::Pair*>(el.recs.ptr);
    pl->refs.wts[i] = el.correlated ? static_cast<const float2*>(el.wts.ptr) : nullptr;
    any_corr = any_corr || el.correlated;
    pl->refs.rec_begin[i + 1] = pl->refs.rec_begin[i] + el.n;
  }
  const int64_t n_recs = pl->refs.rec_begin[ids.size()];
  if (n_recs >= (int64_t(1) << 31) - 1) return fail(c, ARA_EINVAL, "%s: the ELTs hold too many records", who);
  // ---- index
  const int64_t n_words = (static_cast<int64_t>(c->catalogue) + 31) / 32;
  const size_t tmp_words = std::max(ara::scan_tmp_words(n_words), ara::scan_tmp_words(n_recs));
  if ((rc = reserve(c, c->bits, sizeof(uint32_t) * n_words)) ||
      (rc = reserve(c, c->word_cnt, sizeof(uint32_t) * (n_words + 1))) ||
      (rc = reserve(c, c->word_pairs, sizeof(uint32_t) * (n_words + 1))) ||
      (rc = reserve(c, c->rankdir, sizeof(uint2) * n_words)) ||
      (rc = reserve(c, c->mask, sizeof(unsigned long long) * (n_recs + 1))) ||
      (rc = reserve(c, c->slot_cnt, sizeof(uint32_t) * (n_recs + 2))) ||
      (rc = reserve(c, c->pairs, sizeof(ara::Pair) * (n_recs + 1))) ||
      (rc = reserve(c, c->pairs_hot, sizeof(ara::PairHot) * (n_recs + 1))) ||
      (any_corr && (rc = reserve(c, c->pairs_w, sizeof(float2) * (n_recs + 1)))) ||
      (rc = reserve(c, c->pairs_ev, sizeof(int32_t) * (n_recs + 1))) ||
      (rc = reserve(c, c->scan_tmp, sizeof(uint32_t) * (tmp_words + 8))))
    return rc;
  ara::LayerIndex& ix = pl->ix;
  ix.bits = static_cast<uint32_t*>(c->bits.ptr);
  ix.word_cnt = static_cast<uint32_t*>(c->word_cnt.ptr);
  ix.word_pairs = static_cast<uint32_t*>(c->word_pairs.ptr);
  ix.rankdir = static_cast<uint2*>(c->rankdir.ptr);
  ix.mask = static_cast<unsigned long long*>(c->mask.ptr);
  ix.slot_cnt = static_cast<uint32_t*>(c->slot_cnt.ptr);
  ix.pairs = static_cast<ara::Pair*>(c->pairs.ptr);
  ix.hot = static_cast<ara::PairHot*>(c->pairs_hot.ptr);
  ix.pw = any_corr ? static_cast<float2*>(c->pairs_w.ptr) : nullptr;
  ix.pev = static_cast<int32_t*>(c->pairs_ev.ptr);
  ix.scan_tmp = static_cast<uint32_t*>(c->scan_tmp.ptr);
  ix.n_words = n_words;
  ix.n_recs = n_recs;
  // ---- gather
  pl->filt_words = ara::gather_filter_words(n_words, c->max_smem);
  pl->smem = ara::gather_smem_bytes(pl->filt_words);
  if (pl->filt_words < 1 || pl->smem > static_cast<size_t>(c->max_smem))
    return fail(c, ARA_ECUDA, "%s: kernel needs %zu bytes of shared memory, device allows %d", who, pl->smem,
                c->max_smem);
  pl->n_out = t1 - t0;
  pl->n_tiles = (pl->n_out + ara::kWarpTrials - 1) / ara::kWarpTrials;
  pl->e0 = c->h_off[t0];
  const int64_t e1 = c->h_off[t1];
  if ((rc = reserve(c, c->ev_buf, sizeof(uint2) * (e1 - pl->e0 + 1))) ||
      (rc = reserve(c, c->tile_cnt, sizeof(uint32_t) * (pl->n_tiles + 1))) ||
      (rc = reserve(c, c->def_acc, sizeof(double) * (pl->n_out + 1))))
    return rc;
  ara::GatherParams& g = pl->g;
  g.off = static_cast<const int64_t*>(c->yet_off.ptr);
  g.ids = static_cast<const int32_t*>(c->yet_ids.ptr);
  g.t_begin = t0;
  g.t_end = t1;
  g.n_tiles = pl->n_tiles;
  g.e0 = pl->e0;
  g.rankdir = ix.rankdir;
  g.n_words = n_words;
  g.slot_start = ix.slot_cnt;
  g.filt_words = pl->filt_words;
  g.ev_buf = static_cast<uint2*>(c->ev_buf.ptr);
  g.tile_cnt = static_cast<uint32_t*>(c->tile_cnt.ptr);
  g.queue = static_cast<unsigned long long*>(c->counters.ptr) + 4;
  const int64_t warps_per_sm = ara::kGatherThreads / 32;
  pl->grid = static_cast<int>(std::min<int64_t>(c->num_sms, (pl->n_tiles + warps_per_sm - 1) / warps_per_sm));
  return ARA_OK;
}

// Index build and gather on the context stream (with their timing events).
static int launch_index(ara_ctx* c, const PassPlan& pl, const char* who, int* launched) {
  cudaEvent_t ia, ib;
  if (!timed_pair(c, 1, &ia, &ib)) return fail(c, ARA_ECUDA, "%s: cannot create timing events", who);
  ARA_CUDA(c, cudaMemsetAsync(c->counters.ptr, 0, 8 * sizeof(unsigned long long), c->stream));
  ARA_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  ARA_CUDA(c, record_ev(ia, c->stream));
  ARA_CUDA(c, ara::build_layer_index(pl.refs, const_cast<ara::LayerIndex&>(pl.ix), c->stream, launched));
  ARA_CUDA(c, record_ev(ib, c->stream));
  ARA_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  ARA_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
  return ARA_OK;
}

static int launch_index_and_gather(ara_ctx* c, const PassPlan& pl, const char* who, int* launched) {
  int rc = launch_index(c, pl, who, launched);
  if (rc) return rc;
  cudaEvent_t ka, kb;
  if (!timed_pair(c, 0, &ka, &kb)) return fail(c, ARA_ECUDA, "%s: cannot create timing events", who);
  ARA_CUDA(c, record_ev(ka, c->stream));
  ARA_CUDA(c, ara::launch_gather(pl.g, pl.grid, pl.smem, c->stream));
  ARA_CUDA(c, record_ev(kb, c->stream));
  *launched += 1;
  return ARA_OK;
}

static void fill_philox_keys(uint64_t seed, uint32_t (&rk)[20]) {
  const uint32_t lo = static_cast<uint32_t>(seed & 0xFFFFFFFFull), hi = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {  // Weyl key schedule of Philox4x32
    rk[2 * r] = lo + static_cast<uint32_t>(r) * 0x9E3779B9u;
    rk[2 * r + 1] = hi + static_cast<uint32_t>(r) * 0xBB67AE85u;
  }
}

static void record_pass_stats(ara_ctx* c, const PassPlan& pl, int64_t t0, int64_t t1, int64_t elts) {
  c->stats = ara_stats{};
  c->stats.n_events = c->h_off[t1] - c->h_off[t0];
  c->stats.n_evals = c->stats.n_events * elts;
  c->stats.grid = pl.grid;
  c->stats.block = ara::kGatherThreads;
  c->stats.smem_bytes = static_cast<int32_t>(pl.smem);
  c->stats.filter_bits = pl.filt_words * 32;
  c->stats.kernel_ms = -1.0f;  // device times are read lazily by ara_get_stats
}

// The rows of ara_run_layer_events after the losses kernel wrote O_k beside
// the records: row bases per tile, the row count (read back), then the rows.
static int emit_event_rows(ara_ctx* c, const PassPlan& pl, const ara::LossParams& p, ara_event_rows* evr,
                           int* launched) {
  const int64_t n_tiles = pl.n_tiles, n_out = pl.n_out;
  int rc;
  const size_t tmp_words = ara::scan_tmp_words(n_tiles);
  if ((rc = reserve(c, c->row_base, sizeof(uint32_t) * (n_tiles + 1 + tmp_words + 8)))) return rc;
  uint32_t* d_base = static_cast<uint32_t*>(c->row_base.ptr);
  ARA_CUDA(c, ara::scan_exclusive_u32(p.tile_cnt, d_base, n_tiles, d_base + n_tiles + 1, c->stream, launched));
  uint32_t total = 0;
  ARA_CUDA(c, cudaMemcpyAsync(&total, d_base + n_tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  const int64_t n_rows = total;
  const int64_t n_w = std::min<int64_t>(evr->capacity, n_rows);
  // device targets: the caller's arrays, or slices of the staging buffer
  void* user[5] = {evr->trial, evr->event_index, evr->event_id, evr->occ_loss, evr->agg_inc};
  const size_t esz[5] = {sizeof(int64_t), sizeof(int32_t), sizeof(int32_t), sizeof(double), sizeof(double)};
  bool staged[5];
  size_t stage_bytes = 0, at[6];
  for (int i = 0; i < 5; ++i) {
    staged[i] = user[i] && n_w > 0 && !is_device_ptr(user[i]);
    at[i] = stage_bytes;
    if (staged[i]) stage_bytes += (esz[i] * static_cast<size_t>(n_w) + 15) & ~size_t(15);
  }
  const bool max_staged = evr->max_occ && !is_device_ptr(evr->max_occ);
  at[5] = stage_bytes;
  if (max_staged) stage_bytes += sizeof(double) * static_cast<size_t>(n_out);
  if (stage_bytes > 0 && (rc = reserve(c, c->evr_stage, stage_bytes))) return rc;
  char* stage = static_cast<char*>(c->evr_stage.ptr);
  void* dev[6];
  for (int i = 0; i < 5; ++i) dev[i] = staged[i] ? static_cast<void*>(stage + at[i]) : (n_w > 0 ? user[i] : nullptr);
  dev[5] = max_staged ? static_cast<void*>(stage + at[5]) : static_cast<void*>(evr->max_occ);
  ara::EventRowsParams q{};
  q.off = pl.g.off;
  q.pair_event = pl.ix.pev;
  q.t_begin = p.t_begin;
  q.t_end = p.t_end;
  q.n_tiles = n_tiles;
  q.e0 = p.e0;
  q.ev_buf = p.ev_buf;
  q.occ = p.occ;
  q.tile_cnt = p.tile_cnt;
  q.row_base = d_base;
  q.agg_r = p.agg_r;
  q.agg_l = p.agg_l;
  q.cap = n_w;
  q.row_trial = static_cast<int64_t*>(dev[0]);
  q.row_k = static_cast<int32_t*>(dev[1]);
  q.row_event = static_cast<int32_t*>(dev[2]);
  q.row_occ = static_cast<double*>(dev[3]);
  q.row_inc = static_cast<double*>(dev[4]);
  q.max_occ = static_cast<double*>(dev[5]);
  if (q.max_occ) ARA_CUDA(c, cudaMemsetAsync(q.max_occ, 0, sizeof(double) * n_out, c->stream));
  ARA_CUDA(c, ara::launch_event_rows(q, c->num_sms, c->stream));
  *launched += 1;
  for (int i = 0; i < 5; ++i)
    if (staged[i])
      ARA_CUDA(c, cudaMemcpyAsync(user[i], dev[i], esz[i] * n_w, cudaMemcpyDeviceToHost, c->stream));
  if (max_staged)
    ARA_CUDA(c, cudaMemcpyAsync(evr->max_occ, dev[5], sizeof(double) * n_out, cudaMemcpyDeviceToHost, c->stream));
  evr->n_rows = n_rows;
  return ARA_OK;
}

static int run_layer_impl(ara_ctx* c, const ara_layer* L, uint64_t seed, int64_t t0, int64_t t1, double* ylt_out,
                          const ara_diag* diag, ara_event_rows* evr = nullptr) {
  const char* who = evr ? "ara_run_layer_events" : "ara_run_layer";
  int rc = bind(c);
  if (rc) return rc;
  if (!L || !ylt_out) return fail(c, ARA_EINVAL, "%s: layer and ylt_out are required", who);
  std::vector<int32_t> ids;
  if ((rc = check_trial_range(c, t0, t1, who)) || (rc = check_layer(c, L, who, &ids))) return rc;
  PassPlan pl;
  if ((rc = plan_pass(c, ids, t0, t1, who, &pl))) return rc;
  ara::LossParams p{};
  for (size_t i = 0; i < ids.size(); ++i) {
    const Elt& el = c->pool.find(ids[i])->second;
    p.elt_id[i] = philox_elt_word(ids[i], L->flags);
    p.tab[i] = static_cast<const float4*>(el.tab.ptr);
    p.tabf[i] = static_cast<const float4*>(el.tabf.ptr);
    p.t_ret[i] = el.terms.retention;
    p.t_lim[i] = el.terms.limit;
    p.t_share[i] = el.terms.share;
  }
  // ---- outputs
  const int64_t n_out = pl.n_out;
  const bool ylt_dev = is_device_ptr(ylt_out);
  double* d_ylt = ylt_out;
  if (!ylt_dev) {
    if ((rc = reserve(c, c->ylt_tmp, sizeof(double) * n_out))) return rc;
    d_ylt = static_cast<double*>(c->ylt_tmp.ptr);
  }
  int64_t* d_hits = nullptr;
  uint64_t* d_hash = nullptr;
  const bool hits_dev = diag && diag->hits && is_device_ptr(diag->hits);
  const bool hash_dev = diag && diag->hit_hash && is_device_ptr(diag->hit_hash);
  if (diag && (diag->hits || diag->hit_hash)) {
    if ((rc = reserve(c, c->diag_tmp, 2 * sizeof(int64_t) * n_out))) return rc;
    if (diag->hits) d_hits = hits_dev ? diag->hits : static_cast<int64_t*>(c->diag_tmp.ptr);
    if (diag->hit_hash) d_hash = hash_dev ? diag->hit_hash : reinterpret_cast<uint64_t*>(static_cast<int64_t*>(c->diag_tmp.ptr) + n_out);
  }
  // ---- losses parameters
  p.off = pl.g.off;
  p.t_begin = t0;
  p.t_end = t1;
  p.n_tiles = pl.n_tiles;
  p.e0 = pl.e0;
  p.ev_buf = pl.g.ev_buf;
  p.tile_cnt = pl.g.tile_cnt;
  p.pairs = pl.ix.pairs;
  p.hot = pl.ix.hot;
  p.pw = pl.ix.pw;
  p.n_elts = L->n_elts;
  p.occ_r = static_cast<float>(L->occ_retention);
  p.occ_l = static_cast<float>(L->occ_limit);
  p.agg_r = L->agg_retention;
  p.agg_l = L->agg_limit;
  p.seed_lo = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  p.seed_hi = static_cast<uint32_t>(seed >> 32);
  fill_philox_keys(seed, p.rk);
  p.primary_only = (L->flags & ARA_PRIMARY_ONLY) ? 1 : 0;
  p.newton_only = (L->flags & ARA_NEWTON_ONLY) ? 1 : 0;
  p.ylt = d_ylt;
  p.def_acc = static_cast<double*>(c->def_acc.ptr);
  p.diag_hits = d_hits;
  p.diag_hash = d_hash;
  p.counters = static_cast<unsigned long long*>(c->counters.ptr);
  if (evr) {
    const int64_t n_ev = c->h_off[t1] - pl.e0;
    if (n_ev >= (int64_t(1) << 32) - 1)
      return fail(c, ARA_EINVAL, "%s: the trial range holds %lld YET entries (at most 2^32 - 2)", who,
                  (long long)n_ev);
    if ((rc = reserve(c, c->ev_occ, sizeof(float) * (n_ev + 1)))) return rc;
    p.occ = static_cast<float*>(c->ev_occ.ptr);
  }
  const int64_t loss_warps = ara::kLossThreads / 32;
  const int loss_grid = static_cast<int>(std::min<int64_t>(c->num_sms * ara::kLossBlocksPerSm,
                                                           (pl.n_tiles + loss_warps - 1) / loss_warps));
  // ---- launch
  int launched = 0;
  if ((rc = launch_index_and_gather(c, pl, who, &launched))) return rc;
  cudaEvent_t la, lb;
  if (!timed_pair(c, 3, &la, &lb)) return fail(c, ARA_ECUDA, "%s: cannot create timing events", who);
  ARA_CUDA(c, record_ev(la, c->stream));
  ARA_CUDA(c, ara::launch_losses(p, loss_grid, c->stream));
  ARA_CUDA(c, record_ev(lb, c->stream));
  ARA_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  launched += 1;
  if (evr && (rc = emit_event_rows(c, pl, p, evr, &launched))) return rc;
  c->launches += launched;
  if (!ylt_dev)
    ARA_CUDA(c, cudaMemcpyAsync(ylt_out, d_ylt, sizeof(double) * n_out, cudaMemcpyDeviceToHost, c->stream));
  if (d_hits && !hits_dev)
    ARA_CUDA(c, cudaMemcpyAsync(diag->hits, d_hits, sizeof(int64_t) * n_out, cudaMemcpyDeviceToHost, c->stream));
  if (d_hash && !hash_dev)
    ARA_CUDA(c, cudaMemcpyAsync(diag->hit_hash, d_hash, sizeof(uint64_t) * n_out, cudaMemcpyDeviceToHost, c->stream));
  if (!ylt_dev || (d_hits && !hits_dev) || (d_hash && !hash_dev) || evr)
    ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  record_pass_stats(c, pl, t0, t1, L->n_elts);
  return ARA_OK;
}

// Fixed-point exponent of a batched layer: a trial's sum of occurrence losses
// is counted as O * 2^e in 64 bits.  O is at most O_max (the layer's occurrence
// limit, or its largest possible event loss above the retention), a trial has
// at most n_max events, so e = 61 - ceil(log2(n_max + 1)) - ceil(log2(O_max))
// keeps every sum below 2^61.  e is kept within FP32's normal exponents (2^e
// is then an FP32 number); only an O_max below 2^-80 or above 2^150 meets the
// bounds.
static int batch_scale_exp(double o_max, int64_t n_max) {
  if (!(o_max > 0.0) || !std::isfinite(o_max)) return 0;
  const int e = 61 - static_cast<int>(std::ceil(std::log2(static_cast<double>(n_max) + 1.0))) -
                static_cast<int>(std::ceil(std::log2(o_max)));
  return std::max(-126, std::min(127, e));
}

// layer_t_end (NULL: t1 for every layer): layer l's trials end at
// min(layer_t_end[l], t1); later trials cost no loss computations and get no
// output (the serving loop's requests over their own prefixes).  ylt_l (NULL:
// ylt_out, layer-major): per layer, a device array that receives the year
// losses of trials [t0, layer end) from index 0; the call then neither copies
// nor synchronises.
static int run_layers_impl(ara_ctx* c, int32_t n_layers, const ara_layer* layers, uint64_t seed, int64_t t0,
                           int64_t t1, double* ylt_out, const int64_t* layer_t_end = nullptr,
                           double* const* ylt_l = nullptr) {
  static const char* who = "ara_run_layers";
  int rc = bind(c);
  if (rc) return rc;
  if (n_layers < 1 || n_layers > ARA_MAX_BATCH_LAYERS || !layers || (!ylt_out && !ylt_l))
    return fail(c, ARA_EINVAL, "%s: need 1..%d layers and ylt_out", who, ARA_MAX_BATCH_LAYERS);
  if ((rc = check_trial_range(c, t0, t1, who))) return rc;
  std::vector<std::vector<int32_t>> lids(n_layers);
  std::vector<int32_t> uni;
  for (int32_t l = 0; l < n_layers; ++l) {
    if ((rc = check_layer(c, &layers[l], who, &lids[l]))) return rc;
    if (layers[l].flags != layers[0].flags) return fail(c, ARA_EINVAL, "%s: the layers' flags differ", who);
    uni.insert(uni.end(), lids[l].begin(), lids[l].end());
  }
  std::sort(uni.begin(), uni.end());
  uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
  if (uni.size() > static_cast<size_t>(ARA_MAX_BATCH_ELTS))
    return fail(c, ARA_EINVAL, "%s: the layers cover %zu ELTs (at most %d)", who, uni.size(), ARA_MAX_BATCH_ELTS);
  PassPlan pl;
  if ((rc = plan_pass(c, uni, t0, t1, who, &pl))) return rc;
  ara::BatchParams p{};
  std::vector<float> gmax(n_layers, 0.0f);
  for (size_t i = 0; i < uni.size(); ++i) {
    const Elt& el = c->pool.find(uni[i])->second;
    p.elt_id[i] = philox_elt_word(uni[i], layers[0].flags);
    p.tab[i] = static_cast<const float4*>(el.tab.ptr);
    p.tabf[i] = static_cast<const float4*>(el.tabf.ptr);
    p.t_ret[i] = el.terms.retention;
    p.t_lim[i] = el.terms.limit;
    p.t_share[i] = el.terms.share;
  }
  for (int32_t l = 0; l < n_layers; ++l) {
    const ara_layer& L = layers[l];
    double g_max = 0.0;  // the layer's largest possible event loss after ELT terms
    for (int32_t id : lids[l]) {
      const size_t pos = std::lower_bound(uni.begin(), uni.end(), id) - uni.begin();
      p.layers_of[pos] |= 1ull << l;
      const Elt& el = c->pool.find(id)->second;
      const double lj = std::min(static_cast<double>(el.terms.limit),
                                 std::max(0.0, static_cast<double>(el.max_loss) - el.terms.retention));
      g_max += static_cast<double>(el.terms.share) * lj;
    }
    const double o_max = std::min(L.occ_limit, std::max(0.0, g_max - L.occ_retention));
    p.occ_r[l] = static_cast<float>(L.occ_retention);
    p.occ_l[l] = static_cast<float>(L.occ_limit);
    p.agg_r[l] = L.agg_retention;
    p.agg_l[l] = L.agg_limit;
    const int e = batch_scale_exp(o_max, c->max_trial_events);
    p.scale[l] = std::ldexp(1.0f, e);
    p.inv_scale[l] = std::ldexp(1.0, -e);
    p.layer_t_end[l] = layer_t_end ? std::min(layer_t_end[l], t1) : t1;
  }
  // ---- outputs
  const int64_t n_out = pl.n_out;
  const bool ylt_dev = ylt_l || is_device_ptr(ylt_out);
  double* d_ylt = ylt_out;
  if (!ylt_dev) {
    if ((rc = reserve(c, c->ylt_tmp, sizeof(double) * n_out * n_layers))) return rc;
    d_ylt = static_cast<double*>(c->ylt_tmp.ptr);
  }
  for (int32_t l = 0; l < n_layers; ++l) p.ylt_l[l] = ylt_l ? ylt_l[l] : d_ylt + static_cast<int64_t>(l) * n_out;
  p.off = pl.g.off;
  p.t_begin = t0;
  p.t_end = t1;
  p.n_tiles = pl.n_tiles;
  p.e0 = pl.e0;
  p.ev_buf = pl.g.ev_buf;
  p.tile_cnt = pl.g.tile_cnt;
  p.pairs = pl.ix.pairs;
  p.hot = pl.ix.hot;
  p.pw = pl.ix.pw;
  p.n_elts = static_cast<int32_t>(uni.size());
  p.n_layers = n_layers;
  fill_philox_keys(seed, p.rk);
  p.primary_only = (layers[0].flags & ARA_PRIMARY_ONLY) ? 1 : 0;
  p.newton_only = (layers[0].flags & ARA_NEWTON_ONLY) ? 1 : 0;
  p.counters = static_cast<unsigned long long*>(c->counters.ptr);
  // expected hit records per trial: each union ELT's records over the catalogue, times the
  // events per trial, weighted by the share of the pass's trials its layers reach
  double recs_per_trial = 0.0;
  for (size_t i = 0; i < uni.size(); ++i) {
    double reach = 0.0;
    for (int32_t l = 0; l < n_layers; ++l)
      if ((p.layers_of[i] >> l) & 1ull)
        reach = std::max(reach, static_cast<double>(p.layer_t_end[l] - t0) / static_cast<double>(t1 - t0));
    recs_per_trial += reach * static_cast<double>(c->pool.find(uni[i])->second.n);
  }
  recs_per_trial *= static_cast<double>(c->n_events) / (static_cast<double>(c->n_trials) * c->catalogue);
  // The losses kernel's configuration: the work item and the CTAs per SM.  Default
  // rule: the dense item with all the CTAs an SM holds.  Every configuration adds
  // the same fixed-point numbers, so none changes a result.
  const std::vector<int64_t> shape = {n_layers, static_cast<int64_t>(uni.size()), t1 - t0,
                                      static_cast<int64_t>(std::lround(4.0 * std::log2(recs_per_trial + 1.0)))};
  const int dense_max = ara::losses_dense_blocks_per_sm(n_layers);
  if (dense_max < 1) return fail(c, ARA_ECUDA, "%s: the dense losses kernel fits no SM", who);
  const int idx_max = c->yix_ready ? ara::losses_indexed_blocks_per_sm() : 0;
  if (c->yix_ready && idx_max < 1) return fail(c, ARA_ECUDA, "%s: the indexed losses kernel fits no SM", who);
  auto max_blocks = [&](int it) {
    return it == ara::kItemDense ? dense_max : it == ara::kItemIndexed ? idx_max : ara::kBatchBlocksPerSm;
  };
  // with the YET's event-major index built, the default is the indexed item (no gather)
  int item = c->yix_ready ? ara::kItemIndexed : ara::kItemDense, blocks = max_blocks(item);
  std::vector<int64_t> tshape = shape;
  tshape.push_back(c->yix_ready ? 1 : 0);
  const auto cached = c->tune_cache.find(tshape);
  const bool forced = c->force_item != ARA_BATCH_AUTO;
  const bool tune = !forced && cached == c->tune_cache.end() && (layers[0].flags & ARA_AUTOTUNE);
  if (forced) {
    if (c->force_item == ara::kItemIndexed && !c->yix_ready)
      return fail(c, ARA_EINVAL, "%s: the indexed work item needs ara_build_yet_index first", who);
    item = c->force_item;
    blocks = c->force_blocks > 0 ? std::min(c->force_blocks, max_blocks(item)) : max_blocks(item);
  } else if (cached != c->tune_cache.end()) {
    item = cached->second.first;
    blocks = cached->second.second;
  }
  const int64_t warps = ara::kBatchThreads / 32;
  auto grid_of = [&](int it, int b) {
    const int64_t items = it == ara::kItemTrial     ? pl.n_tiles * ara::kWarpTrials
                          : it == ara::kItemIndexed ? pl.ix.n_recs
                                                    : pl.n_tiles;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(static_cast<int64_t>(c->num_sms) * b,
                                                                   (items + warps - 1) / warps)));
  };
  // the indexed pass: the union's distinct events, and per-layer fixed-point sums
  ara::IndexedParams q{};
  const bool use_index = item == ara::kItemIndexed || (tune && c->yix_ready);
  if (use_index) {
    const int64_t n_recs = pl.ix.n_recs;
    if ((rc = reserve(c, c->u_flags, sizeof(uint32_t) * (n_recs + 1))) ||
        (rc = reserve(c, c->u_scan, sizeof(uint32_t) * (n_recs + 1))) ||
        (rc = reserve(c, c->u_event, sizeof(int32_t) * (n_recs + 1))) ||
        (rc = reserve(c, c->u_first, sizeof(uint32_t) * (n_recs + 1))) ||
        (rc = reserve(c, c->idx_acc,
                      sizeof(unsigned long long) * (n_layers * n_out + idx_queue_words(t0, t1, n_layers)))))
      return rc;
    q.b = p;
    q.occ = static_cast<const unsigned long long*>(c->yix_occ.ptr);
    q.ev_grid = static_cast<const uint32_t*>(c->yix_grid.ptr);
    q.grid_cells = ara::yet_grid_cells(c->n_trials, kYetGridShift);
    q.grid_shift = kYetGridShift;
    q.slice_shift = idx_slice_shift(n_layers);
    q.u_event = static_cast<const int32_t*>(c->u_event.ptr);
    q.u_first = static_cast<const uint32_t*>(c->u_first.ptr);
    q.n_u = static_cast<const uint32_t*>(c->u_scan.ptr) + n_recs;
    q.acc = static_cast<unsigned long long*>(c->idx_acc.ptr);
    q.yet_trials = c->n_trials;
    q.slice_queue = reinterpret_cast<uint32_t*>(q.acc + n_layers * n_out);
  }
  // the sums and the slices' queues, zeroed by one memset
  const size_t acc_bytes = sizeof(unsigned long long) * (n_layers * n_out + idx_queue_words(t0, t1, n_layers));
  auto launch_item = [&](int it, int b) -> cudaError_t {
    if (it != ara::kItemIndexed) return ara::launch_losses_batch(p, it, grid_of(it, b), c->stream);
    cudaError_t e = cudaMemsetAsync(q.acc, 0, acc_bytes, c->stream);
    if (e == cudaSuccess) e = ara::launch_losses_indexed(q, grid_of(it, b), c->stream);
    if (e == cudaSuccess) e = ara::launch_indexed_years(q, c->stream);
    return e;
  };
  int launched = 0;
  if (item == ara::kItemIndexed && !tune) {
    if ((rc = launch_index(c, pl, who, &launched))) return rc;
  } else if ((rc = launch_index_and_gather(c, pl, who, &launched))) {
    return rc;
  }
  if (use_index) {
    cudaEvent_t ua, ub;  // the union's events stand where the gather stands in a pass's timing
    if (!timed_pair(c, 0, &ua, &ub)) return fail(c, ARA_ECUDA, "%s: cannot create timing events", who);
    ARA_CUDA(c, record_ev(ua, c->stream));
    ARA_CUDA(c, ara::launch_union_events(pl.ix.pev, pl.ix.n_recs, static_cast<uint32_t*>(c->u_flags.ptr),
                                         static_cast<uint32_t*>(c->u_scan.ptr), pl.ix.scan_tmp,
                                         static_cast<int32_t*>(c->u_event.ptr), static_cast<uint32_t*>(c->u_first.ptr),
                                         c->stream, &launched));
    ARA_CUDA(c, record_ev(ub, c->stream));
  }
  if (tune) {
    // every candidate once on this pass's records, timed on the stream; the fastest is kept
    float best = 0.0f;
    for (auto& e : c->tune_ev)
      if (!e) ARA_CUDA(c, cudaEventCreate(&e));
    for (int it : {static_cast<int>(ara::kItemTile), static_cast<int>(ara::kItemTrial),
                   static_cast<int>(ara::kItemDense), ara::kItemIndexed})
      for (int b = 2; b <= max_blocks(it); ++b) {
        ARA_CUDA(c, cudaMemsetAsync(c->counters.ptr, 0, 4 * sizeof(unsigned long long), c->stream));
        ARA_CUDA(c, cudaEventRecord(c->tune_ev[0], c->stream));
        ARA_CUDA(c, launch_item(it, b));
        ARA_CUDA(c, cudaEventRecord(c->tune_ev[1], c->stream));
        ARA_CUDA(c, cudaEventSynchronize(c->tune_ev[1]));
        float ms = 0.0f;
        ARA_CUDA(c, cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]));
        launched += it == ara::kItemIndexed ? 2 : 1;
        if (best == 0.0f || ms < best) {
          best = ms;
          item = it;
          blocks = b;
        }
      }
    c->tune_cache[tshape] = {item, blocks};
    ARA_CUDA(c, cudaMemsetAsync(c->counters.ptr, 0, 4 * sizeof(unsigned long long), c->stream));
  }
  cudaEvent_t la, lb;
  if (!timed_pair(c, 3, &la, &lb)) return fail(c, ARA_ECUDA, "%s: cannot create timing events", who);
  ARA_CUDA(c, record_ev(la, c->stream));
  ARA_CUDA(c, launch_item(item, blocks));
  ARA_CUDA(c, record_ev(lb, c->stream));
  ARA_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  launched += item == ara::kItemIndexed ? 2 : 1;
  c->last_item = item;
  c->last_blocks = blocks;
  c->last_tuned = !forced && (cached != c->tune_cache.end() || tune) ? 1 : 0;
  c->launches += launched;
  if (!ylt_dev) {
    ARA_CUDA(c, cudaMemcpyAsync(ylt_out, d_ylt, sizeof(double) * n_out * n_layers, cudaMemcpyDeviceToHost,
                                c->stream));
    ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  int64_t elts = 0;
  for (int32_t l = 0; l < n_layers; ++l) elts += static_cast<int64_t>(lids[l].size());
  record_pass_stats(c, pl, t0, t1, elts);
  c->stats.batch_item = c->last_item;
  c->stats.batch_blocks_per_sm = c->last_blocks;
  c->stats.batch_tuned = c->last_tuned;
  return ARA_OK;
}

int ara_run_layer(ara_ctx* c, const ara_layer* L, uint64_t seed, int64_t t0, int64_t t1, double* ylt_out) {
  return run_layer_impl(c, L, seed, t0, t1, ylt_out, nullptr);
}

int ara_run_layers(ara_ctx* c, int32_t n_layers, const ara_layer* layers, uint64_t seed, int64_t t0, int64_t t1,
                   double* ylt_out) {
  return run_layers_impl(c, n_layers, layers, seed, t0, t1, ylt_out);
}

static_assert(ARA_BATCH_ITEM_TILE == ara::kItemTile && ARA_BATCH_ITEM_TRIAL == ara::kItemTrial &&
                  ARA_BATCH_ITEM_DENSE == ara::kItemDense && ARA_BATCH_ITEM_INDEXED == ara::kItemIndexed,
              "work items of the ABI and the kernels");

int ara_build_yet_index(ara_ctx* c) {
  static const char* who = "ara_build_yet_index";
  int rc = bind(c);
  if (rc) return rc;
  if ((rc = yet_finish(c))) return rc;
  if (!c->yet_loaded) return fail(c, ARA_ENOTLOADED, "%s: no YET loaded", who);
  if (c->yix_ready) return ARA_OK;
  if (!c->serve_queue.empty() || !c->serve_active.empty() || !c->serve_rounds.empty())
    return fail(c, ARA_EINVAL, "%s: served requests are queued or running", who);
  if (c->n_events >= (int64_t(1) << 32) - 1)
    return fail(c, ARA_EINVAL, "%s: the YET holds 2^32 or more events", who);
  const int64_t n = c->n_events;
  const int64_t cells = ara::yet_grid_cells(c->n_trials, kYetGridShift);
  DevBuf scratch;
  if ((rc = reserve(c, c->yix_occ, sizeof(unsigned long long) * (n + 1))) ||
      (rc = reserve(c, c->yix_grid, sizeof(uint32_t) * (static_cast<size_t>(c->catalogue) * (cells + 1) + 1))) ||
      (rc = reserve(c, scratch, ara::yet_bucket_scratch_bytes(c->catalogue, cells)))) {
    release(c, scratch);
    release(c, c->yix_occ);
    release(c, c->yix_grid);
    return rc;
  }
  const int64_t* off = static_cast<const int64_t*>(c->yet_off.ptr);
  const int32_t* ids = static_cast<const int32_t*>(c->yet_ids.ptr);
  unsigned long long* occ = static_cast<unsigned long long*>(c->yix_occ.ptr);
  uint32_t* grid = static_cast<uint32_t*>(c->yix_grid.ptr);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
  int launched = 0;
  // buckets per (event, grid cell) while the largest is small; else the radix sort
  uint32_t max_bucket = 0;
  if (e == cudaSuccess)
    e = ara::yet_index_count(off, ids, c->n_trials, c->catalogue, kYetGridShift, grid, scratch.ptr, c->stream,
                             &launched);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&max_bucket, ara::yet_index_max_bucket(scratch.ptr, c->catalogue, cells), sizeof max_bucket,
                        cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  const bool buckets = max_bucket <= kYetBucketSortMax;
  if (e == cudaSuccess && buckets)
    e = ara::yet_index_fill(off, ids, c->n_trials, c->catalogue, kYetGridShift, grid, occ, scratch.ptr, c->stream,
                            &launched);
  if (e == cudaSuccess && !buckets) {
    release(c, scratch);
    if ((rc = reserve(c, scratch, ara::yet_index_scratch_bytes(n, c->catalogue)))) {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      release(c, c->yix_occ);
      release(c, c->yix_grid);
      return rc;
    }
    e = ara::build_yet_index(off, ids, c->n_trials, n, c->catalogue, kYetGridShift, occ, grid, scratch.ptr, c->stream,
                             &launched);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  release(c, scratch);
  c->launches += launched;
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(c, c->yix_occ);
    release(c, c->yix_grid);
    return fail(c, ARA_ECUDA, "%s: %s", who, cudaGetErrorString(e));
  }
  c->yix_sorted = !buckets;
  c->yix_ready = true;
  c->yix_build_ms = ms;
  c->serve_ready = false;  // the serving arena is sized again around the index
  return ARA_OK;
}

int ara_yet_index_info(const ara_ctx* c, int32_t* built, int64_t* bytes, float* build_ms, int32_t* method) {
  if (!c) return ARA_EINVAL;
  if (built) *built = c->yix_ready ? 1 : 0;
  if (method) *method = c->yix_ready ? (c->yix_sorted ? 1 : 0) : -1;
  if (bytes) *bytes = c->yix_ready ? static_cast<int64_t>(c->yix_occ.bytes + c->yix_grid.bytes) : 0;
  if (build_ms) *build_ms = c->yix_ready ? c->yix_build_ms : 0.0f;
  return ARA_OK;
}

int ara_set_batch_config(ara_ctx* c, int32_t item, int32_t blocks_per_sm) {
  int rc = bind(c);
  if (rc) return rc;
  if (item != ARA_BATCH_AUTO && item != ARA_BATCH_ITEM_TILE && item != ARA_BATCH_ITEM_TRIAL &&
      item != ARA_BATCH_ITEM_DENSE && item != ARA_BATCH_ITEM_INDEXED)
    return fail(c, ARA_EINVAL, "ara_set_batch_config: unknown work item %d", item);
  if (blocks_per_sm < 0 || blocks_per_sm > 16)
    return fail(c, ARA_EINVAL, "ara_set_batch_config: blocks_per_sm %d outside 0..16", blocks_per_sm);
  c->force_item = item;
  c->force_blocks = blocks_per_sm;
  return ARA_OK;
}

int ara_run_layer_diag(ara_ctx* c, const ara_layer* L, uint64_t seed, int64_t t0, int64_t t1, double* ylt_out,
                       const ara_diag* diag) {
  return run_layer_impl(c, L, seed, t0, t1, ylt_out, diag);
}

int ara_run_layer_events(ara_ctx* c, const ara_layer* L, uint64_t seed, int64_t t0, int64_t t1, double* ylt_out,
                         ara_event_rows* rows) {
  int rc = bind(c);
  if (rc) return rc;
  if (!rows || rows->capacity < 0)
    return fail(c, ARA_EINVAL, "ara_run_layer_events: rows is NULL or its capacity is negative");
  rows->n_rows = 0;
  return run_layer_impl(c, L, seed, t0, t1, ylt_out, nullptr, rows);
}

int ara_get_stats(const ara_ctx* cc, ara_stats* out) {
  ara_ctx* c = const_cast<ara_ctx*>(cc);
  int rc = bind(c);
  if (rc) return rc;
  if (!out) return fail(c, ARA_EINVAL, "ara_get_stats: out is NULL");
  if (c->stats.kernel_ms < 0.0f) {
    ARA_CUDA(c, cudaEventSynchronize(c->ev[3]));
    float ms = 0.0f;
    ARA_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    c->stats.index_ms = ms;
    ARA_CUDA(c, cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
    c->stats.kernel_ms = ms;
    unsigned long long h[4];
    ARA_CUDA(c, cudaMemcpy(h, c->counters.ptr, sizeof h, cudaMemcpyDeviceToHost));
    c->stats.n_pairs_hit = static_cast<int64_t>(h[1]);
    c->stats.n_nonconverged = static_cast<int64_t>(h[2]);
    c->stats.n_newton = static_cast<int64_t>(h[3]);
  }
  *out = c->stats;
  return ARA_OK;
}

int ara_get_timing(ara_ctx* c, ara_timing* out, int reset) {
  int rc = bind(c);
  if (rc) return rc;
  if (!out) return fail(c, ARA_EINVAL, "ara_get_timing: out is NULL");
  *out = ara_timing{};
  for (const auto& t : c->timed) {
    ARA_CUDA(c, cudaEventSynchronize(t.b));
    float ms = 0.0f;
    ARA_CUDA(c, cudaEventElapsedTime(&ms, t.a, t.b));
    if (t.kind == 0) {
      out->layer_calls += 1;
      out->kernel_ms += ms;
      out->gather_ms += ms;
    } else if (t.kind == 3) {
      out->kernel_ms += ms;
      out->losses_ms += ms;
    } else if (t.kind == 1) {
      out->index_ms += ms;
    } else {
      out->pml_calls += 1;
      out->pml_ms += ms;
    }
  }
  out->kernel_launches = c->launches;
  if (reset) {
    c->timed.clear();
    c->launches = 0;
  }
  return ARA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- serving
// Continuous batching.  A request's trial prefix is cut into chunks of
// kServeChunk trials; an admitted request has a cursor, its next chunk.
// ara_serve_step retires the rounds the device has finished (cudaEventQuery,
// no waiting), admits queued requests whose year losses fit the serving
// arena, and launches one round: batched passes (ara_run_layers over one
// chunk), kServePassesShort at most while kServeShortBacklog or fewer requests
// have chunks to run, else kServePassesPerRound, each for up to ARA_MAX_BATCH_LAYERS
// admitted requests that are at the same chunk, with one seed and flags and
// at most ARA_MAX_BATCH_ELTS ELTs together, every layer writing its chunk
// into its own request's year losses.  Behind a request's last chunk the
// round queues its PML/TVaR select and the copy of the results to pinned
// host memory.  The step returns with the round in flight: requests
// submitted meanwhile join the next round, and at most kServeMaxInFlight
// rounds are in flight.
namespace {

constexpr int64_t kServeChunk = 262144;        // trials per chunk
constexpr size_t kServeSelectPool = size_t{256} << 20;  // scratch of a pass's batched selects, at most
static_assert(kServeChunk == int64_t{1} << kYetGridShift, "served chunks' bounds are the YET index's grid bounds");
constexpr size_t kServeMaxInFlight = 2;        // rounds launched and not retired
constexpr int kServePassesPerRound = 16;       // a round's passes under a long backlog
constexpr int kServePassesShort = 4;           // ... and under a short one
constexpr size_t kServeShortBacklog = 128;     // requests with chunks to run, at most, for a short backlog

// The pool of a pass's batched selects: a batch of the largest jobs (a whole-YET prefix and four
// return periods) within kServeSelectPool, and never less than one of them.
size_t serve_select_pool_bytes(int64_t n_trials) {
  const size_t one = ara::select_job_bytes(n_trials, 4);
  return std::max(one, std::min(kServeSelectPool, one * 32));
}
constexpr int32_t kServeSlots = 1024;          // result slots: admitted requests at most
constexpr int64_t kServeArenaRequests = 96;    // default arena: year losses of this many whole-YET requests
constexpr size_t kArenaAlign = 256;

size_t arena_round(size_t bytes) { return (bytes + kArenaAlign - 1) & ~(kArenaAlign - 1); }

bool arena_alloc(ara_ctx* c, size_t bytes, size_t* off) {
  bytes = arena_round(bytes);
  for (auto it = c->arena_free.begin(); it != c->arena_free.end(); ++it) {
    if (it->second < bytes) continue;
    *off = it->first;
    const size_t rest = it->second - bytes, at = it->first + bytes;
    c->arena_free.erase(it);
    if (rest) c->arena_free[at] = rest;
    return true;
  }
  return false;
}

void arena_release(ara_ctx* c, size_t off, size_t bytes) {
  bytes = arena_round(bytes);
  auto next = c->arena_free.lower_bound(off);
  if (next != c->arena_free.end() && off + bytes == next->first) {
    bytes += next->second;
    next = c->arena_free.erase(next);
  }
  if (next != c->arena_free.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      prev->second += bytes;
      return;
    }
  }
  c->arena_free[off] = bytes;
}

// Device buffers the serving passes use besides the arena, with the sizes they
// need: the event buffer of the largest chunk, the tile counts and deferred
// sums of a chunk, the layer index of the pool's ARA_MAX_BATCH_ELTS largest
// ELTs, the select scratch for the whole YET and the result slots.  The
// serving loop reserves them before it sizes the arena, so that no pass grows
// a buffer while rounds are in flight.
std::vector<std::pair<DevBuf*, size_t>> serve_workspace(ara_ctx* c) {
  int64_t max_ev = 0;
  for (int64_t t0 = 0; t0 < c->n_trials; t0 += kServeChunk) {
    const int64_t t1 = std::min(t0 + kServeChunk, c->n_trials);
    max_ev = std::max(max_ev, c->h_off[t1] - c->h_off[t0]);
  }
  std::vector<int64_t> sizes;
  bool any_corr = false;
  for (const auto& kv : c->pool) {
    sizes.push_back(kv.second.n);
    any_corr = any_corr || kv.second.correlated;
  }
  std::sort(sizes.rbegin(), sizes.rend());
  int64_t n_recs = 0;
  for (size_t i = 0; i < sizes.size() && i < static_cast<size_t>(ARA_MAX_BATCH_ELTS); ++i) n_recs += sizes[i];
  const int64_t n_words = (static_cast<int64_t>(c->catalogue) + 31) / 32;
  const size_t tmp_words = std::max(ara::scan_tmp_words(n_words), ara::scan_tmp_words(n_recs));
  const size_t chunk_tiles = static_cast<size_t>(kServeChunk / ara::kWarpTrials + 2);
  std::vector<std::pair<DevBuf*, size_t>> w = {
      {&c->ev_buf, sizeof(uint2) * static_cast<size_t>(max_ev + 1)},
      {&c->tile_cnt, sizeof(uint32_t) * chunk_tiles},
      {&c->def_acc, sizeof(double) * static_cast<size_t>(kServeChunk + 1)},
      {&c->bits, sizeof(uint32_t) * n_words},
      {&c->word_cnt, sizeof(uint32_t) * (n_words + 1)},
      {&c->word_pairs, sizeof(uint32_t) * (n_words + 1)},
      {&c->rankdir, sizeof(uint2) * n_words},
      {&c->mask, sizeof(unsigned long long) * (n_recs + 1)},
      {&c->slot_cnt, sizeof(uint32_t) * (n_recs + 2)},
      {&c->pairs, sizeof(ara::Pair) * (n_recs + 1)},
      {&c->pairs_hot, sizeof(ara::PairHot) * (n_recs + 1)},
      {&c->pairs_ev, sizeof(int32_t) * (n_recs + 1)},
      {&c->scan_tmp, sizeof(uint32_t) * (tmp_words + 8)},
      {&c->serve_sel, serve_select_pool_bytes(c->n_trials)},
      {&c->u_flags, sizeof(uint32_t) * (n_recs + 1)},
      {&c->u_scan, sizeof(uint32_t) * (n_recs + 1)},
      {&c->u_event, sizeof(int32_t) * (n_recs + 1)},
      {&c->u_first, sizeof(uint32_t) * (n_recs + 1)},
      {&c->idx_acc, sizeof(unsigned long long) * (ARA_MAX_BATCH_LAYERS * static_cast<size_t>(kServeChunk) +
                                                  idx_queue_words(0, kServeChunk, ARA_MAX_BATCH_LAYERS))},
      {&c->serve_out, 2 * sizeof(double) * ARA_SERVE_MAX_RP * kServeSlots},
  };
  if (any_corr) w.push_back({&c->pairs_w, sizeof(float2) * (n_recs + 1)});
  return w;
}

// The arena's size: once prepared, its size; before, what the budget leaves
// once the workspace is reserved, or room for kServeArenaRequests whole-YET
// requests without a budget.
size_t serve_arena_bytes(ara_ctx* c) {
  if (c->serve_ready) return c->serve_arena.bytes;
  if (!c->budget) return arena_round(sizeof(double) * static_cast<size_t>(c->n_trials)) * kServeArenaRequests;
  size_t missing = 0;
  for (const auto& w : serve_workspace(c)) missing += w.second > w.first->bytes ? w.second - w.first->bytes : 0;
  const size_t arena_now = c->serve_arena.bytes;  // released and re-reserved by the preparation
  const size_t used = c->used - arena_now + missing;
  return (c->budget > used ? c->budget - used : 0) & ~(kArenaAlign - 1);
}

// First use (and after a new YET): the workspace, the arena, the result slots.
int serve_prepare(ara_ctx* c, const char* who) {
  if (c->serve_ready) return ARA_OK;
  const size_t arena = serve_arena_bytes(c);
  release(c, c->serve_arena);
  int rc;
  for (const auto& w : serve_workspace(c))
    if ((rc = reserve(c, *w.first, w.second))) return rc;
  if (!c->serve_side && (cudaStreamCreateWithFlags(&c->serve_side, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&c->serve_join, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    return fail(c, ARA_ECUDA, "%s: cannot create the serving side stream", who);
  }
  if (!c->serve_host) {
    void* h = nullptr;
    if (cudaHostAlloc(&h, 2 * sizeof(double) * ARA_SERVE_MAX_RP * kServeSlots, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, ARA_ENOMEM, "%s: cannot allocate pinned result slots", who);
    }
    c->serve_host = static_cast<double*>(h);
  }
  if (arena < kArenaAlign) return fail(c, ARA_ENOMEM, "%s: the HBM budget leaves no room for year losses", who);
  if ((rc = reserve(c, c->serve_arena, arena))) return rc;
  c->arena_free.clear();
  c->arena_free[0] = c->serve_arena.bytes;
  c->serve_slots_free.clear();
  for (int32_t i = kServeSlots - 1; i >= 0; --i) c->serve_slots_free.push_back(i);
  c->serve_ready = true;
  return ARA_OK;
}

// Finishes the requests of the rounds the device has completed, oldest first;
// with `block`, waits for the oldest round first.  *n_done counts them.
int serve_retire(ara_ctx* c, bool block, int32_t* n_done) {
  while (!c->serve_rounds.empty()) {
    ServeRound& r = c->serve_rounds.front();
    const cudaError_t e = block ? cudaEventSynchronize(r.ev) : cudaEventQuery(r.ev);
    if (e == cudaErrorNotReady) {
      cudaGetLastError();
      break;
    }
    int status = ARA_OK;
    if (e != cudaSuccess) status = fail(c, ARA_ECUDA, "ara_serve_step: %s", cudaGetErrorString(e));
    for (int64_t tk : r.finishing) {
      ServeReq& q = c->serve_reqs[tk];
      const size_t m = q.rps.size();
      q.done = true;
      q.status = status;
      if (!status) {
        const double* h = c->serve_host + static_cast<size_t>(q.slot) * 2 * ARA_SERVE_MAX_RP;
        q.pml.assign(h, h + m);
        q.tvar.assign(h + ARA_SERVE_MAX_RP, h + ARA_SERVE_MAX_RP + m);
      }
      arena_release(c, q.ylt_off, q.ylt_bytes);
      c->serve_slots_free.push_back(q.slot);
      c->serve_active.erase(std::find(c->serve_active.begin(), c->serve_active.end(), tk));
      ++c->serve_finished;
      if (n_done) ++*n_done;
    }
    c->serve_ev_free.push_back(r.ev);
    c->serve_rounds.pop_front();
    block = false;
    if (status) return status;
  }
  return ARA_OK;
}

// Queued requests, in arrival order, whose year losses fit the arena (a
// request that does not fit yet stays queued; a later, smaller one may go).
void serve_admit(ara_ctx* c) {
  for (auto it = c->serve_queue.begin(); it != c->serve_queue.end() && !c->serve_slots_free.empty();) {
    ServeReq& q = c->serve_reqs[*it];
    size_t off = 0;
    if (!arena_alloc(c, sizeof(double) * static_cast<size_t>(q.t_end), &off)) {
      ++it;
      continue;
    }
    q.ylt_off = off;
    q.ylt_bytes = sizeof(double) * static_cast<size_t>(q.t_end);
    q.slot = c->serve_slots_free.back();
    c->serve_slots_free.pop_back();
    q.next_chunk = 0;
    q.n_chunks = (q.t_end + kServeChunk - 1) / kServeChunk;
    c->serve_active.push_back(*it);
    it = c->serve_queue.erase(it);
  }
}

// Fails the requests of a pass that could not be launched.
void serve_fail_requests(ara_ctx* c, const std::vector<int64_t>& tks, int status) {
  for (int64_t tk : tks) {
    ServeReq& q = c->serve_reqs[tk];
    q.done = true;
    q.status = status;
    arena_release(c, q.ylt_off, q.ylt_bytes);
    c->serve_slots_free.push_back(q.slot);
    c->serve_active.erase(std::find(c->serve_active.begin(), c->serve_active.end(), tk));
    ++c->serve_finished;
  }
}

int serve_launch_round(ara_ctx* c, const char* who, int32_t* n_failed) {
  std::vector<int64_t> cand;
  for (int64_t tk : c->serve_active) {
    const ServeReq& q = c->serve_reqs[tk];
    if (q.next_chunk < q.n_chunks) cand.push_back(tk);
  }
  if (cand.empty()) return ARA_OK;
  ServeRound round;
  if (!c->serve_ev_free.empty()) {
    round.ev = c->serve_ev_free.back();
    c->serve_ev_free.pop_back();
  } else if (cudaEventCreateWithFlags(&round.ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, ARA_ECUDA, "%s: cannot create an event", who);
  }
  double* arena = static_cast<double*>(c->serve_arena.ptr);
  double* d_out = static_cast<double*>(c->serve_out.ptr);
  std::vector<bool> used(cand.size(), false);
  int passes = 0, status = ARA_OK;
  c->no_timing = true;
  // short rounds while the backlog is short (a request that arrives waits for less), long ones
  // under a long backlog (fewer rounds to launch and retire)
  const int max_passes = cand.size() > kServeShortBacklog ? kServePassesPerRound : kServePassesShort;
  for (size_t i = 0; i < cand.size() && passes < max_passes; ++i) {
    if (used[i]) continue;
    const ServeReq& a = c->serve_reqs[cand[i]];
    std::vector<int64_t> members{cand[i]};
    used[i] = true;
    std::vector<int32_t> uni = a.elt_ids;
    // the pass's other members: requests at the same chunk with the same seed and flags,
    // those whose trials end closest to the first member's within the chunk first (a pass
    // streams its chunk up to its longest member's end), then in arrival order
    const int64_t c_begin = a.next_chunk * kServeChunk;
    auto len_in_chunk = [&](const ServeReq& q) { return std::min(q.t_end, c_begin + kServeChunk) - c_begin; };
    std::vector<std::pair<int64_t, size_t>> order;
    for (size_t j = i + 1; j < cand.size(); ++j) {
      if (used[j]) continue;
      const ServeReq& b = c->serve_reqs[cand[j]];
      if (b.next_chunk != a.next_chunk || b.seed != a.seed || b.layer.flags != a.layer.flags) continue;
      order.emplace_back(std::llabs(len_in_chunk(b) - len_in_chunk(a)), j);
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int64_t, size_t>& x, const std::pair<int64_t, size_t>& y) { return x.first < y.first; });
    for (const auto& o : order) {
      if (members.size() >= static_cast<size_t>(ARA_MAX_BATCH_LAYERS)) break;
      const size_t j = o.second;
      const ServeReq& b = c->serve_reqs[cand[j]];
      std::vector<int32_t> u2 = uni;
      u2.insert(u2.end(), b.elt_ids.begin(), b.elt_ids.end());
      std::sort(u2.begin(), u2.end());
      u2.erase(std::unique(u2.begin(), u2.end()), u2.end());
      if (u2.size() > static_cast<size_t>(ARA_MAX_BATCH_ELTS)) continue;
      members.push_back(cand[j]);
      used[j] = true;
      uni.swap(u2);
    }
    const int64_t t0 = a.next_chunk * kServeChunk;
    int64_t t1 = t0;
    const int32_t nm = static_cast<int32_t>(members.size());
    std::vector<ara_layer> layers(nm);
    std::vector<int64_t> t_ends(nm);
    std::vector<double*> outs(nm);
    for (int32_t m = 0; m < nm; ++m) {
      const ServeReq& q = c->serve_reqs[members[m]];
      layers[m] = q.layer;
      t_ends[m] = q.t_end;
      t1 = std::max(t1, std::min(q.t_end, t0 + kServeChunk));
      outs[m] = arena + q.ylt_off / sizeof(double) + t0;
    }
    int rc = run_layers_impl(c, nm, layers.data(), a.seed, t0, t1, nullptr, t_ends.data(), outs.data());
    // the requests whose last chunk this pass was: their PML/TVaR over their whole prefixes in one
    // batched select, then the results to the host, on the side stream once the pass is done (they
    // overlap the round's later passes)
    std::vector<ara::SelectSpec> specs;
    std::vector<int64_t> done;
    for (int32_t m = 0; m < nm && !rc; ++m) {
      ServeReq& q = c->serve_reqs[members[m]];
      if (++q.next_chunk < q.n_chunks) continue;
      double* slot = d_out + static_cast<size_t>(q.slot) * 2 * ARA_SERVE_MAX_RP;
      specs.push_back({arena + q.ylt_off / sizeof(double), q.t_end, q.rps.data(), static_cast<int32_t>(q.rps.size()),
                       slot, slot + ARA_SERVE_MAX_RP});
      done.push_back(members[m]);
    }
    if (!rc && !specs.empty()) {
      cudaError_t e = cudaEventRecord(c->serve_join, c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->serve_side, c->serve_join, 0);
      int launched = 0;
      if (e == cudaSuccess)
        e = ara::pml_tvar_batch(specs.data(), static_cast<int>(specs.size()), c->serve_sel.ptr, c->serve_sel.bytes,
                                c->serve_side, &launched);
      c->launches += launched;
      for (size_t k = 0; k < done.size() && e == cudaSuccess; ++k) {
        const ServeReq& q = c->serve_reqs[done[k]];
        e = cudaMemcpyAsync(c->serve_host + static_cast<size_t>(q.slot) * 2 * ARA_SERVE_MAX_RP, specs[k].pml,
                            2 * sizeof(double) * ARA_SERVE_MAX_RP, cudaMemcpyDeviceToHost, c->serve_side);
      }
      if (e != cudaSuccess) rc = fail(c, ARA_ECUDA, "%s: %s", who, cudaGetErrorString(e));
      else round.finishing.insert(round.finishing.end(), done.begin(), done.end());
    }
    if (rc) {
      // the pass's requests end with its error; the others of the round go on
      std::vector<int64_t> failed;
      for (int64_t tk : members)
        if (std::find(round.finishing.begin(), round.finishing.end(), tk) == round.finishing.end())
          failed.push_back(tk);
      serve_fail_requests(c, failed, rc);
      if (n_failed) *n_failed += static_cast<int32_t>(failed.size());
      status = rc;
      break;
    }
    ++passes;
  }
  c->no_timing = false;
  // the round is done when both streams are: the side stream waits for the passes, then records
  cudaError_t e = cudaEventRecord(c->serve_join, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->serve_side, c->serve_join, 0);
  if (e == cudaSuccess) e = cudaEventRecord(round.ev, c->serve_side);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->serve_ev_free.push_back(round.ev);
    serve_fail_requests(c, round.finishing, ARA_ECUDA);
    return fail(c, ARA_ECUDA, "%s: %s", who, cudaGetErrorString(e));
  }
  c->serve_rounds.push_back(std::move(round));
  ++c->serve_rounds_launched;
  c->serve_passes += passes;
  return status;
}

}  // namespace

extern "C" {

int ara_submit(ara_ctx* c, const ara_layer* L, uint64_t seed, int64_t t_end, const double* rps, int32_t n_rp,
               int64_t* ticket) {
  static const char* who = "ara_submit";
  int rc = bind(c);
  if (rc) return rc;
  if (!L || !rps || !ticket || n_rp < 1 || n_rp > ARA_SERVE_MAX_RP)
    return fail(c, ARA_EINVAL, "%s: need a layer, 1..%d return periods and a ticket", who, ARA_SERVE_MAX_RP);
  std::vector<int32_t> ids;
  if ((rc = check_trial_range(c, 0, t_end, who)) || (rc = check_layer(c, L, who, &ids))) return rc;
  for (int32_t id : ids)
    if (c->pool.find(id) == c->pool.end()) return fail(c, ARA_ENOTLOADED, "%s: ELT %d is not loaded", who, id);
  for (int32_t i = 0; i < n_rp; ++i)
    if (!(rps[i] >= 1.0) || !std::isfinite(rps[i])) return fail(c, ARA_EINVAL, "%s: return periods must be >= 1", who);
  const size_t arena = serve_arena_bytes(c);
  if (arena_round(sizeof(double) * static_cast<size_t>(t_end)) > arena)
    return fail(c, ARA_ENOMEM, "%s: the request's year losses (%lld bytes) exceed the serving arena (%zu bytes)",
                who, (long long)(sizeof(double) * t_end), arena);
  const int64_t tk = c->next_ticket++;
  ServeReq& r = c->serve_reqs[tk];
  r.elt_ids = ids;
  r.layer = *L;
  r.layer.elt_ids = r.elt_ids.data();
  r.layer.n_elts = static_cast<int32_t>(r.elt_ids.size());
  r.seed = seed;
  r.t_end = t_end;
  r.rps.assign(rps, rps + n_rp);
  c->serve_queue.push_back(tk);
  *ticket = tk;
  return ARA_OK;
}

int ara_serve_step(ara_ctx* c, int32_t* n_done) {
  static const char* who = "ara_serve_step";
  int rc = bind(c);
  if (rc) return rc;
  int32_t n = 0;
  rc = serve_retire(c, false, &n);
  if (!rc && (!c->serve_queue.empty() || !c->serve_active.empty()) && c->serve_rounds.size() < kServeMaxInFlight) {
    rc = serve_prepare(c, who);
    if (!rc) {
      serve_admit(c);
      rc = serve_launch_round(c, who, &n);
    }
  }
  if (n_done) *n_done = n;
  return rc;
}

int ara_serve_stats(ara_ctx* c, ara_serve_info* out) {
  int rc = bind(c);
  if (rc) return rc;
  if (!out) return fail(c, ARA_EINVAL, "ara_serve_stats: out is NULL");
  *out = ara_serve_info{};
  out->queued = static_cast<int64_t>(c->serve_queue.size());
  out->active = static_cast<int64_t>(c->serve_active.size());
  out->rounds_in_flight = static_cast<int64_t>(c->serve_rounds.size());
  out->rounds_launched = c->serve_rounds_launched;
  out->passes_launched = c->serve_passes;
  out->requests_finished = c->serve_finished;
  out->chunk_trials = kServeChunk;
  out->arena_bytes = static_cast<int64_t>(serve_arena_bytes(c));
  return ARA_OK;
}

int ara_poll(ara_ctx* c, int64_t ticket, double* pml_out, double* tvar_out) {
  int rc = bind(c);
  if (rc) return rc;
  auto it = c->serve_reqs.find(ticket);
  if (it == c->serve_reqs.end()) return fail(c, ARA_EINVAL, "ara_poll: unknown ticket %lld", (long long)ticket);
  if (!it->second.done) return ARA_EAGAIN;
  const int status = it->second.status;
  if (status == ARA_OK) {
    if (pml_out) std::copy(it->second.pml.begin(), it->second.pml.end(), pml_out);
    if (tvar_out) std::copy(it->second.tvar.begin(), it->second.tvar.end(), tvar_out);
  }
  c->serve_reqs.erase(it);
  return status;
}

int ara_wait(ara_ctx* c, int64_t ticket, double* pml_out, double* tvar_out, uint64_t timeout_ns) {
  int rc = bind(c);
  if (rc) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    rc = ara_poll(c, ticket, pml_out, tvar_out);
    if (rc != ARA_EAGAIN) return rc;
    if (timeout_ns) {
      const auto dt = std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0);
      if (static_cast<uint64_t>(dt.count()) >= timeout_ns)
        return fail(c, ARA_ETIMEOUT, "ara_wait: ticket %lld not finished within %llu ns", (long long)ticket,
                    (unsigned long long)timeout_ns);
    }
    int32_t n_done = 0;
    if ((rc = ara_serve_step(c, &n_done))) return rc;
    if (n_done > 0) continue;
    // nothing finished in this step: wait on the host for the oldest round in flight
    if (!c->serve_rounds.empty()) {
      if ((rc = serve_retire(c, true, nullptr))) return rc;
    } else if (ara_poll(c, ticket, nullptr, nullptr) == ARA_EAGAIN) {
      return fail(c, ARA_EINVAL, "ara_wait: ticket %lld is queued but no step can run it", (long long)ticket);
    }
  }
}

int ara_pml_tvar(ara_ctx* c, const double* ylt, int64_t n, const double* rps, int32_t n_rp, double* pml_out,
                 double* tvar_out) {
  int rc = bind(c);
  if (rc) return rc;
  if (!ylt || n < 1 || !rps || n_rp < 1 || !pml_out || !tvar_out)
    return fail(c, ARA_EINVAL, "ara_pml_tvar: bad arguments");
  std::vector<double> h_rps(n_rp);
  ARA_CUDA(c, copy_params_to_host(h_rps.data(), rps, sizeof(double) * n_rp));
  for (double r : h_rps)
    if (!(r >= 1.0) || !std::isfinite(r)) return fail(c, ARA_EINVAL, "ara_pml_tvar: return periods must be >= 1");
  const double* d_ylt = ylt;
  if (!is_device_ptr(ylt)) {
    if ((rc = reserve(c, c->in_tmp, sizeof(double) * n))) return rc;
    ARA_CUDA(c, cudaMemcpyAsync(c->in_tmp.ptr, ylt, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    d_ylt = static_cast<const double*>(c->in_tmp.ptr);
  }
  const bool pml_dev = is_device_ptr(pml_out), tvar_dev = is_device_ptr(tvar_out);
  if ((rc = reserve(c, c->sel, ara::select_scratch_bytes(n))) ||
      (rc = reserve(c, c->out_tmp, 2 * sizeof(double) * n_rp)))
    return rc;
  double* d_pml = pml_dev ? pml_out : static_cast<double*>(c->out_tmp.ptr);
  double* d_tvar = tvar_dev ? tvar_out : static_cast<double*>(c->out_tmp.ptr) + n_rp;
  cudaEvent_t pa, pb;
  if (!timed_pair(c, 2, &pa, &pb)) return fail(c, ARA_ECUDA, "ara_pml_tvar: cannot create timing events");
  int launched = 0;
  ARA_CUDA(c, cudaEventRecord(pa, c->stream));
  ARA_CUDA(c, ara::pml_tvar_device(d_ylt, n, h_rps.data(), n_rp, d_pml, d_tvar, c->sel.ptr, c->sel.bytes, c->stream,
                                   &launched));
  ARA_CUDA(c, cudaEventRecord(pb, c->stream));
  c->launches += launched;
  if (!pml_dev) ARA_CUDA(c, cudaMemcpyAsync(pml_out, d_pml, sizeof(double) * n_rp, cudaMemcpyDeviceToHost, c->stream));
  if (!tvar_dev)
    ARA_CUDA(c, cudaMemcpyAsync(tvar_out, d_tvar, sizeof(double) * n_rp, cudaMemcpyDeviceToHost, c->stream));
  if (!pml_dev || !tvar_dev || !is_device_ptr(ylt)) ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  return ARA_OK;
}

int ara_top_m(ara_ctx* c, const double* ylt, int64_t n, int64_t m, int64_t trial_offset, double* values_out,
              int64_t* trials_out) {
  static const char* who = "ara_top_m";
  int rc = bind(c);
  if (rc) return rc;
  if (!ylt || n < 1 || m < 1 || trial_offset < 0 || !values_out || !trials_out)
    return fail(c, ARA_EINVAL, "%s: bad arguments", who);
  if (n >= (int64_t(1) << 31)) return fail(c, ARA_EINVAL, "%s: at most 2^31 - 1 trials", who);
  const double* d_ylt = ylt;
  if (!is_device_ptr(ylt)) {
    if ((rc = reserve(c, c->in_tmp, sizeof(double) * n))) return rc;
    ARA_CUDA(c, cudaMemcpyAsync(c->in_tmp.ptr, ylt, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    d_ylt = static_cast<const double*>(c->in_tmp.ptr);
  }
  const bool vals_dev = is_device_ptr(values_out), trials_dev = is_device_ptr(trials_out);
  // scratch: the sort's, then the order of all n, then staged outputs for host arrays
  const size_t sort_bytes = (ara::sort_scratch_bytes(n) + 255) & ~size_t(255);
  const size_t order_bytes = (sizeof(int64_t) * static_cast<size_t>(n) + 255) & ~size_t(255);
  const size_t stage_bytes = (vals_dev && trials_dev) ? 0 : 2 * sizeof(int64_t) * static_cast<size_t>(m);
  if ((rc = reserve(c, c->sel, sort_bytes + order_bytes + stage_bytes))) return rc;
  char* base = static_cast<char*>(c->sel.ptr);
  int64_t* d_order = reinterpret_cast<int64_t*>(base + sort_bytes);
  double* d_vals = vals_dev ? values_out : reinterpret_cast<double*>(base + sort_bytes + order_bytes);
  int64_t* d_trials = trials_dev ? trials_out : reinterpret_cast<int64_t*>(base + sort_bytes + order_bytes) + m;
  int launched = 0;
  ARA_CUDA(c, ara::sort_desc_device(d_ylt, n, d_order, c->sel.ptr, c->stream, &launched));
  ARA_CUDA(c, ara::top_gather_device(d_ylt, d_order, std::min(m, n), m, trial_offset, d_vals, d_trials, c->stream));
  c->launches += launched + 1;
  if (!vals_dev)
    ARA_CUDA(c, cudaMemcpyAsync(values_out, d_vals, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
  if (!trials_dev)
    ARA_CUDA(c, cudaMemcpyAsync(trials_out, d_trials, sizeof(int64_t) * m, cudaMemcpyDeviceToHost, c->stream));
  if (!vals_dev || !trials_dev || !is_device_ptr(ylt)) ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  return ARA_OK;
}

int ara_merge_top(const double* values, const int64_t* trials, int64_t count, int64_t n_total, const double* rps,
                  int32_t n_rp, double* pml_out, double* tvar_out) {
  if (!values || !trials || count < 1 || n_total < 1 || !rps || n_rp < 1 || !pml_out || !tvar_out)
    return ARA_EINVAL;
  for (int32_t r = 0; r < n_rp; ++r)
    if (!(rps[r] >= 1.0) || !std::isfinite(rps[r])) return ARA_EINVAL;
  // the finite entries, by year loss (largest first), ties by global trial index
  std::vector<int64_t> idx;
  idx.reserve(static_cast<size_t>(count));
  for (int64_t i = 0; i < count; ++i)
    if (std::isfinite(values[i])) idx.push_back(i);
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    return values[a] > values[b] || (values[a] == values[b] && trials[a] < trials[b]);
  });
  for (int32_t r = 0; r < n_rp; ++r) {
    const double mf = std::ceil(static_cast<double>(n_total) / rps[r]);
    const int64_t m = std::min<int64_t>(std::max<int64_t>(static_cast<int64_t>(mf), 1), n_total);
    if (m > static_cast<int64_t>(idx.size())) return ARA_EINVAL;  // a rank sent fewer than m values
    // TVaR: Neumaier's compensated sum in FP64, in the merged order (the same bits on every host)
    double sum = 0.0, comp = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      const double v = values[idx[i]];
      const double t = sum + v;
      comp += (std::fabs(sum) >= std::fabs(v)) ? (sum - t) + v : (v - t) + sum;
      sum = t;
    }
    pml_out[r] = values[idx[m - 1]];
    tvar_out[r] = (sum + comp) / static_cast<double>(m);
  }
  return ARA_OK;
}

int ara_sort_ylt(ara_ctx* c, const double* ylt, int64_t n, int64_t* order_out) {
  int rc = bind(c);
  if (rc) return rc;
  if (!ylt || n < 1 || !order_out) return fail(c, ARA_EINVAL, "ara_sort_ylt: bad arguments");
  if (n >= (int64_t(1) << 31)) return fail(c, ARA_EINVAL, "ara_sort_ylt: at most 2^31 - 1 trials");
  const double* d_ylt = ylt;
  if (!is_device_ptr(ylt)) {
    if ((rc = reserve(c, c->in_tmp, sizeof(double) * n))) return rc;
    ARA_CUDA(c, cudaMemcpyAsync(c->in_tmp.ptr, ylt, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    d_ylt = static_cast<const double*>(c->in_tmp.ptr);
  }
  const bool out_dev = is_device_ptr(order_out);
  if ((rc = reserve(c, c->sel, ara::sort_scratch_bytes(n)))) return rc;
  int64_t* d_order = order_out;
  if (!out_dev) {
    if ((rc = reserve(c, c->out_tmp, sizeof(int64_t) * n))) return rc;
    d_order = static_cast<int64_t*>(c->out_tmp.ptr);
  }
  int launched = 0;
  ARA_CUDA(c, ara::sort_desc_device(d_ylt, n, d_order, c->sel.ptr, c->stream, &launched));
  c->launches += launched;
  if (!out_dev) {
    ARA_CUDA(c, cudaMemcpyAsync(order_out, d_order, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->stream));
    ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  } else if (!is_device_ptr(ylt)) {
    ARA_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return ARA_OK;
}

int ara_debug_uniforms(ara_ctx* c, uint64_t seed, int64_t n, const int64_t* trials, const int32_t* ks,
                       const int32_t* elts, float* out) {
  int rc = bind(c);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!trials || !ks || !elts || !out))) return fail(c, ARA_EINVAL, "ara_debug_uniforms: bad arguments");
  if (n == 0) return ARA_OK;
  DevBuf tmp;
  const size_t bytes = static_cast<size_t>(n) * (sizeof(int64_t) + 2 * sizeof(int32_t) + sizeof(float));
  if ((rc = reserve(c, tmp, bytes))) return rc;
  int64_t* d_t = static_cast<int64_t*>(tmp.ptr);
  int32_t* d_k = reinterpret_cast<int32_t*>(d_t + n);
  int32_t* d_e = d_k + n;
  float* d_o = reinterpret_cast<float*>(d_e + n);
  cudaError_t e = cudaMemcpyAsync(d_t, trials, sizeof(int64_t) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_k, ks, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_e, elts, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess)
    e = ara::launch_debug_uniforms(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), n, d_t, d_k, d_e, d_o,
                                   c->stream);
  c->launches += 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_o, sizeof(float) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  release(c, tmp);
  if (e != cudaSuccess) return fail(c, ARA_ECUDA, "ara_debug_uniforms: %s", cudaGetErrorString(e));
  return ARA_OK;
}

int ara_debug_record_losses(ara_ctx* c, int64_t n, const float* mean, const float* sigma, const float* exposure,
                            const float* z, int32_t newton_only, float* out, int32_t* iters_out) {
  int rc = bind(c);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!mean || !sigma || !exposure || !z || !out)))
    return fail(c, ARA_EINVAL, "ara_debug_record_losses: bad arguments");
  if (n == 0) return ARA_OK;
  DevBuf tmp;
  if (n >= static_cast<int64_t>(ara::kMaxEltRecords))
    return fail(c, ARA_EINVAL, "ara_debug_record_losses: at most %u records per call", ara::kMaxEltRecords - 1);
  const size_t bytes = static_cast<size_t>(n) * (sizeof(ara::Pair) + 6 * sizeof(float) + sizeof(int32_t) +
                                                 sizeof(ara::BetaShape) + sizeof(float4) * ara::kTabNodes) +
                       sizeof(float4) * ara::kTabFineStride * (ara::fine_table_cap(n) + 1) +
                       sizeof(uint32_t) * ara::build_tables_work_words(n) + 256;
  if ((rc = reserve(c, tmp, bytes))) return rc;
  ara::Pair* d_p = static_cast<ara::Pair*>(tmp.ptr);
  float* d_mu = reinterpret_cast<float*>(d_p + n);
  float* d_sg = d_mu + n;
  float* d_ex = d_sg + n;
  float* d_z = d_ex + n;
  float* d_o = d_z + n;
  int32_t* d_ev = reinterpret_cast<int32_t*>(d_o + n);
  int32_t* d_it = d_ev + n;
  ara::BetaShape* d_sh =
      reinterpret_cast<ara::BetaShape*>((reinterpret_cast<uintptr_t>(d_it + n) + 15) & ~uintptr_t(15));
  float4* d_tab = reinterpret_cast<float4*>(d_sh + n);
  float4* d_tabf = d_tab + n * ara::kTabNodes;
  uint32_t* d_work = reinterpret_cast<uint32_t*>(d_tabf + ara::kTabFineStride * (ara::fine_table_cap(n) + 1));
  uint32_t* flags = static_cast<uint32_t*>(c->flags.ptr);
  int32_t* max_ev = reinterpret_cast<int32_t*>(flags + 1);
  cudaError_t e = cudaMemcpyAsync(d_mu, mean, sizeof(float) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sg, sigma, sizeof(float) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ex, exposure, sizeof(float) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_z, z, sizeof(float) * n, cudaMemcpyDefault, c->stream);
  // the preparation kernel checks event order; give it strictly increasing ids
  std::vector<int32_t> ev(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) ev[i] = static_cast<int32_t>(i);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ev, ev.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 2 * sizeof(uint32_t), c->stream);
  if (e == cudaSuccess)
    e = ara::launch_prepare_records(d_ev, d_mu, d_sg, d_ex, n, d_p, d_sh, flags, max_ev, nullptr, c->stream);
  int launched = 2;
  if (e == cudaSuccess) e = ara::launch_build_tables(d_p, d_sh, n, d_tab, d_tabf, d_work, c->stream, &launched);
  if (e == cudaSuccess) e = ara::launch_debug_losses(d_p, d_tab, d_tabf, d_z, n, newton_only, d_o, d_it, c->stream);
  c->launches += launched;
  uint32_t hf = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_o, sizeof(float) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && iters_out)
    e = cudaMemcpyAsync(iters_out, d_it, sizeof(int32_t) * n, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  release(c, tmp);
  if (e != cudaSuccess) return fail(c, ARA_ECUDA, "ara_debug_record_losses: %s", cudaGetErrorString(e));
  if (hf & (ara::kBadValue | ara::kBadExposure))
    return fail(c, ARA_EINVAL, "ara_debug_record_losses: invalid record values");
  return ARA_OK;
}

const char* ara_last_error(const ara_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

void ara_destroy(ara_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  if (c->serve_side) cudaStreamSynchronize(c->serve_side);
  for (auto& kv : c->pool) {
    release(c, kv.second.events);
    release(c, kv.second.recs);
    release(c, kv.second.tab);
    release(c, kv.second.tabf);
    release(c, kv.second.wts);
  }
  DevBuf* bufs[] = {&c->elt_stage,  &c->elt_recs_stage, &c->elt_tab_stage, &c->elt_tabf_stage, &c->elt_work,
                    &c->elt_flags,  &c->ev_buf,         &c->tile_cnt,      &c->def_acc,        &c->yet_off,
                    &c->yet_ids,    &c->bits,           &c->word_cnt,      &c->word_pairs,     &c->rankdir,
                    &c->mask,       &c->slot_cnt,       &c->pairs,         &c->pairs_hot,     &c->pairs_w,          &c->pairs_ev,         &c->scan_tmp,       &c->flags,
                    &c->counters,   &c->ylt_tmp,        &c->diag_tmp,      &c->sel,            &c->in_tmp,
                    &c->out_tmp,    &c->serve_arena,    &c->serve_out,      &c->yix_occ,        &c->yix_grid,       &c->u_flags,
                    &c->u_scan,        &c->u_event,        &c->u_first,        &c->idx_acc,      &c->serve_sel,      &c->ev_occ,        &c->row_base,
                    &c->evr_stage,  &c->yet_flags};
  for (DevBuf* b : bufs) release(c, *b);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->ev_pool) cudaEventDestroy(e);
  for (auto& r : c->serve_rounds) cudaEventDestroy(r.ev);
  for (auto& e : c->tune_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->serve_ev_free) cudaEventDestroy(e);
  if (c->serve_join) cudaEventDestroy(c->serve_join);
  if (c->serve_side) cudaStreamDestroy(c->serve_side);
  if (c->serve_host) cudaFreeHost(c->serve_host);
  if (c->yet_ready) cudaEventDestroy(c->yet_ready);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->h_yet_flags) cudaFreeHost(c->h_yet_flags);
  cudaGetLastError();
  delete c;
}

}  // extern "C"
