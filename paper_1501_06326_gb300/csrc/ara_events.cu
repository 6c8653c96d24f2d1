// Per-event output of a layer (the Algorithm 1 loop, Section 2.2, read per
// event): from the hit-event records of each tile, in (trial, event index)
// order as k_gather wrote them, and the occurrence losses O_k that k_losses
// stored beside them, each trial's running sum S_k in event order,
// A_k = min(max(S_k - AggR, 0), AggL) and inc_k = A_k - A_{k-1}; one row per
// record (trial, k, event id, O_k, inc_k) and each trial's largest O_k.  The
// event id comes from the record's first pair (a per-pair array of the layer
// index, resident in L2), not from the YET.
//
// One warp per tile, 32 records at a time: a segmented scan over the lanes
// (segments = trials, which are contiguous) plus the carry of the trial open
// at the previous chunk's end; the loads of four chunks are issued together.  S_k, A_k and inc_k are carried in
// double-float arithmetic (48 bits; FP64 runs at a small fraction of the FP32
// rate on this GPU and bound this kernel), or in FP64 when the aggregate
// terms lie beyond the FP32 range.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "ara_df.cuh"
#include "ara_internal.h"

namespace ara {
namespace {

__device__ __forceinline__ uint32_t ev_lane() { return threadIdx.x & 31; }

// The running sums in double-float (DF) or FP64 (double): the same kernel.
__device__ __forceinline__ DF acc_of(float v, DF) { return DF{v, 0.0f}; }
__device__ __forceinline__ double acc_of(float v, double) { return static_cast<double>(v); }
__device__ __forceinline__ DF acc_add(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ DF acc_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ double acc_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double acc_val(DF a) { return df_val_fast(a); }
__device__ __forceinline__ double acc_val(double a) { return a; }
__device__ __forceinline__ DF acc_shfl_up(DF v, uint32_t d) {
  return DF{__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}
__device__ __forceinline__ double acc_shfl_up(double v, uint32_t d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ DF acc_shfl(DF v, uint32_t src) {
  return DF{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ double acc_shfl(double v, uint32_t src) { return __shfl_sync(0xffffffffu, v, src); }

// min(max(s - r, 0), l): in double-float (r and a finite l within the FP32
// range; a normalized double-float has the sign of its high part), or FP64.
struct AggTerms {
  DF r, l;
  bool l_inf;
  double rd, ld;
};
__device__ __forceinline__ DF acc_clamp(DF s, const AggTerms& t) {
  DF v = df_add(s, DF{-t.r.hi, -t.r.lo});
  if (!(v.hi > 0.0f)) v = DF{0.0f, 0.0f};
  if (!t.l_inf && (v.hi > t.l.hi || (v.hi == t.l.hi && v.lo > t.l.lo))) v = t.l;
  return v;
}
__device__ __forceinline__ double acc_clamp(double s, const AggTerms& t) { return clamp_terms_d(s, t.rd, t.ld); }

// Carry of the trial open at the end of the previous chunk: its sum, A and
// largest O.
template <typename Acc>
struct RowCarry {
  uint32_t tl;
  Acc S, A;
  float M;
};

// One chunk of 32 records (record i = base + lane): the segmented scan, A_k,
// inc_k, the row writes and the trials' largest O_k.  tl_after is the trial
// of the record after the chunk (any other key when there is none).
template <typename Acc>
__device__ __forceinline__ void rows_chunk(const EventRowsParams& q, const AggTerms& terms, int64_t ta, int64_t row0,
                                           uint32_t n, uint32_t base, uint32_t lane, uint2 rec, float O, int32_t ev,
                                           uint32_t tl_after, RowCarry<Acc>& c) {
  const Acc zero = acc_of(0.0f, Acc{});
  const uint32_t i = base + lane;
  const bool valid = i < n;
  const uint32_t x = rec.x;
  // lanes past the tile's last record get keys no trial has
  const uint32_t tl = valid ? (x >> kRecTrialShift) : 0x100u + lane;
  Acc S = acc_of(O, Acc{});
  float M = O;
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const Acc S_up = acc_shfl_up(S, d);
    const float M_up = __shfl_up_sync(0xffffffffu, M, d);
    const uint32_t tl_up = __shfl_up_sync(0xffffffffu, tl, d);
    if (lane >= d && tl_up == tl) {
      S = acc_add(S, S_up);
      M = fmaxf(M, M_up);
    }
  }
  if (tl == c.tl) {
    S = acc_add(S, c.S);
    M = fmaxf(M, c.M);
  }
  const Acc A = acc_clamp(S, terms);
  const Acc A_up = acc_shfl_up(A, 1);
  const uint32_t tl_prev = __shfl_up_sync(0xffffffffu, tl, 1);
  const Acc A_prev = (lane > 0 && tl_prev == tl) ? A_up : (tl == c.tl ? c.A : zero);
  // the trial's last record in the tile: the next record belongs to another trial
  uint32_t tl_next = __shfl_down_sync(0xffffffffu, tl, 1);
  if (lane == 31) tl_next = tl_after;
  if (valid) {
    const int64_t t = ta + tl;
    const int64_t row = row0 + i;
    if (row < q.cap) {
      if (q.row_trial) q.row_trial[row] = t;
      if (q.row_k) q.row_k[row] = static_cast<int32_t>(x & kRecKMask);
      if (q.row_event) q.row_event[row] = ev;
      if (q.row_occ) q.row_occ[row] = f32_to_f64(O);
      if (q.row_inc) q.row_inc[row] = acc_val(acc_sub(A, A_prev));
    }
    if (q.max_occ && tl_next != tl) q.max_occ[t - q.t_begin] = f32_to_f64(M);
  }
  // carry: the state of the chunk's last record
  const uint32_t last = (n - base < 32u) ? n - base - 1u : 31u;
  c.tl = __shfl_sync(0xffffffffu, tl, last);
  c.S = acc_shfl(S, last);
  c.A = acc_shfl(A, last);
  c.M = __shfl_sync(0xffffffffu, M, last);
}

// One warp per tile; kRowChunks chunks of 32 records are loaded together (the
// records, their O_k and then their event ids), so that each warp keeps
// kRowChunks times the bytes in flight that one chunk would: the kernel is
// bound by the latency of these loads, not by arithmetic.
constexpr int kRowChunks = 4;

template <typename Acc>
__global__ void __launch_bounds__(kEventRowsThreads) k_event_rows(const EventRowsParams q) {
  const uint32_t lane = ev_lane();
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  AggTerms terms;
  terms.l_inf = isinf(q.agg_l);
  terms.r = df_of(q.agg_r);
  terms.l = terms.l_inf ? DF{0.0f, 0.0f} : df_of(q.agg_l);
  terms.rd = q.agg_r;
  terms.ld = q.agg_l;
  for (int64_t tile = warp; tile < q.n_tiles; tile += n_warps) {
    const int64_t ta = q.t_begin + tile * kWarpTrials;
    const int64_t rb = __ldg(&q.off[ta]) - q.e0;
    const uint32_t n = __ldg(&q.tile_cnt[tile]);
    const int64_t row0 = __ldg(&q.row_base[tile]);
    RowCarry<Acc> c{0xFFFFFFFFu, acc_of(0.0f, Acc{}), acc_of(0.0f, Acc{}), 0.0f};
    for (uint32_t base = 0; base < n; base += 32 * kRowChunks) {
      uint2 rec[kRowChunks];
      float O[kRowChunks];
      int32_t ev[kRowChunks];
#pragma unroll
      for (int j = 0; j < kRowChunks; ++j) {
        const uint32_t i = base + 32 * j + lane;
        rec[j] = i < n ? __ldg(&q.ev_buf[rb + i]) : make_uint2(0u, 0u);
        O[j] = i < n ? __ldg(&q.occ[rb + i]) : 0.0f;
      }
      // the trial of the record after this batch (all lanes read the same word)
      const uint32_t end = base + 32 * kRowChunks;
      const uint32_t tl_end = end < n ? (__ldg(&q.ev_buf[rb + end].x) >> kRecTrialShift) : 0xFFFFFFFFu;
#pragma unroll
      for (int j = 0; j < kRowChunks; ++j)
        ev[j] = (q.row_event && base + 32 * j + lane < n) ? __ldg(&q.pair_event[rec[j].y]) : 0;
#pragma unroll
      for (int j = 0; j < kRowChunks; ++j) {
        const uint32_t b = base + 32 * j;
        if (b >= n) break;
        const uint32_t x0 = __shfl_sync(0xffffffffu, rec[j < kRowChunks - 1 ? j + 1 : j].x, 0);
        const uint32_t tl_after =
            j < kRowChunks - 1 ? (b + 32 < n ? (x0 >> kRecTrialShift) : 0xFFFFFFFFu) : tl_end;
        rows_chunk<Acc>(q, terms, ta, row0, n, b, lane, rec[j], O[j], ev[j], tl_after, c);
      }
    }
  }
}

}  // namespace

cudaError_t launch_event_rows(const EventRowsParams& q, int num_sms, cudaStream_t s) {
  if (q.n_tiles <= 0) return cudaSuccess;
  // double-float when the aggregate terms lie within the FP32 range
  const bool df = q.agg_r < 1.0e38 && (std::isinf(q.agg_l) || q.agg_l < 1.0e38);
  const void* fn = df ? reinterpret_cast<const void*>(k_event_rows<DF>) : reinterpret_cast<const void*>(k_event_rows<double>);
  // one wave of resident blocks, each warp striding over the tiles
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEventRowsThreads, 0);
  if (err != cudaSuccess) return err;
  const int64_t warps_per_block = kEventRowsThreads / 32;
  const int64_t need = (q.n_tiles + warps_per_block - 1) / warps_per_block;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(num_sms) * std::max(per_sm, 1))));
  if (df)
    k_event_rows<DF><<<grid, kEventRowsThreads, 0, s>>>(q);
  else
    k_event_rows<double><<<grid, kEventRowsThreads, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace ara
