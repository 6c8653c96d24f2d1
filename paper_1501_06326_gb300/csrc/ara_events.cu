// Per-event output of a layer (the Algorithm 1 loop, Section 2.2, read per
// event): from the hit-event records of each tile, in (trial, event index)
// order as k_gather wrote them, and the occurrence losses O_k that k_losses
// stored beside them, each trial's running sum S_k in event order,
// A_k = min(max(S_k - AggR, 0), AggL) and inc_k = A_k - A_{k-1}; one row per
// record (trial, k, event id, O_k, inc_k) and each trial's largest O_k.
//
// One warp per tile, 32 records at a time: a segmented scan over the lanes
// (segments = trials, which are contiguous) plus the carry of the trial open
// at the previous chunk's end.  S_k, A_k and inc_k are carried in
// double-float arithmetic (48 bits; FP64 runs at a small fraction of the FP32
// rate on this GPU and bound this kernel), or in FP64 when the aggregate
// terms lie beyond the FP32 range.

#include <cuda_runtime.h>

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
__device__ __forceinline__ double acc_val(DF a) { return df_val(a); }
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
  const Acc zero = acc_of(0.0f, Acc{});
  for (int64_t tile = warp; tile < q.n_tiles; tile += n_warps) {
    const int64_t ta = q.t_begin + tile * kWarpTrials;
    const int64_t rb = __ldg(&q.off[ta]) - q.e0;
    const uint32_t n = __ldg(&q.tile_cnt[tile]);
    const int64_t row0 = __ldg(&q.row_base[tile]);
    // the trial open at the end of the previous chunk: its sum, A and largest O
    uint32_t c_tl = 0xFFFFFFFFu;
    Acc c_S = zero, c_A = zero;
    float c_M = 0.0f;
    for (uint32_t base = 0; base < n; base += 32) {
      const uint32_t i = base + lane;
      const bool valid = i < n;
      const uint32_t x = valid ? __ldg(&q.ev_buf[rb + i].x) : 0u;
      const float O = valid ? __ldg(&q.occ[rb + i]) : 0.0f;
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
      if (tl == c_tl) {
        S = acc_add(S, c_S);
        M = fmaxf(M, c_M);
      }
      const Acc A = acc_clamp(S, terms);
      const Acc A_up = acc_shfl_up(A, 1);
      const uint32_t tl_prev = __shfl_up_sync(0xffffffffu, tl, 1);
      const Acc A_prev = (lane > 0 && tl_prev == tl) ? A_up : (tl == c_tl ? c_A : zero);
      // the trial's last record in the tile: the next record belongs to another trial
      uint32_t tl_next = __shfl_down_sync(0xffffffffu, tl, 1);
      if (lane == 31) tl_next = (base + 32 < n) ? (__ldg(&q.ev_buf[rb + base + 32].x) >> kRecTrialShift) : 0xFFFFFFFFu;
      if (valid) {
        const int64_t t = ta + tl;
        const int64_t row = row0 + i;
        if (row < q.cap) {
          const uint32_t k = x & kRecKMask;
          if (q.row_trial) q.row_trial[row] = t;
          if (q.row_k) q.row_k[row] = static_cast<int32_t>(k);
          if (q.row_event) q.row_event[row] = __ldg(&q.ids[__ldg(&q.off[t]) + k]);
          if (q.row_occ) q.row_occ[row] = static_cast<double>(O);
          if (q.row_inc) q.row_inc[row] = acc_val(acc_sub(A, A_prev));
        }
        if (q.max_occ && tl_next != tl) q.max_occ[t - q.t_begin] = static_cast<double>(M);
      }
      // carry: the state of the chunk's last record
      const uint32_t last = (n - base < 32u) ? n - base - 1u : 31u;
      c_tl = __shfl_sync(0xffffffffu, tl, last);
      c_S = acc_shfl(S, last);
      c_A = acc_shfl(A, last);
      c_M = __shfl_sync(0xffffffffu, M, last);
    }
  }
}

}  // namespace

cudaError_t launch_event_rows(const EventRowsParams& q, int grid, cudaStream_t s) {
  if (q.n_tiles <= 0) return cudaSuccess;
  // double-float when the aggregate terms lie within the FP32 range
  const bool df = q.agg_r < 1.0e38 && (std::isinf(q.agg_l) || q.agg_l < 1.0e38);
  if (df)
    k_event_rows<DF><<<grid, kEventRowsThreads, 0, s>>>(q);
  else
    k_event_rows<double><<<grid, kEventRowsThreads, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace ara
