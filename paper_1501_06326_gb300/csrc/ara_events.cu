// Per-event output of a layer (the Algorithm 1 loop, Section 2.2, read per
// event): from the hit-event records of each tile, in (trial, event index)
// order as k_gather wrote them, and the occurrence losses O_k that k_losses
// stored beside them, each trial's running sum S_k in FP64 and event order,
// A_k = min(max(S_k - AggR, 0), AggL) and inc_k = A_k - A_{k-1}; one row per
// record (trial, k, event id, O_k, inc_k) and each trial's largest O_k.
//
// One warp per tile, 32 records at a time: a segmented scan over the lanes
// (segments = trials, which are contiguous) plus the carry of the trial open
// at the previous chunk's end.

#include <cuda_runtime.h>

#include <cstdint>

#include "ara_internal.h"

namespace ara {
namespace {

__device__ __forceinline__ uint32_t ev_lane() { return threadIdx.x & 31; }

__global__ void __launch_bounds__(kEventRowsThreads) k_event_rows(const EventRowsParams q) {
  const uint32_t lane = ev_lane();
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t tile = warp; tile < q.n_tiles; tile += n_warps) {
    const int64_t ta = q.t_begin + tile * kWarpTrials;
    const int64_t rb = __ldg(&q.off[ta]) - q.e0;
    const uint32_t n = __ldg(&q.tile_cnt[tile]);
    const int64_t row0 = __ldg(&q.row_base[tile]);
    // the trial open at the end of the previous chunk: its sum, A and largest O
    uint32_t c_tl = 0xFFFFFFFFu;
    double c_S = 0.0, c_A = 0.0;
    float c_M = 0.0f;
    for (uint32_t base = 0; base < n; base += 32) {
      const uint32_t i = base + lane;
      const bool valid = i < n;
      const uint32_t x = valid ? __ldg(&q.ev_buf[rb + i].x) : 0u;
      const float O = valid ? __ldg(&q.occ[rb + i]) : 0.0f;
      // lanes past the tile's last record get keys no trial has
      const uint32_t tl = valid ? (x >> kRecTrialShift) : 0x100u + lane;
      double S = static_cast<double>(O);
      float M = O;
#pragma unroll
      for (uint32_t d = 1; d < 32; d <<= 1) {
        const double S_up = __shfl_up_sync(0xffffffffu, S, d);
        const float M_up = __shfl_up_sync(0xffffffffu, M, d);
        const uint32_t tl_up = __shfl_up_sync(0xffffffffu, tl, d);
        if (lane >= d && tl_up == tl) {
          S += S_up;
          M = fmaxf(M, M_up);
        }
      }
      if (tl == c_tl) {
        S += c_S;
        M = fmaxf(M, c_M);
      }
      const double A = clamp_terms_d(S, q.agg_r, q.agg_l);
      const double A_up = __shfl_up_sync(0xffffffffu, A, 1);
      const uint32_t tl_prev = __shfl_up_sync(0xffffffffu, tl, 1);
      const double A_prev = (lane > 0 && tl_prev == tl) ? A_up : (tl == c_tl ? c_A : 0.0);
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
          if (q.row_inc) q.row_inc[row] = A - A_prev;
        }
        if (q.max_occ && tl_next != tl) q.max_occ[t - q.t_begin] = static_cast<double>(M);
      }
      // carry: the state of the chunk's last record
      const uint32_t last = (n - base < 32u) ? n - base - 1u : 31u;
      c_tl = __shfl_sync(0xffffffffu, tl, last);
      c_S = __shfl_sync(0xffffffffu, S, last);
      c_A = __shfl_sync(0xffffffffu, A, last);
      c_M = __shfl_sync(0xffffffffu, M, last);
    }
  }
}

}  // namespace

cudaError_t launch_event_rows(const EventRowsParams& q, int grid, cudaStream_t s) {
  if (q.n_tiles <= 0) return cudaSuccess;
  k_event_rows<<<grid, kEventRowsThreads, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace ara
