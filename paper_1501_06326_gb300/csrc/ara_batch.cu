// Several layers in one pass (a batch): the losses kernel after k_gather has
// found, over the union of the batch's ELTs, the hit events of each tile.
//
// Each (event occurrence, ELT) loss after ELT terms (Philox uniform, inverse
// Beta through the record's quantile table, ELT terms; Section 3.3) is
// computed once and serves every layer of the batch that holds the ELT.  Per
// layer, the event's losses over the layer's ELTs are summed (Algorithm 1),
// the occurrence terms applied, and the occurrence loss is added to the
// layer's sum for the trial: a 64-bit fixed-point integer in shared memory, so
// that the sum is exact for the FP32 occurrence losses and independent of the
// order of the (atomic) additions.  The aggregate terms of each layer then give
// its year losses.
#include <cuda_runtime.h>

#include <cstdint>

#include "ara_internal.h"

namespace ara {

namespace {

constexpr int kBatchQueue = 64;  // multi-ELT events queued per warp

struct BatchWarp {
  unsigned long long acc[kBatchLayers][kWarpTrials];  // per layer and trial: sum of occurrence losses (fixed point)
  float gbuf[kBatchLayers][32];                       // per layer and lane: a multi-ELT event's loss sum
  uint2 mq[kBatchQueue];                              // queued multi-ELT events (records)
  int32_t tr_beg[kWarpTrials + 1];                    // first record of each trial of the tile
};

struct BatchShared {
  const float4* tab[kMaxIndexElts];
  const float4* tabf[kMaxIndexElts];
  uint32_t elt_id[kMaxIndexElts];
  float ret[kMaxIndexElts], lim[kMaxIndexElts], share[kMaxIndexElts];
  unsigned long long layers_of[kMaxIndexElts];
  float occ_r[kBatchLayers], occ_l[kBatchLayers];
  int32_t sexp[kBatchLayers];
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// O * 2^e as an unsigned 64-bit integer, rounded to nearest (O >= 0 finite,
// O * 2^e < 2^62): the FP32 significand shifted into place.
__device__ __forceinline__ unsigned long long fixed_of(float O, int e) {
  const uint32_t u = __float_as_uint(O);
  const int x = static_cast<int>((u >> 23) & 255u);
  if (x == 0) return 0ull;  // zero (subnormal losses are below any scale in use)
  const unsigned long long m = static_cast<unsigned long long>((u & 0x7FFFFFu) | 0x800000u);
  const int s = x - 150 + e;  // O = m 2^(x - 150)
  if (s >= 0) return m << s;
  if (s <= -64) return 0ull;
  return (m + (1ull << (-s - 1))) >> (-s);
}

// Loss after ELT terms of one pair; the Halley iteration when the record's
// table is not exact (or when the layers ask for it).
__device__ __noinline__ float pair_loss_slow(const BatchParams& p, const Pair& pr, int64_t trial, uint32_t k,
                                             unsigned long long* nc) {
  const uint32_t pos = pair_pos(pr.meta);
  const float z = philox_uniform_rk(p.rk, trial, k, static_cast<uint32_t>(p.elt_id[pos]));
  const bool fine = pair_fine(pr.meta);
  const float4* tab = fine ? p.tabf[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabFineStride
                           : p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes;
  BetaSolveStats st;
  const float x = pair_quantile_newton(pr, z, p.newton_only ? -1.0f : tab_quantile(tab, z, fine), &st);
  if (!st.converged) ++*nc;
  return p.t_share[pos] * clamp_terms_f(pr.max_l * x, p.t_ret[pos], p.t_lim[pos]);
}

__device__ __forceinline__ float pair_loss_batch(const BatchParams& p, const BatchShared& bs, uint32_t pair_index,
                                                 int64_t trial, uint32_t k, unsigned long long* nc) {
  const PairHot h = p.hot[pair_index];
  const uint32_t kind = pair_kind(h.meta);
  const uint32_t pos = pair_pos(h.meta);
  float loss = h.mu;
  if (kind == kKindZero) {
    loss = 0.0f;
  } else if (!p.primary_only && kind == kKindBeta) {
    if (p.newton_only || !pair_tab_exact(h.meta)) return pair_loss_slow(p, p.pairs[pair_index], trial, k, nc);
    const float z = philox_uniform_rk(p.rk, trial, k, bs.elt_id[pos]);
    const bool fine = pair_fine(h.meta);
    const float4* tb = (fine ? bs.tabf[pos] : bs.tab[pos]) + h.node;
    loss = h.max_l * tab_quantile(tb, z, fine);
  }
  return bs.share[pos] * clamp_terms_f(loss, bs.ret[pos], bs.lim[pos]);
}

__device__ __forceinline__ void add_occurrence(BatchWarp& ws, const BatchShared& bs, int layer, uint32_t tl,
                                               float G) {
  const float O = clamp_terms_f(G, bs.occ_r[layer], bs.occ_l[layer]);
  if (O > 0.0f) atomicAdd(&ws.acc[layer][tl], fixed_of(O, bs.sexp[layer]));
}

// The queued multi-ELT events, one per lane: the event's pair losses (each
// once) are summed per layer in the pairs' (canonical) order, then each
// layer's occurrence loss is added.
__device__ __noinline__ void batch_multi(const BatchParams& p, const BatchShared& bs, BatchWarp& ws, int nq,
                                         int64_t ta, unsigned long long* nc) {
  const uint32_t lane = lane_id();
  for (int i0 = 0; i0 < nq; i0 += 32) {
    const int i = i0 + static_cast<int>(lane);
    if (i < nq) {
      const uint2 r = ws.mq[i];
      const uint32_t cnt = ((r.x >> kRecCntShift) & kRecCntMask) + 1u;
      const uint32_t tl = r.x >> kRecTrialShift, k = r.x & kRecKMask;
      unsigned long long touched = 0ull;
      for (uint32_t j = 0; j < cnt; ++j) touched |= bs.layers_of[pair_pos(p.hot[r.y + j].meta)];
      for (unsigned long long m = touched; m; m &= m - 1ull) ws.gbuf[__ffsll(m) - 1][lane] = 0.0f;
      for (uint32_t j = 0; j < cnt; ++j) {
        const float L = pair_loss_batch(p, bs, r.y + j, ta + tl, k, nc);
        for (unsigned long long m = bs.layers_of[pair_pos(p.hot[r.y + j].meta)]; m; m &= m - 1ull)
          ws.gbuf[__ffsll(m) - 1][lane] += L;
      }
      for (unsigned long long m = touched; m; m &= m - 1ull) {
        const int l = __ffsll(m) - 1;
        add_occurrence(ws, bs, l, tl, ws.gbuf[l][lane]);
      }
    }
  }
  __syncwarp();
}

}  // namespace

// One warp per tile of kWarpTrials trials; its lanes are spread over the
// tile's trials (four per trial), so that atomic additions to one trial's
// sums come from at most four lanes at a time.
__global__ void __launch_bounds__(kBatchThreads, kBatchBlocksPerSm) k_losses_batch(const BatchParams p) {
  __shared__ BatchWarp bw[kBatchThreads / 32];
  __shared__ BatchShared bs;
  const uint32_t lane = lane_id();
  BatchWarp& ws = bw[threadIdx.x >> 5];
  for (int i = threadIdx.x; i < kMaxIndexElts; i += blockDim.x) {
    const bool in = i < p.n_elts;
    bs.tab[i] = in ? p.tab[i] : nullptr;
    bs.tabf[i] = in ? p.tabf[i] : nullptr;
    bs.elt_id[i] = in ? static_cast<uint32_t>(p.elt_id[i]) : 0u;
    bs.ret[i] = in ? p.t_ret[i] : 0.0f;
    bs.lim[i] = in ? p.t_lim[i] : 0.0f;
    bs.share[i] = in ? p.t_share[i] : 0.0f;
    bs.layers_of[i] = in ? p.layers_of[i] : 0ull;
  }
  for (int i = threadIdx.x; i < kBatchLayers; i += blockDim.x) {
    bs.occ_r[i] = p.occ_r[i];
    bs.occ_l[i] = p.occ_l[i];
    bs.sexp[i] = p.scale_exp[i];
  }
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t my_t = lane & (kWarpTrials - 1), my_sub = lane / kWarpTrials;
  constexpr uint32_t kLanesPerTrial = 32 / kWarpTrials;
  unsigned long long nc = 0ull;
  uint32_t n_pairs = 0;

  for (;;) {
    int64_t tile = 0;
    if (lane == 0) tile = static_cast<int64_t>(atomicAdd(&p.counters[0], 1ull));
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= p.n_tiles) break;
    const int64_t ta = p.t_begin + tile * kWarpTrials;
    const int64_t tb = (ta + kWarpTrials < p.t_end) ? ta + kWarpTrials : p.t_end;
    const int ntr = static_cast<int>(tb - ta);
    const uint2* recs = p.ev_buf + (__ldg(&p.off[ta]) - p.e0);
    const int32_t n = static_cast<int32_t>(__ldg(&p.tile_cnt[tile]));
    for (int i = lane; i < p.n_layers * kWarpTrials; i += 32) ws.acc[i / kWarpTrials][i % kWarpTrials] = 0ull;
    // each trial's records (sorted by trial): the first record with trial >= t
    if (lane <= static_cast<uint32_t>(kWarpTrials)) {
      int32_t lo = 0, hi = n;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if ((__ldg(&recs[mid].x) >> kRecTrialShift) < lane) lo = mid + 1; else hi = mid;
      }
      ws.tr_beg[lane] = lo;
    }
    __syncwarp();
    const int32_t beg = ws.tr_beg[my_t], end = ws.tr_beg[my_t + 1];
    int nq = 0;
    for (int32_t idx = beg + static_cast<int32_t>(my_sub);; idx += kLanesPerTrial) {
      const bool active = static_cast<int>(my_t) < ntr && idx < end;
      if (!__any_sync(0xffffffffu, active)) break;
      const uint2 r = active ? __ldcs(&recs[idx]) : make_uint2(0u, 0u);
      const uint32_t cnt = ((r.x >> kRecCntShift) & kRecCntMask) + 1u;
      const bool single = active && cnt == 1u;
      if (single) {
        const uint32_t k = r.x & kRecKMask;
        const float L = pair_loss_batch(p, bs, r.y, ta + my_t, k, &nc);
        for (unsigned long long m = bs.layers_of[pair_pos(p.hot[r.y].meta)]; m; m &= m - 1ull)
          add_occurrence(ws, bs, __ffsll(m) - 1, my_t, L);
      }
      const bool multi = active && cnt > 1u;
      n_pairs += single ? 1u : (multi ? cnt : 0u);
      const uint32_t mmask = __ballot_sync(0xffffffffu, multi);
      if (mmask) {
        if (nq + __popc(mmask) > kBatchQueue) {
          __syncwarp();
          batch_multi(p, bs, ws, nq, ta, &nc);
          nq = 0;
        }
        if (multi) ws.mq[nq + __popc(mmask & lt_mask)] = r;
        nq += __popc(mmask);
        __syncwarp();
      }
    }
    if (nq > 0) batch_multi(p, bs, ws, nq, ta, &nc);
    __syncwarp();
    // ---- year losses: aggregate terms of each layer's sum
    for (int i = lane; i < p.n_layers * ntr; i += 32) {
      const int l = i / ntr, t = i % ntr;
      const double S = __ull2double_rn(ws.acc[l][t]) * p.inv_scale[l];
      p.ylt[static_cast<int64_t>(l) * p.n_out + (ta + t - p.t_begin)] = clamp_terms_d(S, p.agg_r[l], p.agg_l[l]);
    }
    __syncwarp();
  }
  n_pairs = __reduce_add_sync(0xffffffffu, n_pairs);
  for (int d = 16; d > 0; d >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, d);
  if (lane == 0) {
    if (n_pairs) atomicAdd(&p.counters[1], static_cast<unsigned long long>(n_pairs));
    if (nc) atomicAdd(&p.counters[2], nc);
  }
}

cudaError_t launch_losses_batch(const BatchParams& p, int grid, cudaStream_t s) {
  k_losses_batch<<<grid, kBatchThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ara
