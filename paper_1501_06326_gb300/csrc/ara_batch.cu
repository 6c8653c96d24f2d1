// Several layers in one pass (a batch): the losses kernel after k_gather has
// found, over the union of the batch's ELTs, the hit events of each tile.
//
// Each (event occurrence, ELT) loss after ELT terms (Philox uniform, inverse
// Beta through the record's quantile table, ELT terms; Section 3.3) is
// computed once and serves every layer of the batch that holds the ELT.  Per
// layer, the event's losses over the layer's ELTs are summed (Algorithm 1),
// the occurrence terms applied, and the occurrence loss is added to the
// layer's sum for the trial: a 64-bit fixed-point integer (each loss rounded
// to the layer's unit, about 2^-61 of its largest possible trial sum), so that
// the sum is exact in those units and independent of the order of the
// (atomic) additions.  The aggregate terms of each layer then give its year
// losses.  Three kernels do this with different work items (a lane per record
// over a tile or over one trial, or a lane per pair over a tile); they add the
// same fixed-point numbers and give the same results.
#include <cuda_runtime.h>

#include <cstdint>

#include "ara_batch.h"

namespace ara {

namespace {

constexpr int kBatchQueue = 64;  // multi-ELT events queued per warp

struct BatchWarp {
  unsigned long long acc[kBatchLayers][32];  // per layer and lane: the lane's sum for its current trial (fixed point)
  unsigned long long (*tacc)[kWarpTrials];  // per layer and trial of the tile: the trial's sum (tiles only)
  uint32_t act[kWarpTrials];                 // per trial of the tile: the layers whose trials reach it
  uint2 mq[kBatchQueue];                     // queued multi-ELT events (records)
  float wl[32];                              // a window's pair losses
  unsigned long long wm[32];                 // a window's pairs: layers holding the pair's ELT
};

struct BatchShared {
  const float4* tab[kMaxIndexElts];
  const float4* tabf[kMaxIndexElts];
  uint32_t elt_id[kMaxIndexElts];
  float ret[kMaxIndexElts], lim[kMaxIndexElts], share[kMaxIndexElts];
  unsigned long long layers_of[kMaxIndexElts];
  float occ_r[kBatchLayers], occ_l[kBatchLayers];
  float scale[kBatchLayers];
  int64_t t_end[kBatchLayers];
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// O in a layer's fixed-point units: O * scale rounded to the nearest integer
// (ties to even).  O >= 0 is finite and scale a power of two, so the product is
// exact (or below one unit) and O * scale < 2^62 by the choice of scale.
__device__ __forceinline__ unsigned long long fixed_units(float O, float scale) {
  return __float2ull_rn(O * scale);
}

// The table argument t = Phi^-1(z) of pair `pi` (a record of kind Beta or
// BetaC) in occurrence (trial, k); false when t lies beyond the tables' range
// (only a combined normal can).
__device__ __forceinline__ bool batch_pair_normal(const BatchParams& p, uint32_t kind, uint32_t elt, uint32_t pi,
                                                  int64_t trial, uint32_t k, float* t) {
  if (kind == kKindBetaC) {
    *t = correlated_normal(p.rk, trial, k, elt, p.pw[pi]);
    return fabsf(*t) <= kTabT1f;
  }
  *t = normcdfinvf(philox_uniform_rk(p.rk, trial, k, elt));
  return true;
}

// Loss after ELT terms of pair `pi` by the Halley iteration: when the record's
// table is not exact, when a combined normal lies beyond the tables' range, or
// when the layers ask for it.
__device__ __noinline__ float pair_loss_slow(const BatchParams& p, const Pair& pr, uint32_t pi, int64_t trial,
                                             uint32_t k, unsigned long long* nc) {
  const uint32_t pos = pair_pos(pr.meta);
  const uint32_t elt = static_cast<uint32_t>(p.elt_id[pos]);
  const bool fine = pair_fine(pr.meta);
  const float4* tab = fine ? p.tabf[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabFineStride
                           : p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes;
  BetaSolveStats st;
  float x;
  if (pair_kind(pr.meta) == kKindBetaC) {
    const float t = correlated_normal(p.rk, trial, k, elt, p.pw[pi]);
    x = pair_quantile_newton_zc(pr, normcdff(t), normcdff(-t), p.newton_only ? -1.0f : tab_quantile_t(tab, t, fine),
                                &st);
  } else {
    const float z = philox_uniform_rk(p.rk, trial, k, elt);
    x = pair_quantile_newton(pr, z, p.newton_only ? -1.0f : tab_quantile(tab, z, fine), &st);
  }
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
  } else if (!p.primary_only && kind_is_beta(kind)) {
    if (p.newton_only || !pair_tab_exact(h.meta))
      return pair_loss_slow(p, p.pairs[pair_index], pair_index, trial, k, nc);
    float t;
    if (!batch_pair_normal(p, kind, bs.elt_id[pos], pair_index, trial, k, &t))
      return pair_loss_slow(p, p.pairs[pair_index], pair_index, trial, k, nc);
    const bool fine = pair_fine(h.meta);
    const float4* tb = (fine ? bs.tabf[pos] : bs.tab[pos]) + h.node;
    loss = h.max_l * tab_quantile_t(tb, t, fine);
  }
  return bs.share[pos] * clamp_terms_f(loss, bs.ret[pos], bs.lim[pos]);
}

// Adds a layer's occurrence loss (from the event's loss sum G over the
// layer's ELTs) to the lane's fixed-point sum for its current trial.
__device__ __forceinline__ void add_occurrence(BatchWarp& ws, const BatchShared& bs, int layer, uint32_t lane,
                                               float G, uint32_t* dirty) {
  const float O = clamp_terms_f(G, bs.occ_r[layer], bs.occ_l[layer]);
  if (O > 0.0f) {
    ws.acc[layer][lane] += fixed_units(O, bs.scale[layer]);
    *dirty |= 1u << layer;
  }
}

// The same, straight into the trial's sum of the tile (events whose lane is
// not tracking their trial: the multi-ELT ones).
__device__ __forceinline__ void add_occurrence_trial(BatchWarp& ws, const BatchShared& bs, int layer, uint32_t tl,
                                                     float G) {
  const float O = clamp_terms_f(G, bs.occ_r[layer], bs.occ_l[layer]);
  if (O > 0.0f) atomicAdd(&ws.tacc[layer][tl], fixed_units(O, bs.scale[layer]));
}

// Moves the lane's sums of the layers in `dirty` into the tile's sums of
// trial tl.
__device__ __forceinline__ void flush_lane(BatchWarp& ws, uint32_t lane, uint32_t tl, uint32_t dirty) {
  for (uint32_t m = dirty; m; m &= m - 1u) {
    const int l = __ffs(m) - 1;
    atomicAdd(&ws.tacc[l][tl], ws.acc[l][lane]);
    ws.acc[l][lane] = 0ull;
  }
}

// A multi-ELT event with more pairs than a window holds, by one lane: for each
// layer it touches, its pair losses over the layer's ELTs summed in the pairs'
// order (each pair's loss recomputed per layer: such events are rare).
template <bool kPerTrial>
__device__ __noinline__ void batch_long_event(const BatchParams& p, const BatchShared& bs, BatchWarp& ws, uint2 r,
                                              int64_t ta, unsigned long long* nc) {
  const uint32_t cnt = ((r.x >> kRecCntShift) & kRecCntMask) + 1u;
  const uint32_t k = r.x & kRecKMask;
  const uint32_t tl = r.x >> kRecTrialShift;
  unsigned long long touched = 0ull;
  for (uint32_t j = 0; j < cnt; ++j) touched |= bs.layers_of[pair_pos(p.hot[r.y + j].meta)];
  for (unsigned long long m = touched & ws.act[tl]; m; m &= m - 1ull) {
    const int l = __ffsll(m) - 1;
    float G = 0.0f;
    for (uint32_t j = 0; j < cnt; ++j)
      if ((bs.layers_of[pair_pos(p.hot[r.y + j].meta)] >> l) & 1ull) G += pair_loss_batch(p, bs, r.y + j, ta + tl, k, nc);
    if (kPerTrial) {
      uint32_t unused = 0u;
      add_occurrence(ws, bs, l, lane_id(), G, &unused);
    } else {
      add_occurrence_trial(ws, bs, l, tl, G);
    }
  }
}

// The queued multi-ELT events of a tile, in windows of at most 32 pairs
// (one per lane): each pair's loss once, then for each layer the window's
// events touch, each event's last lane sums the event's pair losses of that
// layer from left to right (the pairs' canonical order), applies the
// occurrence terms and adds the result to its trial's sum.  A left-to-right
// sum does not change when pairs of other layers' ELTs are present, so an
// event's per-layer losses are the same in any batch.  Only the layers that
// reach the event's trial are served; a pair of none of them is not computed.
// kPerTrial: all events are of one trial, and the end lanes add into their own
// sums (no contention); else into the trial's sum of the tile.
template <bool kPerTrial>
__device__ __noinline__ uint32_t batch_multi(const BatchParams& p, const BatchShared& bs, BatchWarp& ws, int nq,
                                             int64_t ta, unsigned long long* nc) {
  const uint32_t q = lane_id();
  const uint32_t upto = 0xffffffffu >> (31u - q);  // lanes 0..q
  uint32_t n_pairs = 0;
  for (int i0 = 0; i0 < nq;) {
    const int ie = i0 + static_cast<int>(q);
    const uint2 r = (ie < nq) ? ws.mq[ie] : make_uint2(0u, 0u);
    const uint32_t cnt = (ie < nq) ? ((r.x >> kRecCntShift) & kRecCntMask) + 1u : 0u;
    if (__shfl_sync(0xffffffffu, cnt, 0) > 32u) {  // a long event first in line: by lane 0
      if (q == 0) batch_long_event<kPerTrial>(p, bs, ws, r, ta, nc);
      n_pairs += __shfl_sync(0xffffffffu, cnt, 0);
      __syncwarp();
      ++i0;
      continue;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (q >= static_cast<uint32_t>(d)) incl += o;
    }
    const uint32_t pre = incl - cnt;
    const bool take = cnt != 0 && incl <= 32u;
    const int n_take = __popc(__ballot_sync(0xffffffffu, take));
    const uint32_t np = __shfl_sync(0xffffffffu, incl, n_take - 1);
    const uint32_t starts = __reduce_or_sync(0xffffffffu, take ? (1u << pre) : 0u);
    const uint32_t ev = static_cast<uint32_t>(__popc(starts & upto)) - 1u;  // lane q's event
    const uint32_t ex = __shfl_sync(0xffffffffu, r.x, ev);
    const uint32_t ey = __shfl_sync(0xffffffffu, r.y, ev);
    const uint32_t epre = __shfl_sync(0xffffffffu, pre, ev);
    const uint32_t ecnt = __shfl_sync(0xffffffffu, cnt, ev);
    const uint32_t etl = ex >> kRecTrialShift;
    float L = 0.0f;
    unsigned long long lm = 0ull;
    if (q < np) {
      lm = bs.layers_of[pair_pos(p.hot[ey + (q - epre)].meta)] & ws.act[etl];
      if (lm) L = pair_loss_batch(p, bs, ey + (q - epre), ta + etl, ex & kRecKMask, nc);
    }
    ws.wl[q] = L;
    ws.wm[q] = lm;
    n_pairs += np;
    const bool end = q < np && q == epre + ecnt - 1u;
    unsigned long long touched = lm;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) touched |= __shfl_xor_sync(0xffffffffu, touched, d);
    __syncwarp();
    for (unsigned long long m = touched; m; m &= m - 1ull) {
      const int l = __ffsll(m) - 1;
      if (end) {
        float G = 0.0f;
        for (uint32_t j = epre; j <= q; ++j)
          if ((ws.wm[j] >> l) & 1ull) G += ws.wl[j];
        if (kPerTrial) {
          uint32_t unused = 0u;
          add_occurrence(ws, bs, l, q, G, &unused);
        } else {
          add_occurrence_trial(ws, bs, l, etl, G);
        }
      }
    }
    __syncwarp();
    i0 += n_take;
  }
  __syncwarp();
  return n_pairs;
}

// First record in [0, n) whose trial is >= key (n if none), by the whole warp:
// each round probes 32 evenly spaced records and keeps the gap between the
// last probe below key and the first at or above it.
__device__ __forceinline__ int32_t first_record_of(const uint2* recs, int32_t n, uint32_t key, uint32_t lane) {
  int32_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (lo < hi) {
    const int32_t step = (hi - lo + 31) / 32;
    const int32_t pos = lo + static_cast<int32_t>(lane) * step;
    const bool ge = pos < hi && (__ldg(&recs[pos].x) >> kRecTrialShift) >= key;
    const uint32_t b = __ballot_sync(0xffffffffu, ge);
    if (b == 0u) {
      const int32_t probes = (hi - lo + step - 1) / step;  // positions lo + j step < hi
      lo += (probes - 1) * step + 1;
    } else {
      const int32_t f = __ffs(b) - 1;
      hi = lo + f * step;
      if (f > 0) lo += (f - 1) * step + 1;
    }
  }
  return lo;
}

}  // namespace

// One warp per item, the item's hit-event records two per lane per round
// (records two rounds ahead and single-ELT hot pairs one round ahead in
// flight); every lane keeps its own fixed-point sum per layer.
// kPerTrial = false: an item is a tile of kWarpTrials trials.  A lane's
//   records come in trial order, so its sums are for its current trial and
//   move into the tile's per-trial sums (shared-memory atomics) when the
//   trial changes.  Few records per trial fill the lanes this way.
// kPerTrial = true: an item is one trial of a tile (its records found by a
//   warp search), and the lanes' sums are added once at the item's end.
//   Many records per trial (many ELTs in the batch) keep the lanes busy, and
//   the lanes do not contend for the same sums.
// Multi-ELT events add into the per-trial sums directly.  At the item's end
// the aggregate terms of each layer give the year losses.  Both kinds add the
// same fixed-point numbers, so they give the same results.
template <bool kPerTrial>
__global__ void __launch_bounds__(kBatchThreads, kBatchBlocksPerSm) k_losses_batch(const BatchParams p) {
  __shared__ BatchWarp bw[kBatchThreads / 32];
  __shared__ BatchShared bs;
  // (one-trial items need none: a placeholder keeps the block within the shared-memory
  // carveout that leaves L1 its room)
  __shared__ unsigned long long tacc_all[kPerTrial ? 1 : kBatchThreads / 32][kPerTrial ? 1 : kBatchLayers][kWarpTrials];
  const uint32_t lane = lane_id();
  BatchWarp& ws = bw[threadIdx.x >> 5];
  if (lane == 0) ws.tacc = tacc_all[kPerTrial ? 0 : threadIdx.x >> 5];
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
    bs.scale[i] = p.scale[i];
    bs.t_end[i] = i < p.n_layers ? p.layer_t_end[i] : 0;
  }
  __syncthreads();
  static_assert(kBatchLayers <= 32, "one lane per layer");
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int nl = p.n_layers;
  unsigned long long nc = 0ull;
  uint32_t n_pairs = 0;
  for (int l = 0; l < nl; ++l) ws.acc[l][lane] = 0ull;
  const int64_t n_items = kPerTrial ? p.n_tiles * kWarpTrials : p.n_tiles;

  // items are claimed one ahead, so that the claim's latency overlaps an item's work
  unsigned long long next = 0ull;
  if (lane == 0) next = atomicAdd(&p.counters[0], 1ull);
  for (;;) {
    const int64_t item = static_cast<int64_t>(__shfl_sync(0xffffffffu, next, 0));
    if (item >= n_items) break;
    if (lane == 0) next = atomicAdd(&p.counters[0], 1ull);
    const int64_t tile = kPerTrial ? item / kWarpTrials : item;
    const uint32_t tl0 = kPerTrial ? static_cast<uint32_t>(item % kWarpTrials) : 0u;  // the item's first trial
    const int64_t ta = p.t_begin + tile * kWarpTrials;
    const int ntr = static_cast<int>((ta + kWarpTrials < p.t_end) ? kWarpTrials : p.t_end - ta);
    if (kPerTrial && static_cast<int>(tl0) >= ntr) continue;
    const int t_lo = static_cast<int>(tl0);  // the item's (first) trial in the tile
    // per trial of the item, the layers whose trials reach it (all of them unless a layer ends early)
    uint32_t any = 0u;
#pragma unroll
    for (int t = 0; t < kWarpTrials; ++t) {
      if (kPerTrial && t != t_lo) continue;
      const uint32_t a =
          __ballot_sync(0xffffffffu, t < ntr && lane < static_cast<uint32_t>(nl) && ta + t < bs.t_end[lane]);
      if (lane == 0) ws.act[t] = a;
      any |= a;
    }
    if (!kPerTrial)
      for (int i = static_cast<int>(lane); i < nl * kWarpTrials; i += 32) ws.tacc[i / kWarpTrials][i % kWarpTrials] = 0ull;
    __syncwarp();
    const uint2* recs = p.ev_buf + (__ldg(&p.off[ta]) - p.e0);
    const int32_t n_tile = any ? static_cast<int32_t>(__ldg(&p.tile_cnt[tile])) : 0;
    // the item's records [beg, n) of the tile (records are in trial order)
    const int32_t beg = kPerTrial ? first_record_of(recs, n_tile, tl0, lane) : 0;
    const int32_t n = kPerTrial ? first_record_of(recs, n_tile, tl0 + 1, lane) : n_tile;
    if (kPerTrial) {  // each lane clears its own sums (conflict-free)
      __syncwarp();
      for (int l = 0; l < nl; ++l) ws.acc[l][lane] = 0ull;
    }
    uint32_t cur = tl0, dirty = 0u;  // the lane's current trial, and the layers its sums hold
    const uint32_t act0 = ws.act[t_lo];  // the item's layers (one trial)
    int nq = 0;
    // 64 records per round, two per lane (lane and 32 + lane), so that two table
    // reads are in flight per lane; the next round's records and single-ELT hot
    // pairs are loaded one round ahead
    uint2 rn[2];
    PairHot hn[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int32_t at = beg + 32 * j + static_cast<int32_t>(lane);
      rn[j] = (at < n) ? __ldcs(recs + at) : make_uint2(0u, 0u);
      hn[j] = PairHot{0.0f, 0.0f, kKindZero << kMetaKindShift, 0u};
      if (at < n && ((rn[j].x >> kRecCntShift) & kRecCntMask) == 0u) hn[j] = p.hot[rn[j].y];
    }
    for (int32_t base = beg; base < n; base += 64) {
      uint2 r[2];
      PairHot h[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        r[j] = rn[j];
        h[j] = hn[j];
        const int32_t at = base + 64 + 32 * j + static_cast<int32_t>(lane);
        if (at < n) rn[j] = __ldcs(recs + at);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int32_t at = base + 64 + 32 * j + static_cast<int32_t>(lane);
        if (at < n && ((rn[j].x >> kRecCntShift) & kRecCntMask) == 0u) hn[j] = p.hot[rn[j].y];
      }
      // ---- single-ELT events: uniform, table position, then both table reads, then the losses
      int mode[2];  // 0: none, 1: loss known (no loss / mean), 2: table, 3: Halley
      float val[2], sfrac[2];
      const float4* node[2];
      uint32_t lmask[2];  // the layers the event serves
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const bool valid = base + 32 * j + static_cast<int32_t>(lane) < n;
        const uint32_t cnt = ((r[j].x >> kRecCntShift) & kRecCntMask) + 1u;
        const uint32_t tl = kPerTrial ? tl0 : r[j].x >> kRecTrialShift;
        mode[j] = 0;
        val[j] = 0.0f;
        sfrac[j] = 0.0f;
        node[j] = nullptr;
        lmask[j] = (valid && cnt == 1u)
                       ? static_cast<uint32_t>(bs.layers_of[pair_pos(h[j].meta)]) & (kPerTrial ? act0 : ws.act[tl])
                       : 0u;
        if (lmask[j]) {
          const uint32_t kind = pair_kind(h[j].meta);
          const uint32_t pos = pair_pos(h[j].meta);
          mode[j] = 1;
          val[j] = h[j].mu;
          if (kind == kKindZero) {
            val[j] = 0.0f;
          } else if (!p.primary_only && kind_is_beta(kind)) {
            float t = 0.0f;
            if (p.newton_only || !pair_tab_exact(h[j].meta) ||
                !batch_pair_normal(p, kind, bs.elt_id[pos], r[j].y, ta + tl, r[j].x & kRecKMask, &t)) {
              mode[j] = 3;
            } else {
              mode[j] = 2;
              const bool fine = pair_fine(h[j].meta);
              const int nseg = fine ? kTabFineNodes - 1 : kTabNodes - 1;
              float u = (t + kTabT1f) * (fine ? kTabInvH * kTabRefine : kTabInvH);
              u = fminf(fmaxf(u, 0.0f), static_cast<float>(nseg));
              int i = static_cast<int>(u);
              if (i > nseg - 1) i = nseg - 1;
              sfrac[j] = u - static_cast<float>(i);
              node[j] = (fine ? bs.tabf[pos] : bs.tab[pos]) + h[j].node + i;
            }
          }
        }
      }
      float4 n0[2];
      float2 n1[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (mode[j] == 2) {
          n0[j] = __ldg(node[j]);
          n1[j] = __ldg(reinterpret_cast<const float2*>(node[j] + 1) + 1);
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (mode[j] == 0) continue;
        const uint32_t pos = pair_pos(h[j].meta);
        const uint32_t tl = kPerTrial ? tl0 : r[j].x >> kRecTrialShift;
        float L;
        if (mode[j] == 3) {
          L = pair_loss_slow(p, p.pairs[r[j].y], r[j].y, ta + tl, r[j].x & kRecKMask, &nc);
        } else {
          float loss = val[j];
          if (mode[j] == 2)
            loss = (n0[j].x > 0.0f)
                       ? h[j].max_l * (n0[j].x * expf(tab_increment(sfrac[j], n0[j].y, n0[j].z, n0[j].w, n1[j].x,
                                                                     n1[j].y)))
                       : 0.0f;
          L = bs.share[pos] * clamp_terms_f(loss, bs.ret[pos], bs.lim[pos]);
        }
        if constexpr (!kPerTrial) {
          if (tl != cur) {  // the lane's records have moved on to a later trial
            flush_lane(ws, lane, cur, dirty);
            dirty = 0u;
            cur = tl;
          }
        }
        for (uint32_t m = lmask[j]; m; m &= m - 1u) add_occurrence(ws, bs, __ffs(m) - 1, lane, L, &dirty);
        ++n_pairs;
      }
      // ---- multi-ELT events: queued
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const bool valid = base + 32 * j + static_cast<int32_t>(lane) < n;
        const bool multi = valid && ((r[j].x >> kRecCntShift) & kRecCntMask) != 0u;
        const uint32_t mmask = __ballot_sync(0xffffffffu, multi);
        if (mmask) {
          if (nq + __popc(mmask) > kBatchQueue) {
            __syncwarp();
            const uint32_t np = batch_multi<kPerTrial>(p, bs, ws, nq, ta, &nc);
            if (lane == 0) n_pairs += np;
            nq = 0;
          }
          if (multi) ws.mq[nq + __popc(mmask & lt_mask)] = r[j];
          nq += __popc(mmask);
          __syncwarp();
        }
      }
    }
    if (nq > 0) {
      const uint32_t np = batch_multi<kPerTrial>(p, bs, ws, nq, ta, &nc);
      if (lane == 0) n_pairs += np;
    }
    // ---- the year losses of the item's trials for each layer: the aggregate terms of the trials' sums
    if constexpr (kPerTrial) {
      __syncwarp();
      for (int l = static_cast<int>(lane); l < nl; l += 32) {  // the lanes' sums, one lane per layer
        unsigned long long S = 0ull;
        for (int j = 0; j < 32; ++j) S += ws.acc[l][j];
        const double sd = __ull2double_rn(S) * p.inv_scale[l];
        if (ta + t_lo < p.layer_t_end[l]) p.ylt_l[l][ta + t_lo - p.t_begin] = clamp_terms_d(sd, p.agg_r[l], p.agg_l[l]);
      }
    } else {
      flush_lane(ws, lane, cur, dirty);
      __syncwarp();
      for (int i = static_cast<int>(lane); i < nl * ntr; i += 32) {
        const int l = i / ntr, t = i - l * ntr;
        const double sd = __ull2double_rn(ws.tacc[l][t]) * p.inv_scale[l];
        if (ta + t < p.layer_t_end[l]) p.ylt_l[l][ta + t - p.t_begin] = clamp_terms_d(sd, p.agg_r[l], p.agg_l[l]);
      }
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

namespace {

// ------------------------------------------------------------------ dense kernel
// One warp per tile, one lane per (event occurrence, ELT) pair.  The tile's
// records stream through a per-warp record ring; each record's pairs take
// consecutive slots of a pair ring.  A compute round takes the next 64 pending
// pairs (two per lane, whatever their records), computes each pair's loss
// after ELT terms once, and stores it with the layers it serves.  Records
// whose pairs are all computed are combined up to 64 at a time, with the lanes
// turned into layers: lane (s, l) holds layer l's fixed-point sum for the
// current trial in registers and takes the group's records i = s mod S (S
// record slots: 32 over the layers rounded up to a power of two) that serve
// layer l, found by bit-matrix transposes of the records' layer masks.  For
// each (single-ELT records first, then the others), it sums the record's pair
// losses over the layer's ELTs from left to right (the pairs' order), applies
// the occurrence terms and adds the result.
// When a trial's records are all combined, the slots' sums give its year
// losses.  The fill keeps a round's 64 pairs pending; a record has at most 64
// pairs, so after a combine at most 63 computed pairs and 63 pending ones are
// live, and the next record always fits the rings.
constexpr int kDenseRecs = 128;   // record ring (slots: sequence number mod kDenseRecs)
constexpr int kDensePairs = 256;  // pair ring (slots: pair sequence number mod kDensePairs)
constexpr int kDenseBlocksPerSm = 7;  // 72 registers: 28 warps per SM (measured: 6 and 8 were slower)
static_assert(kDensePairs >= 63 + 64 + 64 && kDenseRecs >= 64 + 32, "ring sizes");
static_assert(kDenseRecs <= 256, "record slots are stored in bytes");

struct DenseWarp {
  uint2 rec[kDenseRecs];        // the ring's records
  uint32_t pre[kDenseRecs];     // each record's first pair (sequence number in the tile)
  float loss[kDensePairs];      // each pair's loss after ELT terms
  uint32_t lmask[kDensePairs];  // each pair's layers: those holding its ELT that reach its trial
  uint8_t owner[kDensePairs];   // each pair's record slot
  uint32_t act[kWarpTrials];    // per trial of the tile: the layers whose trials reach it
  float g_l0[64];               // a combine group's records: first pair's loss,
  uint32_t g_pre[64];           //   first pair (sequence number),
  uint32_t g_cnt[64];           //   pair count
};

struct DenseShared {
  const float4* tab[kMaxIndexElts];
  const float4* tabf[kMaxIndexElts];
  uint32_t elt_id[kMaxIndexElts];
  float ret[kMaxIndexElts], lim[kMaxIndexElts], share[kMaxIndexElts];
  uint32_t layers_of[kMaxIndexElts];
  float4 occ[kBatchLayers];  // (occurrence retention, occurrence limit, fixed-point scale, 0)
  double agg_r[kBatchLayers], agg_l[kBatchLayers], inv_scale[kBatchLayers];
  double* ylt[kBatchLayers];
  int64_t t_end[kBatchLayers];
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= static_cast<uint32_t>(d)) v += o;
  }
  return v;
}

__device__ __forceinline__ uint2 shfl_u2(uint2 v, uint32_t src) {
  return make_uint2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Loss after ELT terms by the Halley iteration, with its non-convergence as
// the second value (0 or 1).
__device__ __noinline__ float2 dense_pair_slow(const BatchParams& p, uint32_t pi, int64_t trial, uint32_t k) {
  unsigned long long nc = 0ull;
  const float L = pair_loss_slow(p, p.pairs[pi], pi, trial, k, &nc);
  return make_float2(L, static_cast<float>(nc));
}

// The pass's per-ELT and per-layer constants in shared memory (the caller syncs).
__device__ __forceinline__ void load_dense_shared(const BatchParams& p, DenseShared& ds) {
  const int nl = p.n_layers;
  for (int i = threadIdx.x; i < kMaxIndexElts; i += blockDim.x) {
    const bool in = i < p.n_elts;
    ds.tab[i] = in ? p.tab[i] : nullptr;
    ds.tabf[i] = in ? p.tabf[i] : nullptr;
    ds.elt_id[i] = in ? static_cast<uint32_t>(p.elt_id[i]) : 0u;
    ds.ret[i] = in ? p.t_ret[i] : 0.0f;
    ds.lim[i] = in ? p.t_lim[i] : 0.0f;
    ds.share[i] = in ? p.t_share[i] : 0.0f;
    ds.layers_of[i] = in ? static_cast<uint32_t>(p.layers_of[i]) : 0u;
  }
  for (int i = threadIdx.x; i < kBatchLayers; i += blockDim.x) {
    const bool in = i < nl;
    ds.occ[i] = make_float4(p.occ_r[i], p.occ_l[i], p.scale[i], 0.0f);
    ds.agg_r[i] = p.agg_r[i];
    ds.agg_l[i] = p.agg_l[i];
    ds.inv_scale[i] = p.inv_scale[i];
    ds.ylt[i] = in ? p.ylt_l[i] : nullptr;
    ds.t_end[i] = in ? p.layer_t_end[i] : 0;
  }
}

// Lane l receives column l of the 32 x 32 bit matrix whose row i is lane i's
// x: bit i of the result is bit l of lane i's x (the off-diagonal blocks of
// halves, quarters, ... exchanged between lanes).
__device__ __forceinline__ uint32_t bit_transpose32(uint32_t x, uint32_t lane) {
  const uint32_t hi[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t j = 16u >> k;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & hi[k]) | ((y & hi[k]) >> j)) : ((x & ~hi[k]) | ((y & ~hi[k]) << j));
  }
  return x;
}

// Year losses of one trial: the slots' sums of each layer added (lanes l of
// slot 0 receive them) through the aggregate terms; the sums are cleared.
__device__ __forceinline__ void dense_finish_trial(const DenseShared& ds, unsigned long long& acc, uint32_t lane,
                                                   int nlp, int nl, int64_t trial, int64_t t_begin) {
  for (int d = nlp; d < 32; d <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane < static_cast<uint32_t>(nl) && trial < ds.t_end[lane])
    ds.ylt[lane][trial - t_begin] =
        clamp_terms_d(__ull2double_rn(acc) * ds.inv_scale[lane], ds.agg_r[lane], ds.agg_l[lane]);
  acc = 0ull;
}

}  // namespace

__global__ void __launch_bounds__(kBatchThreads, kDenseBlocksPerSm)
    k_losses_dense(const __grid_constant__ BatchParams p) {
  __shared__ DenseWarp dwarp[kBatchThreads / 32];
  __shared__ DenseShared ds;
  const uint32_t lane = lane_id();
  DenseWarp& ws = dwarp[threadIdx.x >> 5];
  const int nl = p.n_layers;
  load_dense_shared(p, ds);
  __syncthreads();
  static_assert(kBatchLayers <= 32, "one lane per layer; 32-bit layer masks");
  // the lane's layer l and record slot s; its records in a group: i = s mod S
  int nlp = 1;
  while (nlp < nl) nlp <<= 1;
  const uint32_t my_l = lane & static_cast<uint32_t>(nlp - 1);
  const uint32_t n_slots = 32u / static_cast<uint32_t>(nlp);
  uint32_t my_pattern = 0u;
  for (uint32_t i = lane / static_cast<uint32_t>(nlp); i < 32u; i += n_slots) my_pattern |= 1u << i;
  if (my_l >= static_cast<uint32_t>(nl)) my_pattern = 0u;
  unsigned long long acc = 0ull;       // the layer's sum over the slot's records of the current trial
  const uint2 zero2 = make_uint2(0u, 0u);
  unsigned long long nc = 0ull;
  uint32_t n_pairs = 0;

  unsigned long long next = 0ull;  // tiles are claimed one ahead
  if (lane == 0) next = atomicAdd(&p.counters[0], 1ull);
  for (;;) {
    const int64_t tile = static_cast<int64_t>(__shfl_sync(0xffffffffu, next, 0));
    if (tile >= p.n_tiles) break;
    if (lane == 0) next = atomicAdd(&p.counters[0], 1ull);
    const int64_t ta = p.t_begin + tile * kWarpTrials;
    const int ntr = static_cast<int>((ta + kWarpTrials < p.t_end) ? kWarpTrials : p.t_end - ta);
    uint32_t any = 0u;
#pragma unroll
    for (int t = 0; t < kWarpTrials; ++t) {
      const uint32_t a =
          __ballot_sync(0xffffffffu, t < ntr && lane < static_cast<uint32_t>(nl) && ta + t < ds.t_end[lane]);
      if (lane == 0) ws.act[t] = a;
      any |= a;
    }
    __syncwarp();
    const uint2* recs = p.ev_buf + (__ldg(&p.off[ta]) - p.e0);
    const int32_t n = any ? static_cast<int32_t>(__ldg(&p.tile_cnt[tile])) : 0;
    // lane i holds records rec_next + i (rc) and rec_next + 32 + i (rx)
    int32_t rec_next = 0;
    uint2 rc = (static_cast<int32_t>(lane) < n) ? __ldcs(recs + lane) : zero2;
    uint2 rx = (32 + static_cast<int32_t>(lane) < n) ? __ldcs(recs + 32 + lane) : zero2;
    uint32_t p_fill = 0u, p_done = 0u;  // pairs appended, pairs computed
    uint32_t r_fill = 0u, r_done = 0u;  // records appended, records combined
    int cur = 0;  // the trial whose records are being combined
    for (;;) {
      // ---- fill: whole records, 32 at a time, until a round's 64 pairs are pending
      while (p_fill - p_done < 64u && rec_next < n) {
        const bool valid = rec_next + static_cast<int32_t>(lane) < n;
        const uint32_t cnt = valid ? ((rc.x >> kRecCntShift) & kRecCntMask) + 1u : 0u;
        const uint32_t incl = warp_incl_scan(cnt, lane);
        const uint32_t live = (r_done < r_fill) ? ws.pre[r_done % kDenseRecs] : p_fill;  // oldest live pair
        const bool fits = valid && r_fill - r_done + lane < static_cast<uint32_t>(kDenseRecs) &&
                          p_fill + incl - live <= static_cast<uint32_t>(kDensePairs);
        const uint32_t n_take = __popc(__ballot_sync(0xffffffffu, fits));  // a prefix of the lanes
        if (n_take == 0u) {  // cannot happen (see above); drop the tile's remaining records rather than spin
          if (lane == 0) atomicOr(&p.counters[3], 1ull);
          rec_next = n;
          break;
        }
        if (fits) {
          const uint32_t slot = (r_fill + lane) % kDenseRecs;
          const uint32_t pre = p_fill + incl - cnt;
          ws.rec[slot] = rc;
          ws.pre[slot] = pre;
          for (uint32_t j = 0; j < cnt; ++j) ws.owner[(pre + j) % kDensePairs] = static_cast<uint8_t>(slot);
        }
        p_fill += __shfl_sync(0xffffffffu, incl, n_take - 1u);
        r_fill += n_take;
        rec_next += static_cast<int32_t>(n_take);
        // slide the window of records by n_take
        const uint32_t src = lane + n_take;
        const uint2 a = shfl_u2(rc, src & 31u), b = shfl_u2(rx, src & 31u);
        rc = src < 32u ? a : b;
        const int32_t at = rec_next + 32 + static_cast<int32_t>(lane);
        rx = src < 32u ? b : (at < n ? __ldcs(recs + at) : zero2);
        __syncwarp();
      }
      // ---- compute: up to 64 pending pairs, two per lane
      if (p_done < p_fill) {
        const uint32_t np = min(64u, p_fill - p_done);
        uint32_t q[2], pi[2], kk[2], tl[2], mk[2];
        PairHot h[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t i = 32u * j + lane;
          q[j] = (p_done + i) % kDensePairs;
          pi[j] = 0u;
          kk[j] = 0u;
          tl[j] = 0u;
          h[j] = PairHot{0.0f, 0.0f, kKindZero << kMetaKindShift, 0u};
          if (i < np) {
            const uint32_t o = ws.owner[q[j]];
            const uint2 r = ws.rec[o];
            pi[j] = r.y + (p_done + i - ws.pre[o]);
            tl[j] = r.x >> kRecTrialShift;
            kk[j] = r.x & kRecKMask;
            h[j] = p.hot[pi[j]];
          }
        }
        int mode[2];  // 0: no layer, 1: loss known (no loss / mean), 2: table, 3: Halley
        float val[2], sfrac[2];
        const float4* node[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t pos = pair_pos(h[j].meta);
          mk[j] = (32u * j + lane < np) ? ds.layers_of[pos] & ws.act[tl[j]] : 0u;
          mode[j] = 0;
          val[j] = 0.0f;
          sfrac[j] = 0.0f;
          node[j] = nullptr;
          if (mk[j]) {
            const uint32_t kind = pair_kind(h[j].meta);
            mode[j] = 1;
            val[j] = h[j].mu;
            if (kind == kKindZero) {
              val[j] = 0.0f;
            } else if (!p.primary_only && kind_is_beta(kind)) {
              float t = 0.0f;
              if (p.newton_only || !pair_tab_exact(h[j].meta) ||
                  !batch_pair_normal(p, kind, ds.elt_id[pos], pi[j], ta + tl[j], kk[j], &t)) {
                mode[j] = 3;
              } else {
                mode[j] = 2;
                const bool fine = pair_fine(h[j].meta);
                const int nseg = fine ? kTabFineNodes - 1 : kTabNodes - 1;
                float u = (t + kTabT1f) * (fine ? kTabInvH * kTabRefine : kTabInvH);
                u = fminf(fmaxf(u, 0.0f), static_cast<float>(nseg));
                int ix = static_cast<int>(u);
                if (ix > nseg - 1) ix = nseg - 1;
                sfrac[j] = u - static_cast<float>(ix);
                node[j] = (fine ? ds.tabf[pos] : ds.tab[pos]) + h[j].node + ix;
              }
            }
          }
        }
        float4 n0[2];
        float2 n1[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (mode[j] == 2) {
            n0[j] = __ldg(node[j]);
            n1[j] = __ldg(reinterpret_cast<const float2*>(node[j] + 1) + 1);
          }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float L = 0.0f;
          if (mode[j] == 3) {
            const float2 r = dense_pair_slow(p, pi[j], ta + tl[j], kk[j]);
            L = r.x;
            nc += static_cast<unsigned long long>(r.y);
          } else if (mode[j] != 0) {
            const uint32_t pos = pair_pos(h[j].meta);
            float loss = val[j];
            if (mode[j] == 2)
              loss = (n0[j].x > 0.0f)
                         ? h[j].max_l * (n0[j].x * expf(tab_increment(sfrac[j], n0[j].y, n0[j].z, n0[j].w, n1[j].x,
                                                                       n1[j].y)))
                         : 0.0f;
            L = ds.share[pos] * clamp_terms_f(loss, ds.ret[pos], ds.lim[pos]);
          }
          if (32u * j + lane < np) {
            ws.loss[q[j]] = L;
            ws.lmask[q[j]] = mk[j];
          }
          n_pairs += mk[j] != 0u;
        }
        p_done += np;
        __syncwarp();
      }
      // ---- combine: complete records of the current trial, up to 64 at a time (two per lane)
      for (;;) {
        uint32_t cnt[2], m[2], multi[2], col[2];
        int rt[2];
        bool have[2];
        uint32_t n_ok = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t gi = 32u * h + lane;  // the record's place in the group
          const uint32_t R = r_done + gi;
          have[h] = R < r_fill;
          const uint32_t slot = R % kDenseRecs;
          const uint2 r = have[h] ? ws.rec[slot] : zero2;
          const uint32_t pre = have[h] ? ws.pre[slot] : 0u;
          cnt[h] = ((r.x >> kRecCntShift) & kRecCntMask) + 1u;
          rt[h] = static_cast<int>(r.x >> kRecTrialShift);
          // a prefix of the group (records are in trial order; <= rather than == keeps the
          // loop finite whatever the order)
          const bool ok = have[h] && pre + cnt[h] <= p_done && rt[h] <= cur;
          n_ok += __popc(__ballot_sync(0xffffffffu, ok));
          multi[h] = __ballot_sync(0xffffffffu, ok && cnt[h] > 1u);
          m[h] = 0u;  // the layers the record serves
          if (ok) {
            const uint32_t q0 = pre % kDensePairs;
            m[h] = ws.lmask[q0];
            for (uint32_t j = 1; j < cnt[h]; ++j) m[h] |= ws.lmask[(pre + j) % kDensePairs];
            ws.g_l0[gi] = ws.loss[q0];
            ws.g_pre[gi] = pre;
            ws.g_cnt[gi] = cnt[h];
          }
          col[h] = __shfl_sync(0xffffffffu, bit_transpose32(m[h], lane), my_l) & my_pattern;
        }
        __syncwarp();
        // lane (s, l): the group's records of slot s that serve layer l
        unsigned long long one = static_cast<unsigned long long>(col[0] & ~multi[0]) |
                                 (static_cast<unsigned long long>(col[1] & ~multi[1]) << 32);
        unsigned long long many = static_cast<unsigned long long>(col[0] & multi[0]) |
                                  (static_cast<unsigned long long>(col[1] & multi[1]) << 32);
        const float4 oc = ds.occ[my_l];  // the layer's occurrence terms and fixed-point scale
        for (; one; one &= one - 1ull) {  // single-ELT records: the loss of their one pair
          const float O = clamp_terms_f(ws.g_l0[__ffsll(one) - 1], oc.x, oc.y);
          acc += fixed_units(O, oc.z);
        }
        for (; many; many &= many - 1ull) {  // the others: their pairs over the layer's ELTs, left to right
          const int i = __ffsll(many) - 1;
          const uint32_t c = ws.g_cnt[i], pr = ws.g_pre[i];
          float G = 0.0f;
          for (uint32_t j = 0; j < c; ++j) {
            const uint32_t qq = (pr + j) % kDensePairs;
            if ((ws.lmask[qq] >> my_l) & 1u) G += ws.loss[qq];
          }
          acc += fixed_units(clamp_terms_f(G, oc.x, oc.y), oc.z);
        }
        __syncwarp();  // the group's staging is rewritten by the next group
        r_done += n_ok;
        if (n_ok == 64u) continue;
        // the first record not combined: of a later trial (the current one is done), or not complete
        const bool hi = n_ok >= 32u;
        const bool stop_have = __shfl_sync(0xffffffffu, (hi ? have[1] : have[0]) ? 1 : 0, n_ok & 31u) != 0;
        const int stop_t = __shfl_sync(0xffffffffu, hi ? rt[1] : rt[0], n_ok & 31u);
        if (stop_have && stop_t > cur) {
          for (; cur < stop_t; ++cur) dense_finish_trial(ds, acc, lane, nlp, nl, ta + cur, p.t_begin);
          continue;
        }
        break;
      }
      if (rec_next >= n && r_done == r_fill) break;
    }
    for (; cur < ntr; ++cur) dense_finish_trial(ds, acc, lane, nlp, nl, ta + cur, p.t_begin);
    __syncwarp();
  }
  n_pairs = __reduce_add_sync(0xffffffffu, n_pairs);
  for (int d = 16; d > 0; d >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, d);
  if (lane == 0) {
    if (n_pairs) atomicAdd(&p.counters[1], static_cast<unsigned long long>(n_pairs));
    if (nc) atomicAdd(&p.counters[2], nc);
  }
}

int losses_dense_blocks_per_sm(int /*n_layers*/) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_losses_dense, kBatchThreads, 0) != cudaSuccess) return 0;
  return b;
}

cudaError_t launch_losses_batch(const BatchParams& p, int item, int grid, cudaStream_t s) {
  switch (item) {
    case kItemTile:
      k_losses_batch<false><<<grid, kBatchThreads, 0, s>>>(p);
      break;
    case kItemTrial:
      k_losses_batch<true><<<grid, kBatchThreads, 0, s>>>(p);
      break;
    case kItemDense:
      k_losses_dense<<<grid, kBatchThreads, 0, s>>>(p);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}


// ------------------------------------------------------------------ indexed kernel
// A warp per distinct event of the pass's ELT union and trial slice (claimed
// from the slice's queue, eight events at a time), over the event's
// occurrences in the slice, 32 at a time (a lane each).  The slice's bounds
// come from the index's trial grid, with a warp search only where a bound is
// inside a grid cell (a pass's ends off the grid).  Every lane of
// the warp works on the same event, so the pairs, their layers and their
// tables are the same across the warp.  For each occurrence and each layer it
// serves, the event's pair losses over the layer's ELTs are summed from left
// to right (per-lane running sums in shared memory when the event has several
// pairs), the occurrence terms applied, and the result added to the trial's
// fixed-point sum with a 64-bit atomic add: the same numbers as the other
// work items, so the same bits.  A second kernel turns the sums into year
// losses.
namespace {

constexpr int kIdxThreads = 128;
constexpr int kIdxBlocksPerSm = 7;
constexpr int kIdxClaim = 8;  // events a warp claims at a time

struct IdxWarp {
  float gacc[kBatchLayers][32];      // per layer and lane: the running sum of an occurrence's pair losses
  uint32_t pmask[kMaxIndexElts];     // the event's pairs: layers holding their ELTs
  uint4 meta[2 * kIdxClaim];         // the claimed events: [j] (first pair, pair end, range of the slice's first
                                     // occurrence), [kIdxClaim + j] (range of its end, -, -)
  int64_t span[2];                   // the trials of the claim's slice
};

// First entry in [lo, hi) of the event's occurrences whose trial is >= key
// (hi if none), by the whole warp: each round probes 32 evenly spaced entries.
__device__ __forceinline__ uint32_t first_occ_at(const unsigned long long* occ, uint32_t lo, uint32_t hi,
                                                 int64_t key, uint32_t lane) {
  while (lo < hi) {
    const uint32_t step = (hi - lo + 31u) / 32u;
    const uint32_t pos = lo + lane * step;
    const bool ge = pos < hi && static_cast<int64_t>(__ldg(occ + pos) >> 32) >= key;
    const uint32_t b = __ballot_sync(0xffffffffu, ge);
    if (b == 0u) {
      const uint32_t probes = (hi - lo + step - 1u) / step;
      lo += (probes - 1u) * step + 1u;
    } else {
      const uint32_t f = static_cast<uint32_t>(__ffs(b) - 1);
      hi = lo + f * step;
      if (f > 0u) lo += (f - 1u) * step + 1u;
    }
  }
  return lo;
}

// Loss after ELT terms of pair pi in occurrence (trial, k): as the other work items compute it.
__device__ __forceinline__ float indexed_pair_loss(const BatchParams& p, const DenseShared& ds, uint32_t pi,
                                                   int64_t trial, uint32_t k, unsigned long long* nc) {
  const PairHot h = p.hot[pi];
  const uint32_t kind = pair_kind(h.meta);
  const uint32_t pos = pair_pos(h.meta);
  float loss = h.mu;
  if (kind == kKindZero) {
    loss = 0.0f;
  } else if (!p.primary_only && kind_is_beta(kind)) {
    float t;
    if (p.newton_only || !pair_tab_exact(h.meta) || !batch_pair_normal(p, kind, ds.elt_id[pos], pi, trial, k, &t))
      return pair_loss_slow(p, p.pairs[pi], pi, trial, k, nc);
    const bool fine = pair_fine(h.meta);
    loss = h.max_l * tab_quantile_t((fine ? ds.tabf[pos] : ds.tab[pos]) + h.node, t, fine);
  }
  return ds.share[pos] * clamp_terms_f(loss, ds.ret[pos], ds.lim[pos]);
}

__global__ void k_event_flags(const int32_t* __restrict__ pev, int64_t n, uint32_t* flags) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    flags[i] = (i == 0 || pev[i] != pev[i - 1]) ? 1u : 0u;
}

__global__ void k_union_events(const int32_t* __restrict__ pev, const uint32_t* __restrict__ flags,
                               const uint32_t* __restrict__ scan, int64_t n, int32_t* u_event, uint32_t* u_first) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    if (flags[i]) {
      u_event[scan[i]] = pev[i];
      u_first[scan[i]] = static_cast<uint32_t>(i);
    }
    if (i == n - 1) u_first[scan[n]] = static_cast<uint32_t>(n);
  }
}

}  // namespace

__global__ void __launch_bounds__(kIdxThreads, kIdxBlocksPerSm)
    k_losses_indexed(const __grid_constant__ IndexedParams q) {
  const BatchParams& p = q.b;
  __shared__ IdxWarp iwarp[kIdxThreads / 32];
  __shared__ DenseShared ds;
  const uint32_t lane = lane_id();
  IdxWarp& ws = iwarp[threadIdx.x >> 5];
  load_dense_shared(p, ds);
  __syncthreads();
  const int nl = p.n_layers;
  const int64_t t0 = p.t_begin, stride = p.t_end - p.t_begin;
  int64_t t_full = p.t_end;  // below it every layer reaches the trial
  for (int l = 0; l < nl; ++l) t_full = min(t_full, ds.t_end[l]);
  const uint32_t all = nl >= 32 ? 0xffffffffu : (1u << nl) - 1u;
  for (int l = 0; l < nl; ++l) ws.gacc[l][lane] = 0.0f;
  const uint32_t n_u = *q.n_u;
  unsigned long long nc = 0ull;
  uint32_t n_pairs = 0;
  // the occurrences (read once) are the first to leave L2, so that the trials' sums, which the atomic
  // adds revisit, stay (batched-16: 5.98 against 6.07 ms a pass)
  uint64_t occ_pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(occ_pol));

  // the queue's groups: kIdxClaim events over one trial slice, every event of a slice before the next
  // slice, so that the sums being added to stay within a slice's trials; a warp moves to the next slice
  // when the slice's queue runs out. For the group's event j, lane j loads its pairs and the grid range
  // that holds the slice's first occurrence, lane kIdxClaim + j the range that holds the slice's end (a
  // bound on the grid is its own range); the next group's loads are issued before this group's events run.
  const int slice_shift = q.slice_shift, grid_shift = q.grid_shift;
  const int64_t k0 = t0 >> slice_shift;
  const uint32_t per_slice = (n_u + kIdxClaim - 1) / kIdxClaim;
  const uint32_t n_slices = static_cast<uint32_t>(indexed_slices(t0, p.t_end, slice_shift));
  uint4 meta = make_uint4(0u, 0u, 0u, 0u);
  uint32_t sl = 0u;  // the slice of the group claimed last
  auto slice_lo = [&](uint32_t j) { return max(t0, (k0 + j) << slice_shift); };
  auto slice_hi = [&](uint32_t j) { return min(p.t_end, (k0 + j + 1) << slice_shift); };
  auto claim = [&]() {
    uint32_t g = 0u;
    for (; sl < n_slices; ++sl) {
      if (lane == 0) g = atomicAdd(q.slice_queue + sl, 1u);
      g = __shfl_sync(0xffffffffu, g, 0);
      if (g < per_slice) break;
    }
    const uint32_t j = lane & static_cast<uint32_t>(kIdxClaim - 1), u = g * kIdxClaim + j;
    if (sl < n_slices && lane < static_cast<uint32_t>(2 * kIdxClaim) && u < n_u) {
      const uint32_t* row = q.ev_grid + static_cast<int64_t>(q.u_event[u]) * (q.grid_cells + 1);
      const bool end = lane >= static_cast<uint32_t>(kIdxClaim);
      const int64_t b = end ? slice_hi(sl) : slice_lo(sl);
      const int64_t cell = b >= q.yet_trials ? q.grid_cells : b >> grid_shift;
      const bool on_grid = b >= q.yet_trials || (b & ((int64_t{1} << grid_shift) - 1)) == 0;
      const uint32_t x = row[cell], y = on_grid ? x : row[cell + 1];
      meta = end ? make_uint4(x, y, 0u, 0u) : make_uint4(q.u_first[u], q.u_first[u + 1], x, y);
    }
    return g;
  };
  uint32_t grp = claim();
  while (sl < n_slices) {
    if (lane < static_cast<uint32_t>(2 * kIdxClaim)) ws.meta[lane] = meta;
    if (lane == 0) {
      ws.span[0] = slice_lo(sl);
      ws.span[1] = slice_hi(sl);
    }
    __syncwarp();
    const int n_here = static_cast<int>(min(static_cast<uint32_t>(kIdxClaim), n_u - grp * kIdxClaim));
    grp = claim();
    for (int g = 0; g < n_here; ++g) {
      const uint4 m4 = ws.meta[g], h4 = ws.meta[kIdxClaim + g];
      const uint32_t ps = m4.x, cnt = m4.y - m4.x;
      // the slice's occurrences: a search only where a bound is inside a grid cell
      const uint32_t lo = first_occ_at(q.occ, m4.z, m4.w, ws.span[0], lane);
      const uint32_t hi = first_occ_at(q.occ, max(lo, h4.x), h4.y, ws.span[1], lane);
      if (lo >= hi) continue;
      for (uint32_t j = lane; j < cnt; j += 32) ws.pmask[j] = ds.layers_of[pair_pos(p.hot[ps + j].meta)];
      __syncwarp();
      for (uint32_t r = lo; r < hi; r += 32) {
        const uint32_t i = r + lane;
        const bool valid = i < hi;
        unsigned long long o = 0ull;
        if (valid)
          asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;"
                       : "=l"(o)
                       : "l"(q.occ + i), "l"(occ_pol));
        const int64_t trial = static_cast<int64_t>(o >> 32);
        const uint32_t k = static_cast<uint32_t>(o);
        uint32_t act = 0u;  // the layers whose trials reach this one
        if (valid) {
          act = all;
          if (trial >= t_full) {
            act = 0u;
            for (int l = 0; l < nl; ++l)
              if (trial < ds.t_end[l]) act |= 1u << l;
          }
        }
        unsigned long long* acc = q.acc + (trial - t0);
        if (cnt == 1u) {
          const uint32_t m = ws.pmask[0] & act;
          if (m) {
            const float L = indexed_pair_loss(p, ds, ps, trial, k, &nc);
            ++n_pairs;
            for (uint32_t mm = m; mm; mm &= mm - 1u) {
              const int l = __ffs(mm) - 1;
              const float4 c = ds.occ[l];
              const float O = clamp_terms_f(L, c.x, c.y);
              if (O > 0.0f) atomicAdd(acc + static_cast<int64_t>(l) * stride, fixed_units(O, c.z));
            }
          }
        } else {
          // the pairs in order: each layer's running sum is the left-to-right sum of its pairs' losses
          uint32_t touched = 0u;
          for (uint32_t j = 0; j < cnt; ++j) {
            const uint32_t m = ws.pmask[j] & act;
            if (m) {
              const float L = indexed_pair_loss(p, ds, ps + j, trial, k, &nc);
              ++n_pairs;
              touched |= m;
              for (uint32_t mm = m; mm; mm &= mm - 1u) ws.gacc[__ffs(mm) - 1][lane] += L;
            }
          }
          for (uint32_t mm = touched; mm; mm &= mm - 1u) {
            const int l = __ffs(mm) - 1;
            const float G = ws.gacc[l][lane];
            ws.gacc[l][lane] = 0.0f;
            const float4 c = ds.occ[l];
            const float O = clamp_terms_f(G, c.x, c.y);
            if (O > 0.0f) atomicAdd(acc + static_cast<int64_t>(l) * stride, fixed_units(O, c.z));
          }
        }
      }
      __syncwarp();  // pmask is rewritten for the next event
    }
    __syncwarp();  // meta is rewritten for the next claim
  }
  n_pairs = __reduce_add_sync(0xffffffffu, n_pairs);
  for (int d = 16; d > 0; d >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, d);
  if (lane == 0) {
    if (n_pairs) atomicAdd(&p.counters[1], static_cast<unsigned long long>(n_pairs));
    if (nc) atomicAdd(&p.counters[2], nc);
  }
}

namespace {

__global__ void k_indexed_years(const __grid_constant__ IndexedParams q) {
  const BatchParams& p = q.b;
  const int64_t stride = p.t_end - p.t_begin;
  const int64_t n = stride * p.n_layers;
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += step) {
    const int l = static_cast<int>(i / stride);
    const int64_t tt = i - static_cast<int64_t>(l) * stride;
    if (p.t_begin + tt < p.layer_t_end[l])
      p.ylt_l[l][tt] = clamp_terms_d(__ull2double_rn(q.acc[i]) * p.inv_scale[l], p.agg_r[l], p.agg_l[l]);
  }
}

int grid_for_n(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

cudaError_t launch_union_events(const int32_t* pev, int64_t n_recs, uint32_t* flags, uint32_t* scan,
                                uint32_t* scan_tmp, int32_t* u_event, uint32_t* u_first, cudaStream_t s,
                                int* n_launch) {
  if (n_recs == 0) return cudaMemsetAsync(scan, 0, sizeof(uint32_t), s);
  k_event_flags<<<grid_for_n(n_recs, 256), 256, 0, s>>>(pev, n_recs, flags);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if ((err = scan_exclusive_u32(flags, scan, n_recs, scan_tmp, s, n_launch)) != cudaSuccess) return err;
  k_union_events<<<grid_for_n(n_recs, 256), 256, 0, s>>>(pev, flags, scan, n_recs, u_event, u_first);
  if (n_launch) *n_launch += 2;
  return cudaGetLastError();
}

int losses_indexed_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_losses_indexed, kIdxThreads, 0) != cudaSuccess) return 0;
  return b;
}

cudaError_t launch_losses_indexed(const IndexedParams& q, int grid, cudaStream_t s) {
  k_losses_indexed<<<grid, kIdxThreads, 0, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_indexed_years(const IndexedParams& q, cudaStream_t s) {
  k_indexed_years<<<grid_for_n((q.b.t_end - q.b.t_begin) * q.b.n_layers, 256), 256, 0, s>>>(q);
  return cudaGetLastError();
}


}  // namespace ara
