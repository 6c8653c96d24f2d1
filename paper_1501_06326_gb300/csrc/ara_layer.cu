// The layer kernels of the ARA engine (Algorithm 1 with the secondary
// uncertainty of Section 3.3, per trial): k_gather streams the YET and finds
// the events of the layer's ELTs, k_losses draws the uniforms, inverts the
// Beta CDFs through the quantile tables, applies the ELT, occurrence and
// aggregate terms and writes the year losses.
#include <cuda_runtime.h>

#include <cstdint>

#include "ara_internal.h"

namespace ara {

namespace {

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

}  // namespace

// =============================================================== layer kernels
//
// k_gather: one persistent CTA of 32 warps per SM.  The CTA folds the layer's
// catalogue bitmap into a shared-memory membership filter once (as many words
// as shared memory holds; word w of the catalogue lands on w mod filt_words);
// then each warp independently takes tiles of kWarpTrials consecutive trials
// and streams the tile's YET ids, 256 per step (two int4 per lane, not L1-allocated,
// two more steps in flight).  Each id is tested against the filter; each
// positive is resolved against the rank directory (8 bytes: the word's bits
// and its pair base) and, if it is a member, becomes an event record written
// in YET order to the tile's region of the event buffer.
//
// k_losses: each warp takes tiles and reads their records one per lane.  An
// event with one (event, ELT) pair is finished by its lane: Philox uniform,
// inverse Beta through the record's quantile table, ELT and occurrence terms,
// and a double-float add into the lane's sum for the event's trial.  Events
// with several pairs are queued and processed in windows of 32 pairs with a
// segmented sum.  Events with a pair whose record's table is not exact are
// deferred and resolved, 32 at a time, by the FP32 Halley iteration.  At the
// end of a tile a reduce-scatter over the lanes gives the trials' sums, and
// the aggregate terms turn each into the trial's year loss.

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }


struct GatherWarp {
  int32_t off[16];      // trial offsets relative to the tile's first event; INT32_MAX past the tile's end
  uint32_t pos_id[256];  // filter positives of one step: event id
  uint8_t pos_q[256];    //   and position in the step
};

}  // namespace

size_t gather_smem_bytes(int filt_words) {
  return sizeof(uint32_t) * static_cast<size_t>(filt_words) + sizeof(GatherWarp) * (kGatherThreads / 32) + 16;
}

// k_gather's shared memory stays within the 196 KB carveout (less the 1 KB
// the driver reserves per block): the L1 that the rest of the SM's 256 KB
// leaves (60 KB) holds the id stream's loads in flight, and a larger carveout
// (L1 28 KB) was measured to slow the stream by a quarter, more than a larger
// filter saves.
constexpr int kGatherSmemBudget = 196 * 1024 - 1024;

int gather_filter_words(int64_t n_words, int max_smem) {
  const int64_t budget = max_smem < kGatherSmemBudget ? max_smem : kGatherSmemBudget;
  const int64_t room = (budget - static_cast<int64_t>(gather_smem_bytes(0))) / 4;
  const int64_t fw_max = room & ~int64_t(31);
  if (fw_max < 32) return 0;
  if (n_words <= 2 * fw_max) return static_cast<int>(n_words <= fw_max ? (n_words > 0 ? n_words : 1) : fw_max);
  int64_t fw = 32;
  while (fw * 2 <= fw_max) fw *= 2;
  return static_cast<int>(fw);
}

namespace {

// State of one warp's pass over one tile.
struct GatherTile {
  const int4* ids4;  // the tile's ids from the 16-byte boundary at or below its first event
  int32_t lead;      // ids before the tile's first event in the first int4
  int32_t nev;       // events of the tile
  int32_t span;      // nev + lead
  uint2* out;        // the tile's region of the event buffer
  uint32_t nout;     // records written
};

// One int4 of YET ids, read once: not allocated in L1, whose capacity holds
// the loads in flight (measured 1% faster than evict-first loads).
__device__ __forceinline__ int4 ld_ids(const int4* a) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(a));
  return v;
}

// Loads step c0 (256 ids: int4 lane and int4 32 + lane of the step).
__device__ __forceinline__ void gather_load(const GatherTile& g, int32_t c0, uint32_t lane, int4& v0, int4& v1) {
  v0 = make_int4(0, 0, 0, 0);
  v1 = make_int4(0, 0, 0, 0);
  const int32_t i0 = c0 + 4 * static_cast<int32_t>(lane);
  if (i0 < g.span) v0 = ld_ids(g.ids4 + (i0 >> 2));
  if (i0 + 128 < g.span) v1 = ld_ids(g.ids4 + ((i0 + 128) >> 2));
}

// Positives of one step whose rank-directory words are in flight: entries
// lane and 32 + lane of the step's staging list.
struct GatherPending {
  uint2 q0, q1;    // (event id, position in the step)
  uint2 rd0, rd1;  // rank-directory words {bits, base}
  int32_t c0;      // the step's first position
  uint32_t npos;   // entries (at most 64; 0 = nothing pending)
};

// Resolves one staged positive per lane (warp-wide call): if the event is a
// member, its record is appended to the tile's records in lane order.
__device__ __forceinline__ void gather_resolve(const GatherParams& p, const GatherWarp& ws, GatherTile& g, int32_t c0,
                                               uint2 q, uint2 rd, bool valid, uint32_t lane) {
  uint32_t key = 0, ps = 0;
  const uint32_t bit = 1u << (q.x & 31);
  const bool hit = valid && (rd.x & bit) != 0u;
  if (hit) {
    const uint32_t below = __popc(rd.x & (bit - 1u));
    uint32_t cnt = 1;
    if (rd.y & 0x80000000u) {
      const uint32_t sl = (rd.y & 0x7FFFFFFFu) + below;
      ps = __ldg(&p.slot_start[sl]);
      cnt = __ldg(&p.slot_start[sl + 1]) - ps;
    } else {
      ps = rd.y + below;
    }
    // trial: the last t with off[t] <= rel (off is padded with INT32_MAX)
    const int32_t rel = c0 + static_cast<int32_t>(q.y) - g.lead;
    int t = (ws.off[4] <= rel) ? 4 : 0;
    t += (ws.off[t + 2] <= rel) ? 2 : 0;
    t += (ws.off[t + 1] <= rel) ? 1 : 0;
    key = ((cnt - 1u) << kRecCntShift) | (static_cast<uint32_t>(t) << kRecTrialShift) |
          static_cast<uint32_t>(rel - ws.off[t]);
  }
  const uint32_t hm = __ballot_sync(0xffffffffu, hit);
  if (hit) g.out[g.nout + __popc(hm & ((1u << lane) - 1u))] = make_uint2(key, ps);
  g.nout += __popc(hm);
}

// Finishes the pending positives of the previous step.
__device__ __forceinline__ void gather_complete(const GatherParams& p, const GatherWarp& ws, GatherTile& g,
                                                const GatherPending& pd, uint32_t lane) {
  if (pd.npos == 0) return;
  gather_resolve(p, ws, g, pd.c0, pd.q0, pd.rd0, lane < pd.npos, lane);
  if (pd.npos > 32) gather_resolve(p, ws, g, pd.c0, pd.q1, pd.rd1, 32 + lane < pd.npos, lane);
}

// One step of 256 YET positions: filter, compact the positives in YET order,
// finish the previous step's positives, then either put this step's in flight
// (up to 64) or resolve them at once.
// kSub: the catalogue has at most twice filt_words words, and word w folds
// onto min(w, w - filt_words) (unsigned); otherwise filt_words is a power of
// two and w folds onto w & (filt_words - 1).  fsel is filt_words or the mask.
template <bool kSub>
__device__ __forceinline__ void gather_step(const GatherParams& p, const uint32_t* __restrict__ filt, uint32_t fsel,
                                            GatherWarp& ws, GatherTile& g, GatherPending& pd, int32_t c0,
                                            uint32_t lane, int4 v0, int4 v1) {
  const uint32_t e[8] = {static_cast<uint32_t>(v0.x), static_cast<uint32_t>(v0.y), static_cast<uint32_t>(v0.z),
                         static_cast<uint32_t>(v0.w), static_cast<uint32_t>(v1.x), static_cast<uint32_t>(v1.y),
                         static_cast<uint32_t>(v1.z), static_cast<uint32_t>(v1.w)};
  // 1. filter (the shift count of a funnel shift is taken mod 32)
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t wi = e[j] >> 5;
    const uint32_t w = filt[kSub ? min(wi, wi - fsel) : (wi & fsel)];
    m |= (__funnelshift_r(w, w, e[j]) & 1u) << j;
  }
  const uint32_t q0 = 4u * lane;  // step positions of the lane's ids: q0 + j, q0 + 128 + j
  if (c0 == 0 || c0 + 256 > g.span) {
    uint32_t vm = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int32_t rel = c0 + static_cast<int32_t>(q0 + (j & 3) + (j >> 2) * 128) - g.lead;
      vm |= (static_cast<uint32_t>(rel) < static_cast<uint32_t>(g.nev) ? 1u : 0u) << j;
    }
    m &= vm;
  }
  // 2. compaction: one scan over both halves (16-bit fields)
  const uint32_t cl = __popc(m & 15u), ch = __popc(m >> 4);
  const uint32_t incl = warp_inclusive_scan(cl | (ch << 16));
  const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
  const uint32_t nlo = tot & 0xFFFFu;
  const uint32_t npos = nlo + (tot >> 16);
  // 3. the previous step's positives (their loads had this step's filter to land)
  gather_complete(p, ws, g, pd, lane);
  pd.npos = 0;
  if (npos == 0) return;
  // 4. this step's positives: staged, then in flight, or resolved at once when there are many
  if (m) {
    uint32_t at = (incl & 0xFFFFu) - cl;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (m & (1u << j)) {
        ws.pos_id[at] = e[j];
        ws.pos_q[at] = static_cast<uint8_t>(q0 + j);
        ++at;
      }
    at = nlo + (incl >> 16) - ch;
#pragma unroll
    for (int j = 4; j < 8; ++j)
      if (m & (1u << j)) {
        ws.pos_id[at] = e[j];
        ws.pos_q[at] = static_cast<uint8_t>(q0 + 124 + j);
        ++at;
      }
  }
  __syncwarp();
  if (npos <= 64) {
    pd.npos = npos;
    pd.c0 = c0;
    pd.q0 = lane < npos ? make_uint2(ws.pos_id[lane], ws.pos_q[lane]) : make_uint2(0u, 0u);
    pd.q1 = 32 + lane < npos ? make_uint2(ws.pos_id[32 + lane], ws.pos_q[32 + lane]) : make_uint2(0u, 0u);
    pd.rd0 = lane < npos ? __ldg(&p.rankdir[pd.q0.x >> 5]) : make_uint2(0u, 0u);
    pd.rd1 = 32 + lane < npos ? __ldg(&p.rankdir[pd.q1.x >> 5]) : make_uint2(0u, 0u);
  } else {
    for (uint32_t r0 = 0; r0 < npos; r0 += 32) {
      const bool valid = r0 + lane < npos;
      const uint2 q = valid ? make_uint2(ws.pos_id[r0 + lane], ws.pos_q[r0 + lane]) : make_uint2(0u, 0u);
      const uint2 rd = valid ? __ldg(&p.rankdir[q.x >> 5]) : make_uint2(0u, 0u);
      gather_resolve(p, ws, g, c0, q, rd, valid, lane);
    }
  }
  __syncwarp();
}

}  // namespace

template <bool kSub>
__global__ void __launch_bounds__(kGatherThreads, 1) k_gather(const GatherParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GatherWarp* gw = reinterpret_cast<GatherWarp*>(smem_raw);
  uint32_t* filt = reinterpret_cast<uint32_t*>(gw + (kGatherThreads / 32));
  const uint32_t lane = lane_id();
  GatherWarp& ws = gw[threadIdx.x >> 5];
  const uint32_t fsel = kSub ? static_cast<uint32_t>(p.filt_words) : static_cast<uint32_t>(p.filt_words) - 1u;

  for (int w = threadIdx.x; w < p.filt_words; w += blockDim.x) {
    uint32_t v = 0;
    for (int64_t k = w; k < p.n_words; k += p.filt_words) v |= p.rankdir[k].x;
    filt[w] = v;
  }
  __syncthreads();

  for (;;) {
    int64_t tile = 0;
    if (lane == 0) tile = static_cast<int64_t>(atomicAdd(p.queue, 1ull));
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= p.n_tiles) break;
    const int64_t ta = p.t_begin + tile * kWarpTrials;
    const int64_t tb = (ta + kWarpTrials < p.t_end) ? ta + kWarpTrials : p.t_end;
    const int ntr = static_cast<int>(tb - ta);
    const int64_t ea = __ldg(&p.off[ta]);
    if (lane < 16)
      ws.off[lane] = (lane <= static_cast<uint32_t>(ntr)) ? static_cast<int32_t>(__ldg(&p.off[ta + lane]) - ea)
                                                          : INT32_MAX;
    __syncwarp();
    GatherTile g;
    g.nev = ws.off[ntr];
    g.ids4 = reinterpret_cast<const int4*>(p.ids + (ea & ~int64_t(3)));
    g.lead = static_cast<int32_t>(ea & 3);
    g.span = g.nev + g.lead;
    g.out = p.ev_buf + (ea - p.e0);
    g.nout = 0;
    // three steps of ids in registers, two of them in flight while one is filtered;
    // unrolled by three so that no register of a load in flight is ever moved
    int4 a0, a1, b0, b1, c0v, c1v;
    GatherPending pd;
    pd.npos = 0;
    gather_load(g, 0, lane, a0, a1);
    gather_load(g, 256, lane, b0, b1);
    for (int32_t c0 = 0; c0 < g.span; c0 += 768) {
      gather_load(g, c0 + 512, lane, c0v, c1v);
      gather_step<kSub>(p, filt, fsel, ws, g, pd, c0, lane, a0, a1);
      if (c0 + 256 >= g.span) break;
      gather_load(g, c0 + 768, lane, a0, a1);
      gather_step<kSub>(p, filt, fsel, ws, g, pd, c0 + 256, lane, b0, b1);
      if (c0 + 512 >= g.span) break;
      gather_load(g, c0 + 1024, lane, b0, b1);
      gather_step<kSub>(p, filt, fsel, ws, g, pd, c0 + 512, lane, c0v, c1v);
    }
    gather_complete(p, ws, g, pd, lane);
    if (lane == 0) p.tile_cnt[tile] = g.nout;
    __syncwarp();
  }
}

cudaError_t launch_gather(const GatherParams& p, int grid, size_t smem, cudaStream_t s) {
  const bool sub = p.n_words <= 2 * static_cast<int64_t>(p.filt_words);
  const void* fn = sub ? reinterpret_cast<const void*>(k_gather<true>) : reinterpret_cast<const void*>(k_gather<false>);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  if (sub)
    k_gather<true><<<grid, kGatherThreads, smem, s>>>(p);
  else
    k_gather<false><<<grid, kGatherThreads, smem, s>>>(p);
  return cudaGetLastError();
}

namespace {

constexpr int kQueue = 64;         // multi-ELT events queued per warp
constexpr uint32_t kDefCur = 1u;   // deferred event of the open tile
constexpr uint32_t kDefLast = 2u;  // last deferred event of its trial

struct LossWarp {
  float2 acc[kWarpTrials][32];  // per trial and lane: double-float sum of the lane's occurrence losses
  uint2 mq[kQueue];             // queued multi-ELT events (event records)
  uint32_t mqi[kQueue];         //   their places in the tile's records (per-event output)
  uint32_t d_key[32];           // deferred events: record
  uint32_t d_ps[32];            //   first pair
  int64_t d_o[32];              //   trial (output index)
  int64_t d_idx[32];            //   event buffer entry of the record (per-event output)
  uint32_t d_fl[32];            //   kDefCur | kDefLast
  float d_O[32];                //   occurrence loss, once resolved
  double Sd[kWarpTrials];       // sums of the deferred occurrence losses resolved while the tile is open
  unsigned long long hits[kWarpTrials];
  unsigned long long hash[kWarpTrials];
  unsigned long long n_nc, n_slow;  // non-converged Halley pairs, Halley events
};

// (hi, lo) + (hi2, lo2) in double-float arithmetic (TwoSum, then renormalise).
__device__ __forceinline__ void df_add(float& hi, float& lo, float hi2, float lo2) {
  const float s = hi + hi2;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (hi2 - bb);
  const float e = err + lo + lo2;
  hi = s + e;
  lo = e - (hi - s);
}

// The table argument t = Phi^-1(z) of pair `pi` of an ELT record of kind
// `kind` (Beta or BetaC) in occurrence (trial, k); false when t lies beyond
// the tables' range (only a combined normal can).
__device__ __forceinline__ bool pair_normal(const LossParams& p, uint32_t kind, uint32_t elt, uint32_t pi,
                                            int64_t trial, uint32_t k, float* t) {
  if (kind == kKindBetaC) {
    *t = correlated_normal(p.rk, trial, k, elt, p.pw[pi]);
    return fabsf(*t) <= kTabT1f;
  }
  *t = normcdfinvf(philox_uniform_rk(p.rk, trial, k, elt));
  return true;
}

// Loss after ELT terms of pair `pi`, for the table path; returns false when
// the pair needs the Halley iteration.
__device__ __forceinline__ bool pair_fast(const LossParams& p, const Pair& pr, uint32_t pi, int64_t trial, uint32_t k,
                                          float* out) {
  const uint32_t kind = pair_kind(pr.meta);
  const uint32_t pos = pair_pos(pr.meta);
  float loss = pr.mu;
  if (kind == kKindZero) {
    loss = 0.0f;
  } else if (!p.primary_only && kind_is_beta(kind)) {
    if (p.newton_only || !pair_tab_exact(pr.meta)) return false;
    float t;
    if (!pair_normal(p, kind, static_cast<uint32_t>(p.elt_id[pos]), pi, trial, k, &t)) return false;
    const bool fine = pair_fine(pr.meta);
    const float4* tb = fine ? p.tabf[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabFineStride
                            : p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes;
    loss = pr.max_l * tab_quantile_t(tb, t, fine);
  }
  *out = p.t_share[pos] * clamp_terms_f(loss, p.t_ret[pos], p.t_lim[pos]);
  return true;
}

__device__ __noinline__ float pair_slow(const LossParams& p, const Pair& pr, uint32_t pi, int64_t trial, uint32_t k,
                                        unsigned long long* nc) {
  const uint32_t pos = pair_pos(pr.meta);
  float v;
  if (pair_fast(p, pr, pi, trial, k, &v)) return v;
  const uint32_t elt = static_cast<uint32_t>(p.elt_id[pos]);
  const bool fine = pair_fine(pr.meta);
  const float4* tab = fine ? p.tabf[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabFineStride
                           : p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes;
  BetaSolveStats st;
  float x;
  if (pair_kind(pr.meta) == kKindBetaC) {
    // z = Phi(v) and 1 - z = Phi(-v), each directly
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

// Resolve the warp's deferred events (all lanes call it): lane i computes the
// occurrence loss of entry i, then lane 0 adds them in list order.  A trial's
// deferred losses form their own FP64 sum, in event order, so where the list
// is flushed does not change any result: entries of the open tile go to its
// shared sums, older ones to def_acc, and the last one of a trial finishes
// its year loss.  kEmit: also stores each entry's occurrence loss beside its
// record (per-event output).
template <bool kEmit>
__device__ __noinline__ void resolve_deferred(const LossParams& p, LossWarp& ws, int nd) {
  const uint32_t lane = lane_id();
  float O = 0.0f;
  unsigned long long nc_l = 0;
  unsigned long long* nc = &nc_l;
  if (lane < static_cast<uint32_t>(nd)) {
    const uint32_t key = ws.d_key[lane];
    const uint32_t k = key & kRecKMask;
    const uint32_t cnt = ((key >> kRecCntShift) & kRecCntMask) + 1u;
    const int64_t t = p.t_begin + ws.d_o[lane];
    float G = 0.0f;
    for (uint32_t j = 0; j < cnt; ++j) G += pair_slow(p, p.pairs[ws.d_ps[lane] + j], ws.d_ps[lane] + j, t, k, nc);
    O = clamp_terms_f(G, p.occ_r, p.occ_l);
    if constexpr (kEmit) p.occ[ws.d_idx[lane]] = O;
  }
  const uint32_t nc_w = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(nc_l));
  ws.d_O[lane] = O;
  __syncwarp();
  if (lane == 0) {
    ws.n_nc += nc_w;
    ws.n_slow += static_cast<unsigned long long>(nd);
    double acc = 0.0;
    bool open = false;  // acc holds def_acc of the current run's trial
    for (int i = 0; i < nd; ++i) {
      const float Oi = ws.d_O[i];
      const uint32_t fl = ws.d_fl[i];
      const int64_t o = ws.d_o[i];
      if (fl & kDefCur) {
        ws.Sd[ws.d_key[i] >> kRecTrialShift] += static_cast<double>(Oi);
        continue;
      }
      if (!open) {
        acc = p.def_acc[o];
        open = true;
      }
      acc += static_cast<double>(Oi);
      if (fl & kDefLast) {
        p.ylt[o] = clamp_terms_d(p.ylt[o] + acc, p.agg_r, p.agg_l);
        open = false;
      } else if (i + 1 == nd || ws.d_o[i + 1] != o) {
        p.def_acc[o] = acc;
        open = false;
      }
    }
  }
  __syncwarp();
}

}  // namespace

namespace {

// Appends this lane's event to the deferred list when `defer` (warp-wide call;
// events are listed in lane order), resolving the list first when it is full.
// Returns the new length of the list.  `idx` (kEmit) is the record's event
// buffer entry.
template <bool kEmit>
__device__ __forceinline__ int defer_events(const LossParams& p, LossWarp& ws, int nd, bool defer, uint2 r,
                                            int64_t o, int64_t idx) {
  const uint32_t dmask = __ballot_sync(0xffffffffu, defer);
  if (dmask == 0) return nd;
  if (nd + __popc(dmask) > 32) {
    resolve_deferred<kEmit>(p, ws, nd);
    nd = 0;
  }
  if (defer) {
    const int at = nd + __popc(dmask & ((1u << lane_id()) - 1u));
    ws.d_key[at] = r.x;
    ws.d_ps[at] = r.y;
    ws.d_o[at] = o;
    ws.d_fl[at] = kDefCur;
    if constexpr (kEmit) ws.d_idx[at] = idx;
  }
  __syncwarp();
  return nd + __popc(dmask);
}

// Adds an occurrence loss to the lane's double-float sum of trial tl.
__device__ __forceinline__ void acc_add(LossWarp& ws, uint32_t tl, float O) {
  float2 a = ws.acc[tl][lane_id()];
  df_add(a.x, a.y, O, 0.0f);
  ws.acc[tl][lane_id()] = a;
}

// The layer's ELTs by position, in shared memory (one array per field, so that
// lanes reading different ELTs hit different banks).
struct EltShared {
  const float4* tab[32];
  const float4* tabf[32];
  uint32_t elt_id[32];
  float ret[32], lim[32], share[32];
};

// Loss after ELT terms of one pair from its hot record, for the table path;
// returns false when the pair needs the Halley iteration.
__device__ __forceinline__ bool pair_fast_hot(const LossParams& p, const EltShared& es, const PairHot& h, uint32_t pi,
                                              int64_t trial, uint32_t k, float* out) {
  const uint32_t kind = pair_kind(h.meta);
  const uint32_t pos = pair_pos(h.meta);
  float loss = h.mu;
  if (kind == kKindZero) {
    loss = 0.0f;
  } else if (!p.primary_only && kind_is_beta(kind)) {
    if (p.newton_only || !pair_tab_exact(h.meta)) return false;
    float t;
    if (!pair_normal(p, kind, es.elt_id[pos], pi, trial, k, &t)) return false;
    const bool fine = pair_fine(h.meta);
    const float4* tb = (fine ? es.tabf[pos] : es.tab[pos]) + h.node;
    loss = h.max_l * tab_quantile_t(tb, t, fine);
  }
  *out = es.share[pos] * clamp_terms_f(loss, es.ret[pos], es.lim[pos]);
  return true;
}

// The queued multi-ELT events, in windows of at most 32 pairs (one per lane):
// losses of the pairs, a segmented sum per event (pairs in layer order), the
// occurrence terms at each event's last lane.  Returns (deferred list length,
// pairs processed).  kEmit: the occurrence losses also go beside the records
// (the tile's records start at event buffer entry rb).
template <bool kEmit>
__device__ __forceinline__ int2 process_multi(const LossParams& p, const EltShared& es, LossWarp& ws, int nd, int nq,
                                              int64_t ta, bool diag, int64_t rb) {
  const uint32_t q = lane_id();
  const uint32_t upto = 0xffffffffu >> (31u - q);  // lanes 0..q
  int n_pairs = 0;
#pragma unroll 1
  for (int i0 = 0; i0 < nq;) {
    const int ie = i0 + static_cast<int>(q);
    const uint2 r = (ie < nq) ? ws.mq[ie] : make_uint2(0u, 0u);
    const uint32_t cnt = (ie < nq) ? ((r.x >> kRecCntShift) & kRecCntMask) + 1u : 0u;
    const uint32_t incl = warp_inclusive_scan(cnt);
    const uint32_t pre = incl - cnt;
    const bool take = cnt != 0 && incl <= 32u;
    const int n_take = __popc(__ballot_sync(0xffffffffu, take));
    const uint32_t np = __shfl_sync(0xffffffffu, incl, n_take - 1);
    const uint32_t starts = __reduce_or_sync(0xffffffffu, take ? (1u << pre) : 0u);
    // lane q's event: the last start at or below q
    const uint32_t ev = static_cast<uint32_t>(__popc(starts & upto)) - 1u;
    const uint32_t ex = __shfl_sync(0xffffffffu, r.x, ev);
    const uint32_t ey = __shfl_sync(0xffffffffu, r.y, ev);
    const uint32_t epre = __shfl_sync(0xffffffffu, pre, ev);
    const uint32_t ecnt = __shfl_sync(0xffffffffu, cnt, ev);
    const uint32_t etl = ex >> kRecTrialShift, ek = ex & kRecKMask;
    float L = 0.0f;
    bool slow = false;
    if (q < np) {
      const uint32_t pi = ey + (q - epre);
      const PairHot h = p.hot[pi];
      slow = !pair_fast_hot(p, es, h, pi, ta + etl, ek, &L);
      if (diag) {
        const uint32_t elt = es.elt_id[pair_pos(h.meta)];
        atomicAdd(&ws.hits[etl], 1ull);
        atomicAdd(&ws.hash[etl], static_cast<unsigned long long>(fmix64((static_cast<uint64_t>(ek) << 32) | elt)));
      }
    }
    n_pairs += static_cast<int>(np);
    // segmented inclusive sum within each event's lanes
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
      const float o = __shfl_up_sync(0xffffffffu, L, d);
      if (q >= epre + d) L += o;
    }
    const uint32_t smask = __ballot_sync(0xffffffffu, slow);
    const bool end = q < np && q == epre + ecnt - 1u;
    const bool seg_slow = ((smask >> epre) & (0xffffffffu >> (31u - (q - epre)))) != 0u;
    if (end && !seg_slow) {
      const float O = clamp_terms_f(L, p.occ_r, p.occ_l);
      acc_add(ws, etl, O);
      if constexpr (kEmit) p.occ[rb + ws.mqi[i0 + ev]] = O;
    }
    int64_t idx = 0;  // lane q < np holds a pair of queue entry i0 + ev; only event ends read it
    if constexpr (kEmit)
      if (end) idx = rb + ws.mqi[i0 + ev];
    nd = defer_events<kEmit>(p, ws, nd, end && seg_slow, make_uint2(ex, ey), ta + etl - p.t_begin, idx);
    i0 += n_take;
  }
  __syncwarp();
  return make_int2(nd, n_pairs);
}

// One stage of the reduce-scatter of kWarpTrials double-float values over the
// warp: lanes with bit (4 HALF) clear keep values 0..HALF-1, the others
// HALF..2 HALF-1, each adding its partner's copy of the values it keeps.
template <int HALF>
__device__ __forceinline__ void reduce_scatter_stage(float (&h)[kWarpTrials], float (&l)[kWarpTrials], uint32_t lane) {
  constexpr int d = 4 * HALF;
  const bool up = (lane & d) != 0;
#pragma unroll
  for (int j = 0; j < HALF; ++j) {
    const float sh = up ? h[j] : h[j + HALF], sl = up ? l[j] : l[j + HALF];
    float kh = up ? h[j + HALF] : h[j], kl = up ? l[j + HALF] : l[j];
    df_add(kh, kl, __shfl_xor_sync(0xffffffffu, sh, d), __shfl_xor_sync(0xffffffffu, sl, d));
    h[j] = kh;
    l[j] = kl;
  }
}

}  // namespace

// k_losses: each warp takes tiles and reads their event records one per lane
// (the records two rounds ahead and the hot pair records one round ahead are
// in flight).  An event with one (event, ELT) pair -- nearly all of them -- is
// finished by its lane: Philox uniform, inverse Beta through the record's
// quantile table, ELT terms, occurrence terms, and a double-float add into the
// lane's sum for the event's trial.  Events with several pairs are queued and
// processed in windows of 32 pairs with a segmented sum.  At the end of the
// tile one reduce-scatter over the lanes turns the per-lane sums into the
// trials' sums.  kEmit (per-event output) also stores each hit event's
// occurrence loss beside its record.
template <bool kEmit>
__global__ void __launch_bounds__(kLossThreads, kLossBlocksPerSm) k_losses(const LossParams p) {
  __shared__ LossWarp lw[kLossThreads / 32];
  __shared__ EltShared es;
  const uint32_t lane = lane_id();
  LossWarp& ws = lw[threadIdx.x >> 5];
  if (threadIdx.x < 32) {
    const int i = static_cast<int>(threadIdx.x);
    const bool in = i < p.n_elts;
    es.tab[i] = in ? p.tab[i] : nullptr;
    es.tabf[i] = in ? p.tabf[i] : nullptr;
    es.elt_id[i] = in ? static_cast<uint32_t>(p.elt_id[i]) : 0u;
    es.ret[i] = in ? p.t_ret[i] : 0.0f;
    es.lim[i] = in ? p.t_lim[i] : 0.0f;
    es.share[i] = in ? p.t_share[i] : 0.0f;
  }
  __syncthreads();
  const bool diag = (p.diag_hits != nullptr) || (p.diag_hash != nullptr);
  const uint32_t lt_mask = (1u << lane) - 1u;
  int nd = 0;  // deferred events listed; the list outlives tiles so that resolving keeps the lanes busy
  uint32_t n_pairs = 0;
  if (lane == 0) {
    ws.n_nc = 0ull;
    ws.n_slow = 0ull;
  }

  for (;;) {
    int64_t tile = 0;
    if (lane == 0) tile = static_cast<int64_t>(atomicAdd(&p.counters[0], 1ull));
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= p.n_tiles) break;
    const int64_t ta = p.t_begin + tile * kWarpTrials;
    const int64_t tb = (ta + kWarpTrials < p.t_end) ? ta + kWarpTrials : p.t_end;
    const int ntr = static_cast<int>(tb - ta);
    const int64_t rb = __ldg(&p.off[ta]) - p.e0;  // the tile's first event buffer entry
    const uint2* recs = p.ev_buf + rb;
    const uint32_t n = __ldg(&p.tile_cnt[tile]);
#pragma unroll
    for (int t = 0; t < kWarpTrials; ++t) ws.acc[t][lane] = make_float2(0.0f, 0.0f);
    if (lane < static_cast<uint32_t>(ntr)) {
      ws.Sd[lane] = 0.0;
      ws.hits[lane] = 0ull;
      ws.hash[lane] = 0ull;
    }
    __syncwarp();
    int nq = 0;
    // pipeline: r1 = records of the next round, r0/h0 = this round's record and hot pair
    uint2 r0 = (lane < n) ? __ldcs(recs + lane) : make_uint2(0u, 0u);
    uint2 r1 = (32 + lane < n) ? __ldcs(recs + 32 + lane) : make_uint2(0u, 0u);
    PairHot h0{0.0f, 0.0f, kKindZero << kMetaKindShift, 0u};
    if (lane < n && ((r0.x >> kRecCntShift) & kRecCntMask) == 0u) h0 = p.hot[r0.y];
    for (uint32_t base = 0;;) {
#pragma unroll 1
      for (; base < n && nq <= kQueue - 32; base += 32) {
        const uint2 r = r0;
        const PairHot h = h0;
        const bool valid = base + lane < n;
        r0 = r1;
        if (base + 64 + lane < n) r1 = __ldcs(recs + base + 64 + lane);
        if (base + 32 + lane < n && ((r0.x >> kRecCntShift) & kRecCntMask) == 0u) h0 = p.hot[r0.y];
        const uint32_t cnt = ((r.x >> kRecCntShift) & kRecCntMask) + 1u;
        const uint32_t tl = r.x >> kRecTrialShift, k = r.x & kRecKMask;
        const bool single = valid && cnt == 1u;
        bool slow = false;
        if (single) {
          float L;
          slow = !pair_fast_hot(p, es, h, r.y, ta + tl, k, &L);
          if (!slow) {
            const float O = clamp_terms_f(L, p.occ_r, p.occ_l);
            acc_add(ws, tl, O);
            if constexpr (kEmit) p.occ[rb + base + lane] = O;
          }
          if (diag) {
            const uint32_t elt = es.elt_id[pair_pos(h.meta)];
            atomicAdd(&ws.hits[tl], 1ull);
            atomicAdd(&ws.hash[tl], static_cast<unsigned long long>(fmix64((static_cast<uint64_t>(k) << 32) | elt)));
          }
        }
        n_pairs += __popc(__ballot_sync(0xffffffffu, single));
        nd = defer_events<kEmit>(p, ws, nd, slow, r, ta + tl - p.t_begin, rb + base + lane);
        const uint32_t mmask = __ballot_sync(0xffffffffu, valid && cnt > 1u);
        if (mmask) {
          if (valid && cnt > 1u) {
            ws.mq[nq + __popc(mmask & lt_mask)] = r;
            if constexpr (kEmit) ws.mqi[nq + __popc(mmask & lt_mask)] = base + lane;
          }
          nq += __popc(mmask);
        }
      }
      __syncwarp();
      if (nq > 0) {
        const int2 rv = process_multi<kEmit>(p, es, ws, nd, nq, ta, diag, rb);
        nd = rv.x;
        n_pairs += static_cast<uint32_t>(rv.y);
        nq = 0;
      }
      if (base >= n) break;
    }
    __syncwarp();
    // ---- trials' sums: reduce-scatter of the per-lane double-float sums; lane
    // (b4 b3 b2 b1 b0) ends up holding trial 4 b4 + 2 b3 + b2
    float h8[kWarpTrials], l8[kWarpTrials];
#pragma unroll
    for (int t = 0; t < kWarpTrials; ++t) {
      const float2 a = ws.acc[t][lane];
      h8[t] = a.x;
      l8[t] = a.y;
    }
    reduce_scatter_stage<4>(h8, l8, lane);
    reduce_scatter_stage<2>(h8, l8, lane);
    reduce_scatter_stage<1>(h8, l8, lane);
#pragma unroll
    for (int d = 2; d > 0; d >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h8[0], d);
      const float l2 = __shfl_xor_sync(0xffffffffu, l8[0], d);
      df_add(h8[0], l8[0], h2, l2);
    }
    const uint32_t src = ((lane >> 2) & 1u) << 4 | ((lane >> 1) & 1u) << 3 | (lane & 1u) << 2;
    const float Sh = __shfl_sync(0xffffffffu, h8[0], src);
    const float Sl = __shfl_sync(0xffffffffu, l8[0], src);
    const double S = static_cast<double>(Sh) + static_cast<double>(Sl);
    // ---- tile end: a trial whose deferred events are all resolved is final; one
    // with events still listed keeps its table-path sum in ylt and its partial
    // deferred sum in def_acc until the last of them is resolved
    uint32_t pend = 0;
    {
      const bool cur = lane < static_cast<uint32_t>(nd) && (ws.d_fl[lane] & kDefCur);
      const uint32_t tl = cur ? (ws.d_key[lane] >> kRecTrialShift) : 0xFFu + lane;
      const uint32_t same = __match_any_sync(0xffffffffu, tl);
      if (cur) {
        pend = 1u << tl;
        ws.d_fl[lane] = (lane == 31u - __clz(same)) ? kDefLast : 0u;
      }
    }
    pend = __reduce_or_sync(0xffffffffu, pend);
    __syncwarp();
    if (lane < static_cast<uint32_t>(ntr)) {
      const int64_t o = ta + lane - p.t_begin;
      if ((pend >> lane) & 1u) {
        p.ylt[o] = S;
        p.def_acc[o] = ws.Sd[lane];
      } else {
        p.ylt[o] = clamp_terms_d(S + ws.Sd[lane], p.agg_r, p.agg_l);
      }
      if (p.diag_hits) p.diag_hits[o] = static_cast<int64_t>(ws.hits[lane]);
      if (p.diag_hash) p.diag_hash[o] = ws.hash[lane];
    }
    __syncwarp();
  }
  if (nd > 0) resolve_deferred<kEmit>(p, ws, nd);
  if (lane == 0) {
    const unsigned long long n_nc = ws.n_nc, n_slow = ws.n_slow;
    if (n_pairs) atomicAdd(&p.counters[1], static_cast<unsigned long long>(n_pairs));
    if (n_nc) atomicAdd(&p.counters[2], n_nc);
    if (n_slow) atomicAdd(&p.counters[3], n_slow);
  }
}

cudaError_t launch_losses(const LossParams& p, int grid, cudaStream_t s) {
  if (p.occ)
    k_losses<true><<<grid, kLossThreads, 0, s>>>(p);
  else
    k_losses<false><<<grid, kLossThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ara
