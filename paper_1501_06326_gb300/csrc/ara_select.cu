// PML / TVaR (Section 2.3) and the YLT trial order on the device.
//
// Year losses are mapped to order-preserving 64-bit keys (sign-flipped IEEE
// bits).  PML(RP) is the m-th largest year loss, m = ceil(n / RP): an MSB-first
// radix select with 8-bit digits narrows the key prefix.  With a scratch of
// select_scratch_bytes(n), two histogram passes fix 16 bits, a third pass
// compacts the keys of that 16-bit bucket (in a fixed order) and one block
// finishes the remaining 48 bits on them; with only the select state (the
// allocation-free entry point) all eight passes run over the YLT.  TVaR(RP)
// is the mean of the m largest: the sum of the values whose key exceeds the
// m-th key plus the tied remainder times the m-th value, in FP64 with a fixed
// reduction order (deterministic).  The full trial order
// (largest first, ties by index) is an LSD radix sort of the complemented keys
// with stable per-tile scatter (warp match + per-warp digit offsets).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <utility>

#include "../../include/ara.h"
#include "ara_batch.h"

namespace ara {

namespace {

constexpr int kSelBlocks = 152;  // fixed grid: deterministic reduction order
constexpr int kSelThreads = 1024;
constexpr int kSelUnroll = 4;  // loads in flight per thread
constexpr int kSelGroup = 4;     // return periods selected together (one pass over the YLT serves all)
constexpr int kSelBatchMax = 32;  // jobs of one batched select

__device__ __forceinline__ unsigned long long key_of(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double value_of(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double(static_cast<long long>(b));
}

struct SelState {
  unsigned long long prefix;  // key bits fixed so far
  unsigned long long mask;    // which bits are fixed
  unsigned long long want;    // rank (1-based, from the top) within the prefix bucket
  unsigned long long m;       // target rank
  unsigned int bad;           // a NaN was seen
  unsigned int pad;
};

struct SelScratch {
  SelState st[kSelGroup];
  unsigned int hist[kSelGroup][256];
  double part_sum[kSelBlocks][kSelGroup];
  unsigned long long part_cnt[kSelBlocks][kSelGroup];
  unsigned int done;  // blocks of the current pass that have published their part
};

struct SelMs {
  unsigned long long m[kSelGroup];
};

// The fast path's part of the scratch (after SelScratch): each block's digit
// counts of the second pass, and its sum and count of the values above each
// period's 16-bit bucket.
struct SelFast {
  unsigned int blk_hist[kSelBlocks][kSelGroup][256];
  double above_sum[kSelBlocks][kSelGroup];
  unsigned long long above_cnt[kSelBlocks][kSelGroup];
};

constexpr size_t kSelStateBytes = (sizeof(SelScratch) + 255) & ~size_t(255);
constexpr size_t kSelFastBytes = (sizeof(SelFast) + 255) & ~size_t(255);

__device__ __forceinline__ void sel_init(SelScratch* sc, const SelMs& ms, int g) {
  if (threadIdx.x < g) {
    SelState& st = sc->st[threadIdx.x];
    st.prefix = 0;
    st.mask = 0;
    st.want = ms.m[threadIdx.x];
    st.m = ms.m[threadIdx.x];
    st.bad = 0;
  }
  for (int i = threadIdx.x; i < kSelGroup * 256; i += blockDim.x) (&sc->hist[0][0])[i] = 0;
  if (threadIdx.x == 0) sc->done = 0;
}

__global__ void k_sel_init(SelScratch* sc, SelMs ms, int g) { sel_init(sc, ms, g); }

// True in the block that is the last of the grid to arrive (after each block
// published its part with a fence); that block then sees every part.
__device__ __forceinline__ bool last_block_arrives(SelScratch* sc, int n_blocks) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&sc->done, 1u) == static_cast<unsigned int>(n_blocks) - 1u);
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// One MSB-first digit pass for every return period of the group: histogram of
// the digit among the keys that match each period's prefix (warp-aggregated
// shared-memory counts, then one global add per digit and block); the last
// block to finish picks each period's digit and clears the histogram.
// blk_hist (or NULL): each block also stores its own counts there.  The
// select's grid is nb blocks; this is block bx.
__device__ __forceinline__ void sel_hist(const double* ylt, int64_t n, SelScratch* sc, int g, int shift,
                                         unsigned int* blk_hist, int nb, int bx) {
  __shared__ unsigned int sh[kSelGroup][256];
  for (int i = threadIdx.x; i < kSelGroup * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  unsigned long long prefix[kSelGroup], mask[kSelGroup];
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) {
    prefix[r] = r < g ? sc->st[r].prefix : ~0ull;
    mask[r] = r < g ? sc->st[r].mask : 0ull;
  }
  __syncthreads();
  const int64_t stride = static_cast<int64_t>(nb) * blockDim.x;
  bool nan = false;
  // whole warps take part in every round (the match below needs all lanes)
  const int64_t span = stride * kSelUnroll;
  const int64_t n_round = ((n + span - 1) / span) * span;
  for (int64_t i0 = bx * static_cast<int64_t>(blockDim.x) + threadIdx.x; i0 < n_round; i0 += span) {
    double v[kSelUnroll];
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      v[u] = (i < n) ? ylt[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
      const bool in = i0 + u * stride < n;
      nan |= (v[u] != v[u]);
      const unsigned long long k = key_of(v[u]);
      const unsigned int d = static_cast<unsigned int>((k >> shift) & 255u);
#pragma unroll
      for (int r = 0; r < kSelGroup; ++r) {
        if (r >= g) break;
        const bool hit = in && (k & mask[r]) == prefix[r];
        const unsigned int hm = __ballot_sync(0xffffffffu, hit);
        if (hm == 0u) continue;
        if (__popc(hm) == 1) {  // one key: no aggregation needed
          if (hit) atomicAdd(&sh[r][d], 1u);
          continue;
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, hit ? d : 256u + (threadIdx.x & 31));
        if (hit && (threadIdx.x & 31) == static_cast<unsigned int>(__ffs(peers) - 1))
          atomicAdd(&sh[r][d], static_cast<unsigned int>(__popc(peers)));
      }
    }
  }
  if (nan) atomicOr(&sc->st[0].bad, 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < g * 256; i += blockDim.x) {
    const unsigned int c = (&sh[0][0])[i];
    if (c) atomicAdd(&(&sc->hist[0][0])[i], c);
    if (blk_hist) blk_hist[static_cast<size_t>(bx) * kSelGroup * 256 + i] = c;
  }
  if (!last_block_arrives(sc, nb)) return;
  // ---- pick: per period, the digit holding the wanted rank (a suffix scan of
  // the counts from digit 255 down, thread t holding digit 255 - t)
  __shared__ unsigned int s_warp[kSelThreads / 32];
  for (int r = 0; r < g; ++r) {
    const unsigned int c = (threadIdx.x < 256) ? __ldcg(&sc->hist[r][255 - threadIdx.x]) : 0u;
    unsigned int incl = c;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const unsigned int o = __shfl_up_sync(0xffffffffu, incl, dd);
      if ((threadIdx.x & 31) >= static_cast<unsigned int>(dd)) incl += o;
    }
    if ((threadIdx.x & 31) == 31) s_warp[threadIdx.x >> 5] = incl;
    __syncthreads();
    unsigned int before = 0;
    for (int w = 0; w < static_cast<int>(threadIdx.x >> 5); ++w) before += s_warp[w];
    incl += before;  // counts of digits 255 .. 255 - t
    const unsigned long long want = __ldcg(&sc->st[r].want);
    // the first t (highest digit) whose running count reaches want; digit 0 if none does
    const bool reach = threadIdx.x < 256 && static_cast<unsigned long long>(incl) >= want &&
                       (threadIdx.x == 0 || static_cast<unsigned long long>(incl - c) < want);
    if (reach || (threadIdx.x == 255 && static_cast<unsigned long long>(incl) < want)) {
      SelState& st = sc->st[r];
      st.want = want - (incl - c);
      st.prefix |= static_cast<unsigned long long>(255 - threadIdx.x) << shift;
      st.mask |= 255ull << shift;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kSelGroup * 256; i += blockDim.x) (&sc->hist[0][0])[i] = 0;
  if (threadIdx.x == 0) sc->done = 0;
}

__global__ void k_sel_hist(const double* ylt, int64_t n, SelScratch* sc, int g, int shift, unsigned int* blk_hist) {
  sel_hist(ylt, n, sc, g, shift, blk_hist, static_cast<int>(gridDim.x), static_cast<int>(blockIdx.x));
}

// Sum and count of the values whose key exceeds each selected key.
__global__ void k_sel_tail(const double* ylt, int64_t n, SelScratch* sc, int g, double* pml, double* tvar) {
  __shared__ double s_sum[kSelThreads / 32][kSelGroup];
  __shared__ unsigned long long s_cnt[kSelThreads / 32][kSelGroup];
  unsigned long long kth[kSelGroup];
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) kth[r] = r < g ? sc->st[r].prefix : ~0ull;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  double sum[kSelGroup];
  unsigned long long cnt[kSelGroup];
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) {
    sum[r] = 0.0;
    cnt[r] = 0;
  }
  for (int64_t i0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i0 < n; i0 += stride * kSelUnroll) {
    double v[kSelUnroll];
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      v[u] = (i < n) ? ylt[i] : -INFINITY;
    }
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
      const unsigned long long k = key_of(v[u]);
#pragma unroll
      for (int r = 0; r < kSelGroup; ++r)
        if (i0 + u * stride < n && k > kth[r]) {
          sum[r] += v[u];
          ++cnt[r];
        }
    }
  }
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) {
    for (int d = 16; d > 0; d >>= 1) {
      sum[r] += __shfl_down_sync(0xffffffffu, sum[r], d);
      cnt[r] += __shfl_down_sync(0xffffffffu, cnt[r], d);
    }
    if ((threadIdx.x & 31) == 0) {
      s_sum[threadIdx.x >> 5][r] = sum[r];
      s_cnt[threadIdx.x >> 5][r] = cnt[r];
    }
  }
  __syncthreads();
  if (threadIdx.x < g) {
    const int r = threadIdx.x;
    double t = 0.0;
    unsigned long long c = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
      t += s_sum[w][r];
      c += s_cnt[w][r];
    }
    sc->part_sum[blockIdx.x][r] = t;
    sc->part_cnt[blockIdx.x][r] = c;
  }
  if (!last_block_arrives(sc, static_cast<int>(gridDim.x))) return;
  // ---- finish (the last block): one thread per part, then a tree of fixed
  // shape over the parts, so the sum is deterministic
  __shared__ double s_ps[kSelBlocks];
  __shared__ unsigned long long s_pc[kSelBlocks];
  for (int r = 0; r < g; ++r) {
    const unsigned int i = threadIdx.x;
    if (i < kSelBlocks) {
      s_ps[i] = (i < gridDim.x) ? __ldcg(&sc->part_sum[i][r]) : 0.0;
      s_pc[i] = (i < gridDim.x) ? __ldcg(&sc->part_cnt[i][r]) : 0ull;
    }
    __syncthreads();
    for (unsigned int half = 128; half > 0; half >>= 1) {  // 256 >= kSelBlocks leaves
      if (i < half && i + half < kSelBlocks) {
        s_ps[i] += s_ps[i + half];
        s_pc[i] += s_pc[i + half];
      }
      __syncthreads();
    }
    if (i == 0) {
      const double v = value_of(sc->st[r].prefix);
      const unsigned long long m = sc->st[r].m;
      pml[r] = v;
      tvar[r] = (s_ps[0] + static_cast<double>(m - s_pc[0]) * v) / static_cast<double>(m);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sc->done = 0;
}

// The fast path's third pass: with each period's 16-bit prefix fixed, the
// keys of that bucket are written to cand[r * n ..] in a fixed order (block
// by block, in the order of the block's elements), each block starting at the
// number of bucket keys of the blocks before it (from the second pass's
// per-block counts); each block also publishes the FP64 sum and the count of
// its values above the bucket.  Same grid and element assignment as
// k_sel_hist (a grid of nb blocks; this is block bx).
__device__ __forceinline__ void sel_compact(const double* ylt, int64_t n, const SelScratch* sc, SelFast* sf, int g,
                                            unsigned long long* cand, int nb, int bx) {
  __shared__ unsigned int s_wcnt[kSelThreads / 32][kSelGroup];
  __shared__ unsigned int s_off[kSelGroup];
  __shared__ double s_sum[kSelThreads / 32][kSelGroup];
  __shared__ unsigned long long s_cnt[kSelThreads / 32][kSelGroup];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long prefix[kSelGroup], mask[kSelGroup], top[kSelGroup];
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) {
    prefix[r] = r < g ? sc->st[r].prefix : ~0ull;
    mask[r] = r < g ? sc->st[r].mask : 0ull;
    top[r] = r < g ? (prefix[r] | ~mask[r]) : ~0ull;  // the bucket's largest key
  }
  {
    // this block's first candidate per period: the bucket counts of the blocks
    // before it, summed by the whole block (one earlier block per thread)
    unsigned int part[kSelGroup];
#pragma unroll
    for (int r = 0; r < kSelGroup; ++r) part[r] = 0u;
    for (unsigned int b = threadIdx.x; b < static_cast<unsigned int>(bx); b += blockDim.x) {
#pragma unroll
      for (int r = 0; r < kSelGroup; ++r)
        if (r < g) part[r] += sf->blk_hist[b][r][static_cast<unsigned int>(prefix[r] >> 48) & 255u];
    }
#pragma unroll
    for (int r = 0; r < kSelGroup; ++r) {
      const unsigned int w = __reduce_add_sync(0xffffffffu, part[r]);
      if (lane == 0) s_wcnt[warp][r] = w;
    }
    __syncthreads();
    if (threadIdx.x < static_cast<unsigned int>(g)) {
      unsigned int off = 0;
      for (int w = 0; w < kSelThreads / 32; ++w) off += s_wcnt[w][threadIdx.x];
      s_off[threadIdx.x] = off;
    }
    __syncthreads();
  }
  const int64_t stride = static_cast<int64_t>(nb) * blockDim.x;
  const int64_t span = stride * kSelUnroll;
  const int64_t n_round = ((n + span - 1) / span) * span;
  double sum[kSelGroup];
  unsigned long long cnt[kSelGroup];
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) {
    sum[r] = 0.0;
    cnt[r] = 0;
  }
  for (int64_t i0 = bx * static_cast<int64_t>(blockDim.x) + threadIdx.x; i0 < n_round; i0 += span) {
#pragma unroll 1
    for (int u = 0; u < kSelUnroll; ++u) {
      const bool in = i0 + u * stride < n;
      const double vu = in ? ylt[i0 + u * stride] : 0.0;
      const unsigned long long k = key_of(vu);
      unsigned int bal[kSelGroup];
#pragma unroll
      for (int r = 0; r < kSelGroup; ++r) {
        const bool match = r < g && in && (k & mask[r]) == prefix[r];
        bal[r] = __ballot_sync(0xffffffffu, match);
        if (r < g && in && k > top[r]) {
          sum[r] += vu;
          ++cnt[r];
        }
      }
      if (lane == 0)
#pragma unroll
        for (int r = 0; r < kSelGroup; ++r) s_wcnt[warp][r] = __popc(bal[r]);
      __syncthreads();
      unsigned int total[kSelGroup];
#pragma unroll
      for (int r = 0; r < kSelGroup; ++r) {
        // exclusive prefix of the warps' counts: lane w holds warp w's count
        // (periods r >= g have none)
        const unsigned int c = s_wcnt[lane][r];
        unsigned int incl = c;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const unsigned int o = __shfl_up_sync(0xffffffffu, incl, dd);
          if (lane >= static_cast<unsigned int>(dd)) incl += o;
        }
        const unsigned int before = __shfl_sync(0xffffffffu, incl - c, warp);
        total[r] = __shfl_sync(0xffffffffu, incl, 31);
        if ((bal[r] >> lane) & 1u)
          cand[static_cast<size_t>(r) * n + s_off[r] + before + __popc(bal[r] & ((1u << lane) - 1u))] = k;
      }
      __syncthreads();
      if (threadIdx.x == 0)
#pragma unroll
        for (int r = 0; r < kSelGroup; ++r)
          if (r < g) s_off[r] += total[r];
      __syncthreads();
    }
  }
  // the block's sums above the buckets, in a fixed order
#pragma unroll
  for (int r = 0; r < kSelGroup; ++r) {
    for (int d = 16; d > 0; d >>= 1) {
      sum[r] += __shfl_down_sync(0xffffffffu, sum[r], d);
      cnt[r] += __shfl_down_sync(0xffffffffu, cnt[r], d);
    }
    if (lane == 0) {
      s_sum[warp][r] = sum[r];
      s_cnt[warp][r] = cnt[r];
    }
  }
  __syncthreads();
  if (threadIdx.x < static_cast<unsigned int>(g)) {
    const int r = threadIdx.x;
    double t = 0.0;
    unsigned long long c = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
      t += s_sum[w][r];
      c += s_cnt[w][r];
    }
    sf->above_sum[bx][r] = t;
    sf->above_cnt[bx][r] = c;
  }
}

__global__ void k_sel_compact(const double* ylt, int64_t n, const SelScratch* sc, SelFast* sf, int g,
                              unsigned long long* cand) {
  sel_compact(ylt, n, sc, sf, g, cand, static_cast<int>(gridDim.x), static_cast<int>(blockIdx.x));
}

// The fast path's finish, one block per period: the remaining six digits of
// the m-th key over the bucket's keys, then TVaR from the sums above the
// bucket (the blocks' parts, a tree of fixed shape) and the bucket keys above
// the m-th key (a fixed assignment of keys to threads and a fixed tree).
// Period r's finish (a block).
__device__ __forceinline__ void sel_finish(int64_t n, SelScratch* sc, const SelFast* sf, int n_blk,
                                           const unsigned long long* cand, double* pml, double* tvar, int r) {
  __shared__ unsigned int s_hist[256];
  __shared__ unsigned int s_warp[kSelThreads / 32];
  __shared__ unsigned long long s_prefix, s_mask, s_want;
  __shared__ unsigned int s_c;
  __shared__ double s_ps[256];
  __shared__ unsigned long long s_pc[256];
  const unsigned int t = threadIdx.x, lane = t & 31;
  {
    if (t == 0) {
      s_prefix = sc->st[r].prefix;
      s_mask = sc->st[r].mask;
      s_want = sc->st[r].want;
      const unsigned int d = static_cast<unsigned int>(s_prefix >> 48) & 255u;
      unsigned int c = 0;
      for (int b = 0; b < n_blk; ++b) c += sf->blk_hist[b][r][d];
      s_c = c;
    }
    __syncthreads();
    const unsigned int C = s_c;
    const unsigned long long* ck = cand + static_cast<size_t>(r) * n;
    for (int shift = 40; shift >= 0; shift -= 8) {
      if (t < 256) s_hist[t] = 0;
      __syncthreads();
      const unsigned long long prefix = s_prefix, mask = s_mask;
      for (unsigned int j = t; j < C; j += kSelThreads) {
        const unsigned long long k = ck[j];
        if ((k & mask) == prefix) atomicAdd(&s_hist[(k >> shift) & 255u], 1u);
      }
      __syncthreads();
      // the digit holding the wanted rank (suffix scan, thread t holding digit 255 - t)
      const unsigned int c = (t < 256) ? s_hist[255 - t] : 0u;
      unsigned int incl = c;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const unsigned int o = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= static_cast<unsigned int>(dd)) incl += o;
      }
      if (lane == 31) s_warp[t >> 5] = incl;
      __syncthreads();
      unsigned int before = 0;
      for (unsigned int w = 0; w < (t >> 5); ++w) before += s_warp[w];
      incl += before;
      const unsigned long long want = s_want;
      const bool reach = t < 256 && static_cast<unsigned long long>(incl) >= want &&
                         (t == 0 || static_cast<unsigned long long>(incl - c) < want);
      __syncthreads();
      if (reach || (t == 255 && static_cast<unsigned long long>(incl) < want)) {
        s_want = want - (incl - c);
        s_prefix = prefix | (static_cast<unsigned long long>(255 - t) << shift);
        s_mask = mask | (255ull << shift);
      }
      __syncthreads();
    }
    const unsigned long long kth = s_prefix;
    // bucket keys above the m-th key
    double sum = 0.0;
    unsigned long long cnt = 0;
    for (unsigned int j = t; j < C; j += kSelThreads) {
      const unsigned long long k = ck[j];
      if (k > kth) {
        sum += value_of(k);
        ++cnt;
      }
    }
    for (int d = 16; d > 0; d >>= 1) {
      sum += __shfl_down_sync(0xffffffffu, sum, d);
      cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    }
    if (lane == 0) {
      s_ps[t >> 5] = sum;
      s_pc[t >> 5] = cnt;
    }
    __syncthreads();
    double bucket_sum = 0.0;
    unsigned long long bucket_cnt = 0;
    if (t == 0) {
      for (int w = 0; w < kSelThreads / 32; ++w) {
        bucket_sum += s_ps[w];
        bucket_cnt += s_pc[w];
      }
    }
    __syncthreads();
    // the blocks' parts above the bucket
    if (t < 256) {
      s_ps[t] = (static_cast<int>(t) < n_blk) ? sf->above_sum[t][r] : 0.0;
      s_pc[t] = (static_cast<int>(t) < n_blk) ? sf->above_cnt[t][r] : 0ull;
    }
    __syncthreads();
    for (unsigned int half = 128; half > 0; half >>= 1) {
      if (t < half) {
        s_ps[t] += s_ps[t + half];
        s_pc[t] += s_pc[t + half];
      }
      __syncthreads();
    }
    if (t == 0) {
      const double v = value_of(kth);
      const unsigned long long m = sc->st[r].m;
      const double s_all = s_ps[0] + bucket_sum;
      const unsigned long long c_all = s_pc[0] + bucket_cnt;
      pml[r] = v;
      tvar[r] = (s_all + static_cast<double>(m - c_all) * v) / static_cast<double>(m);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSelThreads) k_sel_finish(int64_t n, SelScratch* sc, const SelFast* sf, int n_blk,
                                                             const unsigned long long* cand, double* pml,
                                                             double* tvar) {
  sel_finish(n, sc, sf, n_blk, cand, pml, tvar, static_cast<int>(blockIdx.x));
}

// ---- batched selects: one launch per pass for several YLTs (jobs), blockIdx.y
// the job; each job runs on its own grid size and scratch exactly as the
// single select does, so it gives the same bits
struct SelJob {
  const double* ylt;
  int64_t n;
  SelScratch* sc;
  SelFast* sf;
  unsigned long long* cand;  // [g][n]
  double* pml;
  double* tvar;
  SelMs ms;
  int g;
  int grid;
};
struct SelBatch {
  SelJob job[kSelBatchMax];
};

__global__ void k_sel_init_batch(const __grid_constant__ SelBatch b) {
  const SelJob& j = b.job[blockIdx.y];
  sel_init(j.sc, j.ms, j.g);
}

__global__ void k_sel_hist_batch(const __grid_constant__ SelBatch b, int shift, int with_blk) {
  const SelJob& j = b.job[blockIdx.y];
  if (static_cast<int>(blockIdx.x) >= j.grid) return;
  sel_hist(j.ylt, j.n, j.sc, j.g, shift, with_blk ? &j.sf->blk_hist[0][0][0] : nullptr, j.grid,
           static_cast<int>(blockIdx.x));
}

__global__ void k_sel_compact_batch(const __grid_constant__ SelBatch b) {
  const SelJob& j = b.job[blockIdx.y];
  if (static_cast<int>(blockIdx.x) >= j.grid) return;
  sel_compact(j.ylt, j.n, j.sc, j.sf, j.g, j.cand, j.grid, static_cast<int>(blockIdx.x));
}

__global__ void __launch_bounds__(kSelThreads) k_sel_finish_batch(const __grid_constant__ SelBatch b) {
  const SelJob& j = b.job[blockIdx.y];
  if (static_cast<int>(blockIdx.x) >= j.g) return;
  sel_finish(j.n, j.sc, j.sf, j.grid, j.cand, j.pml, j.tvar, static_cast<int>(blockIdx.x));
}

int sel_grid(int64_t n) {
  const int64_t blocks = (n + kSelThreads - 1) / kSelThreads;
  return static_cast<int>(blocks < kSelBlocks ? blocks : kSelBlocks);
}

// m = ceil(n / rp), within [1, n]
unsigned long long sel_rank(int64_t n, double rp) {
  int64_t m = static_cast<int64_t>(std::ceil(static_cast<double>(n) / rp));
  if (m < 1) m = 1;
  if (m > n) m = n;
  return static_cast<unsigned long long>(m);
}

cudaError_t launch_sel_batch(const SelBatch& b, int n_jobs, int max_grid, int max_g, cudaStream_t s) {
  const dim3 one(1, n_jobs), wide(max_grid, n_jobs), fin(max_g, n_jobs);
  k_sel_init_batch<<<one, 256, 0, s>>>(b);
  k_sel_hist_batch<<<wide, kSelThreads, 0, s>>>(b, 56, 0);
  k_sel_hist_batch<<<wide, kSelThreads, 0, s>>>(b, 48, 1);
  k_sel_compact_batch<<<wide, kSelThreads, 0, s>>>(b);
  k_sel_finish_batch<<<fin, kSelThreads, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace

size_t select_job_bytes(int64_t n, int n_rp) {
  const int g = n_rp < kSelGroup ? n_rp : kSelGroup;
  const int groups = (n_rp + kSelGroup - 1) / kSelGroup;
  return static_cast<size_t>(groups) * (kSelStateBytes + kSelFastBytes +
                                        ((sizeof(unsigned long long) * g * static_cast<size_t>(n) + 255) & ~size_t(255)));
}

cudaError_t pml_tvar_batch(const SelectSpec* specs, int n_specs, void* pool, size_t pool_bytes, cudaStream_t s,
                           int* n_launch) {
  SelBatch b;
  int n_jobs = 0, max_grid = 1, max_g = 1;
  size_t used = 0;
  unsigned char* base = static_cast<unsigned char*>(pool);
  auto flush = [&]() -> cudaError_t {
    if (n_jobs == 0) return cudaSuccess;
    const cudaError_t e = launch_sel_batch(b, n_jobs, max_grid, max_g, s);
    if (n_launch) *n_launch += 5;
    n_jobs = 0;
    max_grid = max_g = 1;
    used = 0;
    return e;
  };
  for (int i = 0; i < n_specs; ++i) {
    const SelectSpec& q = specs[i];
    if (q.n < 1 || q.n_rp < 1) return cudaErrorInvalidValue;
    for (int r0 = 0; r0 < q.n_rp; r0 += kSelGroup) {
      const int g = (q.n_rp - r0 < kSelGroup) ? (q.n_rp - r0) : kSelGroup;
      const size_t need = kSelStateBytes + kSelFastBytes +
                          ((sizeof(unsigned long long) * g * static_cast<size_t>(q.n) + 255) & ~size_t(255));
      if (need > pool_bytes) return cudaErrorInvalidValue;
      if (n_jobs == kSelBatchMax || used + need > pool_bytes) {
        const cudaError_t e = flush();
        if (e != cudaSuccess) return e;
      }
      SelJob& j = b.job[n_jobs++];
      j.ylt = q.ylt;
      j.n = q.n;
      j.sc = reinterpret_cast<SelScratch*>(base + used);
      j.sf = reinterpret_cast<SelFast*>(base + used + kSelStateBytes);
      j.cand = reinterpret_cast<unsigned long long*>(base + used + kSelStateBytes + kSelFastBytes);
      j.pml = q.pml + r0;
      j.tvar = q.tvar + r0;
      j.ms = SelMs{};
      for (int r = 0; r < g; ++r) j.ms.m[r] = sel_rank(q.n, q.rps[r0 + r]);
      j.g = g;
      j.grid = sel_grid(q.n);
      max_grid = j.grid > max_grid ? j.grid : max_grid;
      max_g = g > max_g ? g : max_g;
      used += need;
    }
  }
  return flush();
}

size_t select_scratch_bytes(int64_t n) {
  return kSelStateBytes + kSelFastBytes + sizeof(unsigned long long) * kSelGroup * static_cast<size_t>(n) + 64;
}

cudaError_t pml_tvar_device(const double* ylt, int64_t n, const double* rps_host, int32_t n_rp, double* pml,
                            double* tvar, void* scratch, size_t scratch_bytes, cudaStream_t s, int* n_launch) {
  SelScratch* sc = static_cast<SelScratch*>(scratch);
  const bool fast = scratch_bytes >= select_scratch_bytes(n);
  SelFast* sf = fast ? reinterpret_cast<SelFast*>(static_cast<unsigned char*>(scratch) + kSelStateBytes) : nullptr;
  unsigned long long* cand =
      fast ? reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(scratch) + kSelStateBytes + kSelFastBytes)
           : nullptr;
  const int grid = sel_grid(n);
  for (int32_t r0 = 0; r0 < n_rp; r0 += kSelGroup) {
    const int g = (n_rp - r0 < kSelGroup) ? (n_rp - r0) : kSelGroup;
    SelMs ms{};
    for (int r = 0; r < g; ++r) ms.m[r] = sel_rank(n, rps_host[r0 + r]);
    k_sel_init<<<1, 256, 0, s>>>(sc, ms, g);
    if (fast) {
      k_sel_hist<<<grid, kSelThreads, 0, s>>>(ylt, n, sc, g, 56, nullptr);
      k_sel_hist<<<grid, kSelThreads, 0, s>>>(ylt, n, sc, g, 48, &sf->blk_hist[0][0][0]);
      k_sel_compact<<<grid, kSelThreads, 0, s>>>(ylt, n, sc, sf, g, cand);
      k_sel_finish<<<g, kSelThreads, 0, s>>>(n, sc, sf, grid, cand, pml + r0, tvar + r0);
      if (n_launch) *n_launch += 5;
    } else {
      for (int shift = 56; shift >= 0; shift -= 8)
        k_sel_hist<<<grid, kSelThreads, 0, s>>>(ylt, n, sc, g, shift, nullptr);
      k_sel_tail<<<grid, kSelThreads, 0, s>>>(ylt, n, sc, g, pml + r0, tvar + r0);
      if (n_launch) *n_launch += 10;
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// =============================================================== LSD radix sort (descending)
namespace {

constexpr int kSortThreads = 1024;  // one key per thread per tile

__global__ void k_sort_keys(const double* ylt, int64_t n, unsigned long long* keys, int64_t* idx) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    keys[i] = ~key_of(ylt[i]);  // ascending order of ~key = descending year loss
    idx[i] = i;
  }
}

__global__ void k_sort_count(const unsigned long long* keys, int64_t n, int shift, unsigned int* counts,
                             int n_tiles) {
  __shared__ unsigned int sh[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kSortThreads + threadIdx.x;
  if (i < n) atomicAdd(&sh[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[static_cast<int64_t>(d) * n_tiles + blockIdx.x] = sh[d];
}

__global__ void k_sort_scatter(const unsigned long long* keys_in, const int64_t* idx_in, int64_t n, int shift,
                               const unsigned int* offsets, int n_tiles, unsigned long long* keys_out,
                               int64_t* idx_out) {
  __shared__ unsigned int s_wc[32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 32 * 256; i += blockDim.x) (&s_wc[0][0])[i] = 0;
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kSortThreads + threadIdx.x;
  const bool valid = i < n;
  const unsigned long long key = valid ? keys_in[i] : 0ull;
  const unsigned int d = valid ? static_cast<unsigned int>((key >> shift) & 255u) : 256u;
  const unsigned int peers = __match_any_sync(0xffffffffu, d);
  const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank == 0) s_wc[warp][d] = __popc(peers);
  __syncthreads();
  if (threadIdx.x < 256) {
    const int dd = threadIdx.x;
    unsigned int run = offsets[static_cast<int64_t>(dd) * n_tiles + blockIdx.x];
    for (int w = 0; w < 32; ++w) {
      const unsigned int c = s_wc[w][dd];
      s_wc[w][dd] = run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    const unsigned int dst = s_wc[warp][d] + rank;
    keys_out[dst] = key;
    idx_out[dst] = idx_in[i];
  }
}

}  // namespace

size_t sort_scratch_bytes(int64_t n) {
  const int64_t tiles = (n + kSortThreads - 1) / kSortThreads;
  const int64_t cnt = 256 * tiles;
  return static_cast<size_t>(n) * (2 * sizeof(unsigned long long) + sizeof(int64_t)) +
         sizeof(unsigned int) * (2 * static_cast<size_t>(cnt) + 1 + scan_tmp_words(cnt)) + 256;
}

cudaError_t sort_desc_device(const double* ylt, int64_t n, int64_t* order, void* scratch, cudaStream_t s,
                             int* n_launch) {
  const int64_t tiles = (n + kSortThreads - 1) / kSortThreads;
  const int64_t cnt = 256 * tiles;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  unsigned long long* keys_a = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* keys_b = keys_a + n;
  int64_t* idx_b = reinterpret_cast<int64_t*>(keys_b + n);
  unsigned int* counts = reinterpret_cast<unsigned int*>(idx_b + n);
  unsigned int* offsets = counts + cnt;
  unsigned int* tmp = offsets + cnt + 1;
  // the final pass must land in `order`; with 8 passes the ping-pong ends where it started
  int64_t* idx_a = order;
  const int grid = static_cast<int>((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  k_sort_keys<<<grid, 256, 0, s>>>(ylt, n, keys_a, idx_a);
  if (n_launch) *n_launch += 1 + 8 * 2;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  unsigned long long *ki = keys_a, *ko = keys_b;
  int64_t *ii = idx_a, *io = idx_b;
  for (int shift = 0; shift < 64; shift += 8) {
    k_sort_count<<<static_cast<int>(tiles), kSortThreads, 0, s>>>(ki, n, shift, counts, static_cast<int>(tiles));
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = scan_exclusive_u32(counts, offsets, cnt, tmp, s, n_launch)) != cudaSuccess) return err;
    k_sort_scatter<<<static_cast<int>(tiles), kSortThreads, 0, s>>>(ki, ii, n, shift, offsets,
                                                                   static_cast<int>(tiles), ko, io);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    unsigned long long* tk = ki;
    ki = ko;
    ko = tk;
    int64_t* ti = ii;
    ii = io;
    io = ti;
  }
  return cudaSuccess;  // 8 swaps: the result is back in idx_a == order
}

size_t sort_pairs_scratch_bytes(int64_t n) {
  const int64_t tiles = (n + kSortThreads - 1) / kSortThreads;
  const int64_t cnt = 256 * tiles;
  return static_cast<size_t>(n) * (sizeof(unsigned long long) + sizeof(int64_t)) +
         sizeof(unsigned int) * (2 * static_cast<size_t>(cnt) + 1 + scan_tmp_words(cnt)) + 256;
}

cudaError_t sort_pairs_ascending(unsigned long long* keys, int64_t* vals, int64_t n, int key_bits, void* scratch,
                                 cudaStream_t s, int* n_launch) {
  const int64_t tiles = (n + kSortThreads - 1) / kSortThreads;
  const int64_t cnt = 256 * tiles;
  const int passes = (key_bits + 7) / 8;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  unsigned long long* keys_b = reinterpret_cast<unsigned long long*>(base);
  int64_t* vals_b = reinterpret_cast<int64_t*>(keys_b + n);
  unsigned int* counts = reinterpret_cast<unsigned int*>(vals_b + n);
  unsigned int* offsets = counts + cnt;
  unsigned int* tmp = offsets + cnt + 1;
  cudaError_t err = cudaSuccess;
  // an odd number of passes ends in the scratch buffers: the data start there, so the result
  // lands in (keys, vals)
  unsigned long long *ki = keys, *ko = keys_b;
  int64_t *ii = vals, *io = vals_b;
  if (passes & 1) {
    if ((err = cudaMemcpyAsync(keys_b, keys, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s)) ||
        (err = cudaMemcpyAsync(vals_b, vals, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s)))
      return err;
    ki = keys_b;
    ko = keys;
    ii = vals_b;
    io = vals;
  }
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    k_sort_count<<<static_cast<int>(tiles), kSortThreads, 0, s>>>(ki, n, shift, counts, static_cast<int>(tiles));
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = scan_exclusive_u32(counts, offsets, cnt, tmp, s, n_launch)) != cudaSuccess) return err;
    k_sort_scatter<<<static_cast<int>(tiles), kSortThreads, 0, s>>>(ki, ii, n, shift, offsets,
                                                                   static_cast<int>(tiles), ko, io);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    std::swap(ki, ko);
    std::swap(ii, io);
  }
  if (n_launch) *n_launch += 2 * passes;
  return cudaSuccess;
}

namespace {

// The first m_valid entries of a descending order: values and global trial
// indices (trial_offset + local index); entries m_valid..m-1 are padding
// (-inf, -1).
__global__ void k_top_gather(const double* ylt, const int64_t* order, int64_t m_valid, int64_t m,
                             int64_t trial_offset, double* vals, int64_t* trials) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m; i += stride) {
    if (i < m_valid) {
      const int64_t t = order[i];
      vals[i] = ylt[t];
      trials[i] = trial_offset + t;
    } else {
      vals[i] = -__longlong_as_double(0x7FF0000000000000ll);
      trials[i] = -1;
    }
  }
}

}  // namespace

cudaError_t top_gather_device(const double* ylt, const int64_t* order, int64_t m_valid, int64_t m, int64_t trial_offset,
                              double* vals, int64_t* trials, cudaStream_t s) {
  const int64_t blocks = (m + 255) / 256;
  k_top_gather<<<static_cast<int>(blocks < 1024 ? (blocks > 0 ? blocks : 1) : 1024), 256, 0, s>>>(
      ylt, order, m_valid, m, trial_offset, vals, trials);
  return cudaGetLastError();
}

}  // namespace ara

// =============================================================== allocation-free PML / TVaR
//
// A fixed block of device memory, owned by the library, holds the select
// state of ara_pml_tvar_noalloc and its device outputs.  In host code the
// name of a __device__ array is only a host-side stand-in; the kernels get
// the block's device address, looked up once per device.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[ARA_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_addr[kNoallocMaxDevices] = {};  // device address of the block, per device

static_assert(ARA_NOALLOC_SCRATCH_BYTES >= 2 * ARA_NOALLOC_MAX_RP * sizeof(double) + sizeof(ara::SelScratch) + 256,
              "fixed block too small for the select state");

}  // namespace

extern "C" ARA_API int ara_pml_tvar_noalloc(const double* ylt, int64_t n, const double* return_periods, int32_t n_rp,
                                            double* pml_out, double* tvar_out, void* cuda_stream) {
  if (!ylt || n < 1 || !return_periods || n_rp < 1 || n_rp > ARA_NOALLOC_MAX_RP || !pml_out || !tvar_out)
    return ARA_EINVAL;
  for (int32_t r = 0; r < n_rp; ++r)
    if (!(return_periods[r] >= 1.0) || !std::isfinite(return_periods[r])) return ARA_EINVAL;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ylt) != cudaSuccess) {
    cudaGetLastError();
    return ARA_EINVAL;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return ARA_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return ARA_ECUDA;
  // memory of another GPU would be read as a peer access
  if (at.type == cudaMemoryTypeDevice && at.device != dev) return ARA_EINVAL;
  // set-up, once per device (with that device current): the block's device address
  if (g_noalloc_addr[dev] == nullptr) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr) {
      cudaGetLastError();
      return ARA_ECUDA;
    }
    g_noalloc_addr[dev] = addr;
  }
  unsigned char* block = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  double* d_out = reinterpret_cast<double*>(block);                      // 2 * ARA_NOALLOC_MAX_RP doubles
  void* state = block + 2 * ARA_NOALLOC_MAX_RP * sizeof(double);          // select state (256-aligned)
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // 0: host memory, 1: device (or managed) memory of this GPU, -1: another GPU's memory
  auto kind_of = [dev](const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
  };
  const int pml_kind = kind_of(pml_out), tvar_kind = kind_of(tvar_out);
  if (pml_kind < 0 || tvar_kind < 0) return ARA_EINVAL;
  const bool pml_dev = pml_kind == 1, tvar_dev = tvar_kind == 1;
  double* d_pml = pml_dev ? pml_out : d_out;
  double* d_tvar = tvar_dev ? tvar_out : d_out + ARA_NOALLOC_MAX_RP;
  // the select kernels reset their own histogram and state on every call
  if (ara::pml_tvar_device(ylt, n, return_periods, n_rp, d_pml, d_tvar, state, sizeof(ara::SelScratch), s, nullptr) !=
      cudaSuccess)
    return ARA_ECUDA;
  if (!pml_dev && cudaMemcpyAsync(pml_out, d_pml, sizeof(double) * n_rp, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return ARA_ECUDA;
  if (!tvar_dev && cudaMemcpyAsync(tvar_out, d_tvar, sizeof(double) * n_rp, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return ARA_ECUDA;
  if ((!pml_dev || !tvar_dev) && cudaStreamSynchronize(s) != cudaSuccess) return ARA_ECUDA;
  return ARA_OK;
}
