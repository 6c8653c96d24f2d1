// Kernels of the ARA engine: input checks and per-record preparation at load
// time, the per-layer event index, and the fused layer kernel (YET stream,
// lookup, Philox, inverse Beta, ELT terms, sum over ELTs, occurrence terms,
// FP64 running sum, aggregate terms, YLT write).
#include <cuda_runtime.h>

#include <cstdint>

#include "ara_internal.h"

namespace ara {

namespace {

__device__ __forceinline__ int4 ld_stream_int4(const int32_t* p) {
  // streamed once: do not keep the YET in L1, evict it first from L2
  return __ldcs(reinterpret_cast<const int4*>(p));
}

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

// Exclusive block scan of one uint32 per thread.  s_warp needs 33 words.
// All threads of the block must call it.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_warps = (blockDim.x + 31) >> 5;
  const uint32_t incl = warp_inclusive_scan(v);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = (lane < n_warps) ? s_warp[lane] : 0u;
    const uint32_t xi = warp_inclusive_scan(x);
    s_warp[lane] = xi - x;
    if (lane == 31) s_warp[32] = xi;
  }
  __syncthreads();
  const uint32_t r = s_warp[warp] + incl - v;
  *total = s_warp[32];
  __syncthreads();
  return r;
}

}  // namespace

// =============================================================== load-time checks
__global__ void k_check_offsets(const int64_t* off, int64_t n_trials, int64_t n_events, uint32_t* flags) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t f = 0;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n_trials; t += stride) {
    const int64_t a = off[t], b = off[t + 1];
    if (b < a) f |= kBadOffsets;
    if (b - a >= (int64_t(1) << 24)) f |= kLongTrial;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (off[0] != 0 || off[n_trials] != n_events) f |= kBadOffsets;
  }
  if (f) atomicOr(flags, f);
}

__global__ void k_check_ids(const int32_t* ids, int64_t n, int32_t catalogue, uint32_t* flags) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int32_t e = ids[i];
    bad |= (e < 0) | (e >= catalogue);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kBadEventId);
}

cudaError_t launch_check_offsets(const int64_t* off, int64_t n_trials, int64_t n_events, uint32_t* flags,
                                 cudaStream_t s) {
  const int64_t blocks = (n_trials + 255) / 256;
  k_check_offsets<<<static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, s>>>(
      off, n_trials, n_events, flags);
  return cudaGetLastError();
}

cudaError_t launch_check_ids(const int32_t* ids, int64_t n, int32_t catalogue, uint32_t* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 1023) / 1024;
  k_check_ids<<<static_cast<int>(blocks < 8192 ? blocks : 8192), 1024, 0, s>>>(ids, n, catalogue, flags);
  return cudaGetLastError();
}

// =============================================================== record preparation (FP64)
namespace {

// Continued fraction of I_x(a, b) (A&S 26.5.8) in FP64, modified Lentz; returns 1/K.
__device__ double beta_cf_f64(double a, double b, double x) {
  const double tiny = 1e-300;
  double K = 1.0, C = 1.0, D = 0.0;
  for (int m = 1; m <= 20000; ++m) {
    const double h = static_cast<double>(m >> 1);
    const double num = (m & 1) ? -(a + h) * (a + b + h) * x / ((a + 2.0 * h) * (a + 2.0 * h + 1.0))
                               : h * (b - h) * x / ((a + 2.0 * h - 1.0) * (a + 2.0 * h));
    D = fma(num, D, 1.0);
    if (fabs(D) < tiny) D = tiny;
    C = 1.0 + num / C;
    if (fabs(C) < tiny) C = tiny;
    D = 1.0 / D;
    const double delta = C * D;
    K *= delta;
    if (fabs(delta - 1.0) < 1e-15) break;
  }
  return 1.0 / K;
}

}  // namespace

// Section 3.4 per record: sigma_b = sigma / max_l, mu_b = mu / max_l,
// sigma_bmax = sqrt(mu_b (1 - mu_b)), sigma_b clipped to (1 - 1e-6) sigma_bmax,
// alpha = mu_b ((sigma_bmax / sigma_b)^2 - 1), beta = (1 - mu_b)(...).
__global__ void k_prepare_records(const int32_t* events, const float* mean, const float* sigma,
                                  const float* exposure, int64_t n, Pair* out, double2* shapes, uint32_t* flags,
                                  int32_t* max_event) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t f = 0;
  int32_t emax = -1;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int32_t e = events[i];
    emax = max(emax, e);
    if (e < 0) f |= kBadEventId;
    if (i > 0 && events[i - 1] >= e) f |= kBadOrder;
    const double mu = mean[i], sg = sigma[i], ex = exposure[i];
    Pair p;
    p.a = p.b = p.m0 = p.c = p.p_half = 0.0f;
    p.max_l = static_cast<float>(ex);
    p.mu = static_cast<float>(mu);
    uint32_t kind = kKindBeta, m0x = 0;
    double sa = 0.0, sb_ = 0.0;
    if (!(mu >= 0.0) || !(sg >= 0.0) || !isfinite(mu) || !isfinite(sg) || !isfinite(ex)) {
      f |= kBadValue;
      kind = kKindZero;
    } else if (mu == 0.0) {
      kind = kKindZero;
    } else if (sg == 0.0) {
      kind = kKindMean;
    } else if (!(ex > mu)) {
      f |= kBadExposure;
      kind = kKindZero;
    } else {
      const double mb = mu / ex, sb0 = sg / ex;
      const double smax = sqrt(mb * (1.0 - mb));
      const double sb = (sb0 >= (1.0 - 1e-6) * smax) ? (1.0 - 1e-6) * smax : sb0;
      const double k = (smax / sb) * (smax / sb) - 1.0;
      const double a = mb * k, b = (1.0 - mb) * k;
      const double x0 = a / (a + b), y0 = b / (a + b);
      const double lnB = lgamma(a) + lgamma(b) - lgamma(a + b);
      const double c = a * log(x0) + b * log(y0) - lnB;
      // I_{1/2}(a, b), only used to pick the side of the root
      const double lfront = -(a + b) * 0.69314718055994530942 - lnB;
      double ph;
      if (0.5 < (a + 1.0) / (a + b + 2.0)) {
        ph = exp(lfront) * beta_cf_f64(a, b, 0.5) / a;
      } else {
        ph = 1.0 - exp(lfront) * beta_cf_f64(b, a, 0.5) / b;
      }
      p.a = static_cast<float>(a);
      p.b = static_cast<float>(b);
      sa = a;
      sb_ = b;
      m0x = (x0 <= y0) ? 1u : 0u;
      p.m0 = static_cast<float>(m0x ? x0 : y0);
      p.c = static_cast<float>(c);
      p.p_half = static_cast<float>(ph);
    }
    p.meta = (kind << 5) | (m0x << 7) | (static_cast<uint32_t>(i) << 9);
    out[i] = p;
    if (shapes) shapes[i] = make_double2(sa, sb_);
  }
  if (f) atomicOr(flags, f);
  // block max of event ids, then one atomic per warp
  for (int d = 16; d > 0; d >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, d));
  if ((threadIdx.x & 31) == 0 && emax >= 0) atomicMax(max_event, emax);
}

cudaError_t launch_prepare_records(const int32_t* events, const float* mean, const float* sigma,
                                   const float* exposure, int64_t n, Pair* out, double2* shapes, uint32_t* flags,
                                   int32_t* max_event, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 127) / 128;
  k_prepare_records<<<static_cast<int>(blocks < 65535 ? blocks : 65535), 128, 0, s>>>(
      events, mean, sigma, exposure, n, out, shapes, flags, max_event);
  return cudaGetLastError();
}

// =============================================================== quantile tables (FP64, load time)
namespace {

// I_x(a, b) and 1 - I_x(a, b), each without cancellation (A&S 26.5.8 with symmetry).
__device__ void beta_inc_pair_f64(double x, double a, double b, double lnB, double* I, double* Ic) {
  if (!(x > 0.0)) {
    *I = 0.0;
    *Ic = 1.0;
    return;
  }
  if (!(x < 1.0)) {
    *I = 1.0;
    *Ic = 0.0;
    return;
  }
  const double front = exp(a * log(x) + b * log1p(-x) - lnB);
  if (x < (a + 1.0) / (a + b + 2.0)) {
    const double v = front * beta_cf_f64(a, b, x) / a;
    *I = v;
    *Ic = 1.0 - v;
  } else {
    const double v = front * beta_cf_f64(b, a, 1.0 - x) / b;
    *Ic = v;
    *I = 1.0 - v;
  }
}

// Root r of I_r(A, B) = p (p <= 1/2) by bracketed Newton in FP64 from `guess`.
__device__ double beta_root_f64(double p, double A, double B, double lnB, double guess) {
  double lo = 0.0, hi = 1.0;
  double r = (guess > 0.0 && guess < 1.0) ? guess : A / (A + B);
  for (int it = 0; it < 200; ++it) {
    double I, Ic;
    beta_inc_pair_f64(r, A, B, lnB, &I, &Ic);
    const double f = I - p;
    if (f == 0.0) return r;
    if (f < 0.0) lo = r; else hi = r;
    const double lpdf = (A - 1.0) * log(r) + (B - 1.0) * log1p(-r) - lnB;
    double rn = r - f * exp(-lpdf);
    if (!(rn > lo && rn < hi)) {
      const double l = fmax(lo, 1e-300);
      if (lo == 0.0 && hi <= 1e-300) return hi;
      rn = (hi > 4.0 * l) ? sqrt(l) * sqrt(hi) : 0.5 * (lo + hi);
    }
    if (fabs(rn - r) <= 1e-14 * rn) return rn;
    r = rn;
  }
  return r;
}

}  // namespace

// One warp per record, lane i = node i at t_i = -T1 + i h.  Each node: the
// FP64 root x_i (seeded by the FP32 Halley solver), w = ln x, w' and w''
// (derivatives in t: w' = phi(t) / (x f(x)), w'' = w' (-t - w' (a - (b-1) x/(1-x)))).
// The stored float4 is {x_i, w_{i+1} - w_i, h w'_i, h^2 w''_i}.  Then each
// segment is checked at s = 1/4, 1/2, 3/4: the FP32 interpolant (as the hot
// path evaluates it) against the FP64 CDF; the record is table-exact when the
// implied relative error of x is within kTabTol everywhere x >= 1e-30.
__global__ void k_build_tables(Pair* recs, const double2* shapes, int64_t n, float4* tab) {
  const int lane = threadIdx.x & 31;
  const int64_t rec = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (rec >= n) return;
  const Pair pr = recs[rec];
  float4* out = tab + rec * kTabNodes;
  if (pair_kind(pr.meta) != kKindBeta) {
    out[lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    return;
  }
  const double a = shapes[rec].x, b = shapes[rec].y;
  const double lnB = lgamma(a) + lgamma(b) - lgamma(a + b);
  const double h = 2.0 * kTabT1 / (kTabNodes - 1);
  const double t = -kTabT1 + h * lane;
  const double zl = normcdf(-fabs(t));  // the smaller tail probability
  // FP32 seed, then FP64 polish on the side where the root keeps relative precision
  BetaSolveStats st;
  const float zf = (t <= 0.0) ? static_cast<float>(zl) : static_cast<float>(1.0 - zl);
  const float seed = pair_quantile_newton(pr, fminf(fmaxf(zf, 5.9604645e-08f), 0.99999994f), -1.0f, &st);
  double w, lny, x;
  if (t <= 0.0) {
    x = beta_root_f64(zl, a, b, lnB, static_cast<double>(seed));
    w = log(x);
    lny = log1p(-x);
  } else {
    const double y = beta_root_f64(zl, b, a, lnB, 1.0 - static_cast<double>(seed));
    x = 1.0 - y;
    w = log1p(-y);
    lny = log(y);
  }
  const double lpdf = (a - 1.0) * w + (b - 1.0) * lny - lnB;
  const double lphi = -0.5 * t * t - 0.91893853320467274178;
  const double D = exp(lphi - w - lpdf);
  const double E = D * (-t - D * (a - (b - 1.0) * exp(w - lny)));
  const double w_next = __shfl_down_sync(0xffffffffu, w, 1);
  const float4 node = make_float4(static_cast<float>(exp(w)), lane < kTabNodes - 1 ? static_cast<float>(w_next - w) : 0.0f,
                                  static_cast<float>(h * D), static_cast<float>(h * h * E));
  out[lane] = node;
  // ---- accuracy check of the interpolant
  const float d1 = __shfl_down_sync(0xffffffffu, node.z, 1);
  const float e1 = __shfl_down_sync(0xffffffffu, node.w, 1);
  bool ok = isfinite(node.x) && isfinite(node.y) && isfinite(node.z) && isfinite(node.w);
  if (lane < kTabNodes - 1) {
    for (int q = 1; q <= 3; ++q) {
      const float sf = 0.25f * q;
      const float xq = (node.x > 0.0f) ? node.x * expf(tab_increment(sf, node.y, node.z, node.w, d1, e1)) : 0.0f;
      if (!(xq >= 1e-30f)) continue;  // negligible losses
      const double tq = t + h * sf;
      const double zq = normcdf(-fabs(tq));
      double I, Ic;
      const double xd = static_cast<double>(xq);
      beta_inc_pair_f64(xd, a, b, lnB, &I, &Ic);
      const double err_z = (tq <= 0.0) ? (I - zq) : (Ic - zq);
      const double lpdf_q = (a - 1.0) * log(xd) + (b - 1.0) * log1p(-xd) - lnB;
      const double rel = fabs(err_z) * exp(-(log(xd) + lpdf_q));
      ok = ok && (rel <= kTabTol) && isfinite(rel);
    }
  }
  const bool all_ok = __all_sync(0xffffffffu, ok);
  if (lane == 0 && all_ok) recs[rec].meta = pr.meta | (1u << 8);
}

cudaError_t launch_build_tables(Pair* recs, const double2* shapes, int64_t n, float4* tab, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 7) / 8;  // 8 warps (records) per block
  k_build_tables<<<static_cast<int>(blocks < 2147483647 ? blocks : 2147483647), 256, 0, s>>>(recs, shapes, n, tab);
  return cudaGetLastError();
}

// =============================================================== check kernels
__global__ void k_debug_uniforms(uint32_t seed_lo, uint32_t seed_hi, int64_t n, const int64_t* trials,
                                 const int32_t* ks, const int32_t* elts, float* out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    out[i] = philox_uniform(seed_lo, seed_hi, trials[i], static_cast<uint32_t>(ks[i]), static_cast<uint32_t>(elts[i]));
}

__global__ void k_debug_losses(const Pair* recs, const float4* tab, const float* z, int64_t n, int newton_only,
                               float* out, int32_t* iters) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    BetaSolveStats st;
    const Pair pr = recs[i];
    out[i] = pair_loss(pr, z[i], false, tab + static_cast<int64_t>(pair_rec(pr.meta)) * kTabNodes, newton_only != 0, &st);
    if (iters) iters[i] = st.converged ? st.iters : -st.iters;
  }
}

cudaError_t launch_debug_uniforms(uint32_t seed_lo, uint32_t seed_hi, int64_t n, const int64_t* trials,
                                  const int32_t* ks, const int32_t* elts, float* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t b = (n + 255) / 256;
  k_debug_uniforms<<<static_cast<int>(b < 65535 ? b : 65535), 256, 0, s>>>(seed_lo, seed_hi, n, trials, ks, elts, out);
  return cudaGetLastError();
}

cudaError_t launch_debug_losses(const Pair* recs, const float4* tab, const float* z, int64_t n, int newton_only,
                                float* out, int32_t* iters, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t b = (n + 127) / 128;
  k_debug_losses<<<static_cast<int>(b < 65535 ? b : 65535), 128, 0, s>>>(recs, tab, z, n, newton_only, out, iters);
  return cudaGetLastError();
}

// =============================================================== exclusive scan (uint32)
namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 8;
constexpr int kScanTile = kScanThreads * kScanPerThread;

// Per-tile sums.
__global__ void k_scan_tile_sums(const uint32_t* in, int64_t n, uint32_t* sums) {
  __shared__ uint32_t s_warp[33];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const int64_t i = base + j;
    if (i < n) v += in[i];
  }
  uint32_t total;
  block_exclusive_scan(v, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of each tile with a starting offset per tile.
__global__ void k_scan_tiles(const uint32_t* in, uint32_t* out, int64_t n, const uint32_t* tile_off,
                             int write_total) {
  __shared__ uint32_t s_warp[33];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t vals[kScanPerThread];
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const int64_t i = base + j;
    vals[j] = (i < n) ? in[i] : 0u;
    v += vals[j];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(v, s_warp, &total) + (tile_off ? tile_off[blockIdx.x] : 0u);
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j) {
    const int64_t i = base + j;
    if (i < n) out[i] = run;
    run += vals[j];
  }
  if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}
}  // namespace

size_t scan_tmp_words(int64_t n) {
  // each level keeps its tile sums and their scan (tiles + tiles + 1 words)
  size_t words = 0;
  int64_t m = n;
  while (m > kScanTile) {
    const int64_t tiles = (m + kScanTile - 1) / kScanTile;
    words += 2 * static_cast<size_t>(tiles) + 1;
    m = tiles;
  }
  return words + 1;
}

cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s,
                               int* n_launch) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
  }
  if (n <= kScanTile) {
    k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, 1);
    if (n_launch) *n_launch += 1;
    return cudaGetLastError();
  }
  if (n_launch) *n_launch += 2;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  uint32_t* sums = tmp;
  uint32_t* sums_scanned = tmp + tiles;  // tiles + 1 words are reserved after the sums by scan_tmp_words
  k_scan_tile_sums<<<static_cast<int>(tiles), kScanThreads, 0, s>>>(in, n, sums);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  // recursive scan of the tile sums (into the space after them)
  err = scan_exclusive_u32(sums, sums_scanned, tiles, tmp + 2 * tiles + 1, s, n_launch);
  if (err != cudaSuccess) return err;
  k_scan_tiles<<<static_cast<int>(tiles), kScanThreads, 0, s>>>(in, out, n, sums_scanned, 1);
  return cudaGetLastError();
}

// =============================================================== layer index
namespace {

__device__ __forceinline__ int find_pos(const LayerEltRefs& r, int64_t i) {
  int p = 0;
  while (p + 1 < r.n_elts && r.rec_begin[p + 1] <= i) ++p;
  return p;
}

__global__ void k_mark_members(LayerEltRefs r, uint32_t* bits) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int32_t e = r.events[p][i - r.rec_begin[p]];
    atomicOr(&bits[e >> 5], 1u << (e & 31));
  }
}

__global__ void k_word_popc(const uint32_t* bits, int64_t n_words, uint32_t* cnt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < n_words; w += stride)
    cnt[w] = __popc(bits[w]);
}

__global__ void k_pack_rankdir(const uint32_t* bits, const uint32_t* base, int64_t n_words, uint2* rankdir) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < n_words; w += stride)
    rankdir[w] = make_uint2(bits[w], base[w]);
}

__device__ __forceinline__ uint32_t rank_of(const uint2* rankdir, int32_t e) {
  const uint2 rd = rankdir[e >> 5];
  const uint32_t bit = 1u << (e & 31);
  return rd.y + __popc(rd.x & (bit - 1u));
}

__global__ void k_mark_positions(LayerEltRefs r, const uint2* rankdir, uint32_t* mask) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int32_t e = r.events[p][i - r.rec_begin[p]];
    atomicOr(&mask[rank_of(rankdir, e)], 1u << p);
  }
}

__global__ void k_slot_counts(const uint32_t* mask, int64_t n, uint32_t* cnt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    cnt[i] = __popc(mask[i]);
}

__global__ void k_fill_pairs(LayerEltRefs r, const uint2* rankdir, const uint32_t* mask,
                             const uint32_t* slot_start, Pair* pairs) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int64_t j = i - r.rec_begin[p];
    const int32_t e = r.events[p][j];
    const uint32_t slot = rank_of(rankdir, e);
    const uint32_t within = __popc(mask[slot] & ((1u << p) - 1u));
    Pair q = r.recs[p][j];
    q.meta = (q.meta & ~31u) | static_cast<uint32_t>(p);
    pairs[slot_start[slot] + within] = q;
  }
}

inline int grid_for(int64_t n, int threads, int cap = 4096) {
  const int64_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t build_layer_index(const LayerEltRefs& refs, LayerIndex& ix, cudaStream_t s, int* n_launch) {
  const int64_t n_recs = refs.rec_begin[refs.n_elts];
  cudaError_t err;
  if ((err = cudaMemsetAsync(ix.bits, 0, sizeof(uint32_t) * ix.n_words, s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(ix.mask, 0, sizeof(uint32_t) * (n_recs > 0 ? n_recs : 1), s)) != cudaSuccess)
    return err;
  int launched = 0;
  if (n_recs > 0) {
    k_mark_members<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.bits);
    ++launched;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  k_word_popc<<<grid_for(ix.n_words, 256), 256, 0, s>>>(ix.bits, ix.n_words, ix.word_cnt);
  ++launched;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // exclusive scan in place (each tile reads its inputs before writing)
  if ((err = scan_exclusive_u32(ix.word_cnt, ix.word_cnt, ix.n_words, ix.scan_tmp, s, &launched)) != cudaSuccess)
    return err;
  k_pack_rankdir<<<grid_for(ix.n_words, 256), 256, 0, s>>>(ix.bits, ix.word_cnt, ix.n_words, ix.rankdir);
  ++launched;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (n_recs > 0) {
    k_mark_positions<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.rankdir, ix.mask);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    k_slot_counts<<<grid_for(n_recs, 256), 256, 0, s>>>(ix.mask, n_recs, ix.slot_cnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = scan_exclusive_u32(ix.slot_cnt, ix.slot_cnt, n_recs, ix.scan_tmp, s, &launched)) != cudaSuccess)
      return err;
    k_fill_pairs<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.rankdir, ix.mask, ix.slot_cnt, ix.pairs);
    launched += 3;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  } else {
    if ((err = cudaMemsetAsync(ix.slot_cnt, 0, sizeof(uint32_t), s)) != cudaSuccess) return err;
  }
  if (n_launch) *n_launch += launched;
  return cudaSuccess;
}

// =============================================================== fused layer kernel
//
// One persistent CTA of 1024 threads per SM takes tiles of kTileTrials
// consecutive trials from a global queue.  For each tile:
//   1. the tile's YET ids stream through in chunks of 4096 (one int4 per
//      thread, evict-first); each id is tested against a shared-memory
//      membership filter of the layer (the catalogue bitmap folded modulo the
//      filter size), and the positives are appended, in YET order, to a
//      shared queue (block scan);
//   2. when the queue holds kFlush entries (or the tile ends) it is flushed:
//      a. each entry is resolved against the exact rank directory: false
//         positives get no pairs, true hits get their slot's pair range;
//      b. a block scan lays the (event, ELT) pairs out densely, so that every
//         lane of every warp inverts one Beta (no lanes idle on misses);
//      c. per pair: Philox uniform, inverse Beta (the record's quantile table,
//         or the Halley iteration for the few records whose table is not
//         exact, in a second dense pass), ELT terms; per event the pair
//         losses are summed in layer order (FP32) and the occurrence terms
//         applied;
//      d. one thread per trial adds its events' occurrence losses, in YET
//         order, into the trial's FP64 running sum;
//   3. at the end of the tile the aggregate terms turn each running sum into
//      the trial's year loss.
// Shared memory layout (dynamic):
//   filt[filt_words] | q_key[kQCap] | q_ps[kQCap] | q_pb[kQCap+1] | q_G[kQCap]
//   | lp[kWin] | s_slow[kWin] | s_off[kTileTrials+1] (8-aligned) | s_S[kTileTrials]
//   | s_hits[kTileTrials] | s_hash[kTileTrials] | s_warp[33] | s_misc[4]

size_t layer_smem_bytes(int filt_words) {
  size_t b = sizeof(uint32_t) * static_cast<size_t>(filt_words);
  b += sizeof(uint32_t) * (4 * static_cast<size_t>(kQCap) + 1);
  b += sizeof(float) * kWin;
  b += sizeof(uint16_t) * kWin;
  b = (b + 7) & ~size_t(7);
  b += sizeof(int64_t) * (kTileTrials + 1);
  b += sizeof(double) * kTileTrials;
  b += sizeof(unsigned long long) * 2 * kTileTrials;
  b += sizeof(uint32_t) * (33 + 4);
  return b;
}

__global__ void __launch_bounds__(kLayerThreads, 1) k_layer(const LayerParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* filt = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* q_key = filt + p.filt_words;
  uint32_t* q_ps = q_key + kQCap;
  uint32_t* q_pb = q_ps + kQCap;
  float* q_G = reinterpret_cast<float*>(q_pb + kQCap + 1);
  float* lp = q_G + kQCap;
  uint16_t* s_slow = reinterpret_cast<uint16_t*>(lp + kWin);
  size_t off_bytes = reinterpret_cast<unsigned char*>(s_slow + kWin) - smem_raw;
  off_bytes = (off_bytes + 7) & ~size_t(7);
  int64_t* s_off = reinterpret_cast<int64_t*>(smem_raw + off_bytes);
  double* s_S = reinterpret_cast<double*>(s_off + kTileTrials + 1);
  unsigned long long* s_hits = reinterpret_cast<unsigned long long*>(s_S + kTileTrials);
  unsigned long long* s_hash = s_hits + kTileTrials;
  uint32_t* s_warp = reinterpret_cast<uint32_t*>(s_hash + kTileTrials);
  uint32_t* s_misc = s_warp + 33;

  const int tid = threadIdx.x;
  const bool diag = (p.diag_hits != nullptr) || (p.diag_hash != nullptr);
  const uint32_t fmask = static_cast<uint32_t>(p.filt_words) - 1u;

  // ---- membership filter: catalogue bitmap folded modulo filt_words
  for (int w = tid; w < p.filt_words; w += blockDim.x) {
    uint32_t v = 0;
    for (int64_t k = w; k < p.n_words; k += p.filt_words) v |= p.rankdir[k].x;
    filt[w] = v;
  }
  __syncthreads();

  unsigned long long local_pairs = 0, local_nc = 0, local_slow = 0;

  for (;;) {
    if (tid == 0) s_misc[0] = static_cast<uint32_t>(atomicAdd(&p.counters[0], 1ull));
    __syncthreads();
    const int64_t tile = s_misc[0];
    __syncthreads();
    if (tile >= p.n_tiles) break;
    const int64_t ta = p.t_begin + tile * kTileTrials;
    const int64_t tb = (ta + kTileTrials < p.t_end) ? ta + kTileTrials : p.t_end;
    const int ntr = static_cast<int>(tb - ta);
    for (int j = tid; j <= ntr; j += blockDim.x) s_off[j] = p.off[ta + j];
    for (int j = tid; j < ntr; j += blockDim.x) {
      s_S[j] = 0.0;
      s_hits[j] = 0ull;
      s_hash[j] = 0ull;
    }
    __syncthreads();
    const int64_t ea = s_off[0], eb = s_off[ntr];

    int qn = 0;
    int64_t c0 = ea & ~int64_t(3);
    int4 cur = make_int4(0, 0, 0, 0);
    {
      const int64_t base = c0 + 4 * tid;
      if (base < eb) cur = ld_stream_int4(p.ids + base);
    }
    while (c0 < eb) {
      const int64_t next = c0 + kChunk;
      int4 nxt = make_int4(0, 0, 0, 0);
      {
        const int64_t base = next + 4 * tid;
        if (base < eb) nxt = ld_stream_int4(p.ids + base);  // prefetch the next chunk
      }
      // ---- 1. filter the chunk
      const int64_t base = c0 + 4 * tid;
      const int32_t ev[4] = {cur.x, cur.y, cur.z, cur.w};
      uint32_t hitmask = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t pos = base + j;
        if (pos >= ea && pos < eb) {
          const uint32_t e = static_cast<uint32_t>(ev[j]);
          const uint32_t word = filt[(e >> 5) & fmask];
          if ((word >> (e & 31)) & 1u) hitmask |= 1u << j;
        }
      }
      uint32_t total;
      uint32_t slot = block_exclusive_scan(__popc(hitmask), s_warp, &total);
      if (hitmask) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (hitmask & (1u << j)) {
            const int64_t pos = base + j;
            // trial of pos: the last s_off[t] <= pos
            int lo = 0, hi = ntr;  // s_off[lo] <= pos < s_off[hi]
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (s_off[mid] <= pos) lo = mid; else hi = mid;
            }
            const uint32_t k = static_cast<uint32_t>(pos - s_off[lo]);
            q_key[qn + slot] = (static_cast<uint32_t>(lo) << 24) | k;
            q_ps[qn + slot] = static_cast<uint32_t>(ev[j]);
            ++slot;
          }
        }
      }
      qn += static_cast<int>(total);
      const bool last = (next >= eb);
      cur = nxt;
      c0 = next;
      if (qn < kFlush && !last) {
        __syncthreads();
        continue;
      }
      __syncthreads();
      // ---- 2a. resolve queued entries against the exact rank directory
      for (int h = tid; h < qn; h += blockDim.x) {
        const uint32_t e = q_ps[h];
        const uint2 rd = __ldg(&p.rankdir[e >> 5]);
        const uint32_t bit = 1u << (e & 31);
        uint32_t ps = 0, cnt = 0;
        if (rd.x & bit) {
          const uint32_t sl = rd.y + __popc(rd.x & (bit - 1u));
          ps = __ldg(&p.slot_start[sl]);
          cnt = __ldg(&p.slot_start[sl + 1]) - ps;
        }
        q_ps[h] = ps;
        q_pb[h] = cnt;
        q_G[h] = 0.0f;
      }
      __syncthreads();
      // ---- 2b. block scan of pair counts (5 entries per thread)
      {
        constexpr int kPer = (kQCap + kLayerThreads - 1) / kLayerThreads;
        uint32_t vals[kPer];
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int h = tid * kPer + j;
          vals[j] = (h < qn) ? q_pb[h] : 0u;
          sum += vals[j];
        }
        uint32_t tot;
        uint32_t run = block_exclusive_scan(sum, s_warp, &tot);
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int h = tid * kPer + j;
          if (h < qn) q_pb[h] = run;
          run += vals[j];
        }
        if (tid == 0) q_pb[qn] = tot;
        __syncthreads();
      }
      const uint32_t n_pairs = q_pb[qn];
      // ---- 2c. secondary uncertainty over dense pair windows.  Pairs whose
      // record is table-exact (or carries no uncertainty) finish in the first
      // pass; the rest are listed and run the Halley iteration in a second,
      // dense pass, so that no warp idles on a few slow lanes.
      for (uint32_t w0 = 0; w0 < n_pairs; w0 += kWin) {
        const uint32_t w1 = (w0 + kWin < n_pairs) ? w0 + kWin : n_pairs;
        if (tid == 0) s_misc[1] = 0;
        __syncthreads();
        for (uint32_t pi = w0 + tid; pi < w1; pi += blockDim.x) {
          int lo = 0, hi = qn;  // q_pb[lo] <= pi < q_pb[hi]
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (q_pb[mid] <= pi) lo = mid; else hi = mid;
          }
          const Pair pr = p.pairs[q_ps[lo] + (pi - q_pb[lo])];
          const uint32_t key = q_key[lo];
          const int tl = static_cast<int>(key >> 24);
          const uint32_t k = key & 0xFFFFFFu;
          const uint32_t pos = pair_pos(pr.meta);
          const uint32_t elt = static_cast<uint32_t>(p.elt_id[pos]);
          ++local_pairs;
          if (diag) {
            atomicAdd(&s_hits[tl], 1ull);
            atomicAdd(&s_hash[tl], static_cast<unsigned long long>(fmix64((static_cast<uint64_t>(k) << 32) | elt)));
          }
          const uint32_t kind = pair_kind(pr.meta);
          float loss = pr.mu;
          if (kind == kKindZero) {
            loss = 0.0f;
          } else if (!p.primary_only && kind == kKindBeta) {
            if (p.newton_only || !pair_tab_exact(pr.meta)) {
              s_slow[atomicAdd(&s_misc[1], 1u)] = static_cast<uint16_t>(pi - w0);
              continue;
            }
            const float z = philox_uniform(p.seed_lo, p.seed_hi, ta + tl, k, elt);
            loss = pr.max_l * tab_quantile(p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes, z);
          }
          lp[pi - w0] = p.t_share[pos] * clamp_terms_f(loss, p.t_ret[pos], p.t_lim[pos]);
        }
        __syncthreads();
        const uint32_t n_slow = s_misc[1];
        for (uint32_t j = tid; j < n_slow; j += blockDim.x) {
          const uint32_t li = s_slow[j];
          const uint32_t pi = w0 + li;
          int lo = 0, hi = qn;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (q_pb[mid] <= pi) lo = mid; else hi = mid;
          }
          const Pair pr = p.pairs[q_ps[lo] + (pi - q_pb[lo])];
          const uint32_t key = q_key[lo];
          const uint32_t pos = pair_pos(pr.meta);
          const float z = philox_uniform(p.seed_lo, p.seed_hi, ta + static_cast<int>(key >> 24), key & 0xFFFFFFu,
                                         static_cast<uint32_t>(p.elt_id[pos]));
          const float4* tab = p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes;
          BetaSolveStats st;
          const float x = pair_quantile_newton(pr, z, p.newton_only ? -1.0f : tab_quantile(tab, z), &st);
          if (!st.converged) ++local_nc;
          ++local_slow;
          lp[li] = p.t_share[pos] * clamp_terms_f(pr.max_l * x, p.t_ret[pos], p.t_lim[pos]);
        }
        __syncthreads();
        // per event: sum its pair losses in layer order
        for (int h = tid; h < qn; h += blockDim.x) {
          uint32_t a = q_pb[h], b = q_pb[h + 1];
          if (a < w0) a = w0;
          if (b > w1) b = w1;
          if (a < b) {
            float g = q_G[h];
            for (uint32_t q = a; q < b; ++q) g += lp[q - w0];
            q_G[h] = g;
          }
        }
        __syncthreads();
      }
      // ---- 2d. occurrence terms and the trials' FP64 running sums, in YET order
      for (int h = tid; h < qn; h += blockDim.x) {
        const uint32_t tr = q_key[h] >> 24;
        if (h == 0 || (q_key[h - 1] >> 24) != tr) {
          double S = s_S[tr];
          for (int i = h; i < qn && (q_key[i] >> 24) == tr; ++i) {
            S += static_cast<double>(clamp_terms_f(q_G[i], p.occ_r, p.occ_l));
          }
          s_S[tr] = S;
        }
      }
      __syncthreads();
      qn = 0;
    }
    // ---- 3. aggregate terms: year loss of each trial of the tile
    for (int j = tid; j < ntr; j += blockDim.x) {
      const int64_t out = ta + j - p.t_begin;
      p.ylt[out] = clamp_terms_d(s_S[j], p.agg_r, p.agg_l);
      if (p.diag_hits) p.diag_hits[out] = static_cast<int64_t>(s_hits[j]);
      if (p.diag_hash) p.diag_hash[out] = s_hash[j];
    }
    __syncthreads();
  }
  // counters: pairs evaluated and non-converged inversions
  for (int d = 16; d > 0; d >>= 1) {
    local_pairs += __shfl_xor_sync(0xffffffffu, local_pairs, d);
    local_nc += __shfl_xor_sync(0xffffffffu, local_nc, d);
    local_slow += __shfl_xor_sync(0xffffffffu, local_slow, d);
  }
  if ((tid & 31) == 0) {
    if (local_pairs) atomicAdd(&p.counters[1], local_pairs);
    if (local_nc) atomicAdd(&p.counters[2], local_nc);
    if (local_slow) atomicAdd(&p.counters[3], local_slow);
  }
}

cudaError_t launch_layer_kernel(const LayerParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(k_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  k_layer<<<grid, kLayerThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ara
