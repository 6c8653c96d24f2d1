// Kernels of the ARA engine: input checks and per-record preparation at load
// time, the per-layer event index, and the fused layer kernel (YET stream,
// lookup, Philox, inverse Beta, ELT terms, sum over ELTs, occurrence terms,
// FP64 running sum, aggregate terms, YLT write).
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
    if (b - a >= static_cast<int64_t>(kMaxTrialEvents)) f |= kLongTrial;
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

// Continued fraction of I_x(a, b) (A&S 26.5.8) in FP64; returns 1/K with
// K = 1 + d1/(1 + d2/(1 + ...)), d_n = p_n / q_n:
//   n = 2m+1: p_n = -(a + m)(a + b + m) x, q_n = (a + 2m)(a + 2m + 1),
//   n = 2m:   p_n = m (b - m) x,            q_n = (a + 2m - 1)(a + 2m).
// The equivalence transformation with c_n = q_n clears the denominators
// (partial numerators q_{n-1} p_n, partial denominators q_n), so the forward
// recurrence A_n = b'_n A_{n-1} + a'_n A_{n-2} (and B_n alike) needs only
// multiply-adds; every 8 terms the pairs are rescaled by 1/B_n, which is where
// convergence of A_n / B_n is tested.  FP64 divisions are slow on this GPU, so
// this costs about a tenth of the modified Lentz method.
__device__ double beta_cf_f64(double a, double b, double x) {
  double A2 = 1.0, B2 = 0.0;  // A_{n-2}, B_{n-2}
  double A1 = 1.0, B1 = 1.0;  // A_{n-1}, B_{n-1}
  double q_prev = 1.0, f_prev = 1.0;
  for (int n = 1; n <= 40000; ++n) {
    const double h = static_cast<double>(n >> 1);
    double pn, qn;
    if (n & 1) {
      pn = -(a + h) * (a + b + h) * x;
      qn = (a + 2.0 * h) * (a + 2.0 * h + 1.0);
    } else {
      pn = h * (b - h) * x;
      qn = (a + 2.0 * h - 1.0) * (a + 2.0 * h);
    }
    const double an = q_prev * pn;  // q_0 = 1 gives a'_1 = p_1
    const double A0 = fma(qn, A1, an * A2);
    const double B0 = fma(qn, B1, an * B2);
    A2 = A1;
    B2 = B1;
    A1 = A0;
    B1 = B0;
    q_prev = qn;
    if ((n & 7) == 0) {
      const double inv = 1.0 / B1;
      A1 *= inv;
      A2 *= inv;
      B2 *= inv;
      B1 = 1.0;
      if (fabs(A1 - f_prev) <= 1e-15 * fabs(A1)) break;
      f_prev = A1;
    }
  }
  return B1 / A1;
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
// The nodes are stored in FP32, so the iteration stops at 2e-10 relative:
// well below FP32 resolution, and above the ~1e-12 relative noise of the FP64
// evaluation of I for large shapes (cancellation in ln B(A, B)), which a
// tighter tolerance would chase for the whole iteration budget.
__device__ double beta_root_f64(double p, double A, double B, double lnB, double guess) {
  double lo = 0.0, hi = 1.0;
  double r = (guess > 0.0 && guess < 1.0) ? guess : A / (A + B);
  for (int it = 0; it < 60; ++it) {
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
    } else if (fabs(rn - r) <= 2e-10 * rn) {
      return rn;
    }
    r = rn;
  }
  return r;
}

// Polish of an FP32 root r of I_r(A, B) = p (p <= 1/2): Newton on u = ln r in
// FP64, where I ~ r^A near 0 makes the step almost exact; at most 3 steps (the
// seed is good to ~1e-6, so one step reaches 1e-12).  A seed that does not
// converge goes to the bracketed solver.
__device__ double beta_polish_f64(double p, double A, double B, double lnB, double seed) {
  double r = seed;
  if (!(r > 0.0 && r < 1.0)) return beta_root_f64(p, A, B, lnB, -1.0);
  double du = 1.0;
  for (int it = 0; it < 3 && fabs(du) > 2e-10; ++it) {
    double I, Ic;
    beta_inc_pair_f64(r, A, B, lnB, &I, &Ic);
    if (!(I > 0.0)) return beta_root_f64(p, A, B, lnB, seed);
    const double lpdf = (A - 1.0) * log(r) + (B - 1.0) * log1p(-r) - lnB;
    const double g = r * exp(lpdf) / I;  // d ln I / d ln r
    du = -log1p((I - p) / p) / g;
    if (!(fabs(du) < 0.5)) return beta_root_f64(p, A, B, lnB, seed);
    const double rn = fma(r, expm1(du), r);
    if (!(rn > 0.0 && rn < 1.0)) return beta_root_f64(p, A, B, lnB, seed);
    r = rn;
  }
  if (fabs(du) > 1e-8) return beta_root_f64(p, A, B, lnB, r);
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
    x = beta_polish_f64(zl, a, b, lnB, static_cast<double>(seed));
    w = log(x);
    lny = log1p(-x);
  } else {
    const double y = beta_polish_f64(zl, b, a, lnB, 1.0 - static_cast<double>(seed));
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

__global__ void k_mark_members(LayerEltRefs r, uint32_t* bits, uint32_t* word_pairs) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int32_t e = r.events[p][i - r.rec_begin[p]];
    atomicOr(&bits[e >> 5], 1u << (e & 31));
    atomicAdd(&word_pairs[e >> 5], 1u);  // every record is one (event, ELT) pair
  }
}

__global__ void k_word_popc(const uint32_t* bits, int64_t n_words, uint32_t* cnt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < n_words; w += stride)
    cnt[w] = __popc(bits[w]);
}

// rankdir[w] = {bits, base}: base = pairs before the word when every event of
// the word has one ELT record (its pair is then base + rank in the word), else
// (1 << 31) | slots before the word (pair range from slot_start).
__global__ void k_pack_rankdir(const uint32_t* bits, const uint32_t* base, const uint32_t* pbase, int64_t n_words,
                               uint2* rankdir) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w < n_words; w += stride) {
    const uint32_t b = bits[w];
    const bool multi = (pbase[w + 1] - pbase[w] != static_cast<uint32_t>(__popc(b)));
    rankdir[w] = make_uint2(b, multi ? (0x80000000u | base[w]) : pbase[w]);
  }
}

// Slot (rank among the layer's events) of a member event e.
__device__ __forceinline__ uint32_t rank_of(const uint32_t* bits, const uint32_t* slot_base, int32_t e) {
  const uint32_t bit = 1u << (e & 31);
  return slot_base[e >> 5] + __popc(bits[e >> 5] & (bit - 1u));
}

__global__ void k_mark_positions(LayerEltRefs r, const uint32_t* bits, const uint32_t* slot_base, uint32_t* mask) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int32_t e = r.events[p][i - r.rec_begin[p]];
    atomicOr(&mask[rank_of(bits, slot_base, e)], 1u << p);
  }
}

__global__ void k_slot_counts(const uint32_t* mask, int64_t n, uint32_t* cnt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    cnt[i] = __popc(mask[i]);
}

__global__ void k_fill_pairs(LayerEltRefs r, const uint32_t* bits, const uint32_t* slot_base, const uint32_t* mask,
                             const uint32_t* slot_start, Pair* pairs) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int64_t j = i - r.rec_begin[p];
    const int32_t e = r.events[p][j];
    const uint32_t slot = rank_of(bits, slot_base, e);
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
  if ((err = cudaMemsetAsync(ix.word_pairs, 0, sizeof(uint32_t) * (ix.n_words + 1), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(ix.mask, 0, sizeof(uint32_t) * (n_recs > 0 ? n_recs : 1), s)) != cudaSuccess)
    return err;
  int launched = 0;
  if (n_recs > 0) {
    k_mark_members<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.bits, ix.word_pairs);
    ++launched;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  k_word_popc<<<grid_for(ix.n_words, 256), 256, 0, s>>>(ix.bits, ix.n_words, ix.word_cnt);
  ++launched;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // exclusive scan in place (each tile reads its inputs before writing)
  if ((err = scan_exclusive_u32(ix.word_cnt, ix.word_cnt, ix.n_words, ix.scan_tmp, s, &launched)) != cudaSuccess)
    return err;
  if ((err = scan_exclusive_u32(ix.word_pairs, ix.word_pairs, ix.n_words, ix.scan_tmp, s, &launched)) != cudaSuccess)
    return err;
  k_pack_rankdir<<<grid_for(ix.n_words, 256), 256, 0, s>>>(ix.bits, ix.word_cnt, ix.word_pairs, ix.n_words,
                                                           ix.rankdir);
  ++launched;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (n_recs > 0) {
    k_mark_positions<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.bits, ix.word_cnt, ix.mask);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    k_slot_counts<<<grid_for(n_recs, 256), 256, 0, s>>>(ix.mask, n_recs, ix.slot_cnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = scan_exclusive_u32(ix.slot_cnt, ix.slot_cnt, n_recs, ix.scan_tmp, s, &launched)) != cudaSuccess)
      return err;
    k_fill_pairs<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.bits, ix.word_cnt, ix.mask, ix.slot_cnt, ix.pairs);
    launched += 3;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  } else {
    if ((err = cudaMemsetAsync(ix.slot_cnt, 0, sizeof(uint32_t), s)) != cudaSuccess) return err;
  }
  if (n_launch) *n_launch += launched;
  return cudaSuccess;
}

// =============================================================== layer kernels
//
// k_gather: one persistent CTA of 32 warps per SM.  The CTA folds the layer's
// catalogue bitmap into a shared-memory membership filter once; then each warp
// independently takes tiles of kWarpTrials consecutive trials and streams the
// tile's YET ids, 128 per step (one int4 per lane, evict-first, the next step
// in flight).  Each id is tested against the filter; each positive is resolved
// against the rank directory (8 bytes: the word's bits and its pair base) and,
// if it is a member, becomes an event record written in YET order to the
// tile's region of the event buffer.
//
// k_losses: each warp takes tiles and reads their records in windows of up to
// 32 events whose (event, ELT) pairs number at most 32, one pair per lane:
// Philox uniform, inverse Beta through the record's quantile table, ELT terms.
// A segmented warp reduction sums each event's pair losses in layer order
// (FP32) and applies the occurrence terms; a segmented double-float reduction
// adds the window's occurrence losses of each trial into the trial's FP64
// running sum (one FP64 add per trial and window).  Events with a pair whose
// record's table is not exact are deferred and resolved, 32 at a time, by the
// FP32 Halley iteration.  The aggregate terms turn each running sum into the
// trial's year loss.

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

constexpr uint32_t kRecTrialShift = 27;
constexpr uint32_t kRecCntShift = 22;
constexpr uint32_t kRecKMask = (1u << 22) - 1u;

struct GatherWarp {
  int32_t off[kWarpTrials + 1];  // trial offsets relative to the tile's first event
  uint32_t pos_e[128];           // filter positives of one step: event id
  int32_t pos_rel[128];          //                               tile-relative position
};

}  // namespace

size_t gather_smem_bytes(int filt_words) {
  return sizeof(uint32_t) * static_cast<size_t>(filt_words) + sizeof(GatherWarp) * (kGatherThreads / 32) + 16;
}

int gather_filter_words(int64_t n_words, int max_smem) {
  int fw = 1;
  while (fw < n_words && gather_smem_bytes(fw * 2) <= static_cast<size_t>(max_smem)) fw *= 2;
  return fw;
}

__global__ void __launch_bounds__(kGatherThreads, 1) k_gather(const GatherParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GatherWarp* gw = reinterpret_cast<GatherWarp*>(smem_raw);
  uint32_t* filt = reinterpret_cast<uint32_t*>(gw + (kGatherThreads / 32));
  const uint32_t lane = lane_id();
  GatherWarp& ws = gw[threadIdx.x >> 5];
  const uint32_t fmask = static_cast<uint32_t>(p.filt_words) - 1u;
  const uint32_t lt_mask = (1u << lane) - 1u;

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
    if (lane <= static_cast<uint32_t>(ntr)) ws.off[lane] = static_cast<int32_t>(__ldg(&p.off[ta + lane]) - ea);
    __syncwarp();
    const int32_t nev = ws.off[ntr];
    const int32_t* ids = p.ids + (ea & ~int64_t(3));
    const int32_t lead = static_cast<int32_t>(ea & 3);
    const int32_t span = nev + lead;
    uint2* out = p.ev_buf + (ea - p.e0);
    uint32_t nout = 0;
    int tcur = 0;
    while (tcur + 1 < ntr && ws.off[tcur + 1] <= 0) ++tcur;
    int4 cur = make_int4(0, 0, 0, 0);
    if (4 * static_cast<int32_t>(lane) < span) cur = __ldcs(reinterpret_cast<const int4*>(ids) + lane);
    for (int32_t c0 = 0; c0 < span; c0 += 128) {
      int4 nxt = make_int4(0, 0, 0, 0);
      if (c0 + 128 + 4 * static_cast<int32_t>(lane) < span)
        nxt = __ldcs(reinterpret_cast<const int4*>(ids + c0 + 128) + lane);
      const int32_t rel0 = c0 + 4 * static_cast<int32_t>(lane) - lead;
      const int32_t ev[4] = {cur.x, cur.y, cur.z, cur.w};
      // 1. filter the lane's four ids (shift counts of a funnel shift are taken mod 32)
      uint32_t m = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t e = static_cast<uint32_t>(ev[j]);
        const uint32_t w = filt[(e >> 5) & fmask];
        const bool in = static_cast<uint32_t>(rel0 + j) < static_cast<uint32_t>(nev);
        m |= (in ? (__funnelshift_r(w, w, e) & 1u) : 0u) << j;
      }
      // 2. compact the positives of the warp, in YET order, into the staging list
      const uint32_t c = __popc(m);
      const uint32_t incl = warp_inclusive_scan(c);
      const uint32_t npos = __shfl_sync(0xffffffffu, incl, 31);
      if (m) {
        uint32_t at = incl - c;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (m & (1u << j)) {
            ws.pos_e[at] = static_cast<uint32_t>(ev[j]);
            ws.pos_rel[at] = rel0 + j;
            ++at;
          }
        }
      }
      __syncwarp();
      // 3. resolve the positives, one per lane, and write the hit-event records
      for (uint32_t r0 = 0; r0 < npos; r0 += 32) {
        const bool valid = r0 + lane < npos;
        uint32_t key = 0, ps = 0;
        bool hit = false;
        int32_t rel = 0;
        if (valid) {
          const uint32_t e = ws.pos_e[r0 + lane];
          rel = ws.pos_rel[r0 + lane];
          const uint2 rd = __ldg(&p.rankdir[e >> 5]);
          const uint32_t bit = 1u << (e & 31);
          if (rd.x & bit) {
            hit = true;
            const uint32_t below = __popc(rd.x & (bit - 1u));
            uint32_t cnt = 1;
            if (rd.y & 0x80000000u) {
              const uint32_t sl = (rd.y & 0x7FFFFFFFu) + below;
              ps = __ldg(&p.slot_start[sl]);
              cnt = __ldg(&p.slot_start[sl + 1]) - ps;
            } else {
              ps = rd.y + below;
            }
            int t = tcur;
            while (t + 1 < ntr && ws.off[t + 1] <= rel) ++t;
            key = ((cnt - 1u) << kRecCntShift) | (static_cast<uint32_t>(t) << kRecTrialShift) |
                  static_cast<uint32_t>(rel - ws.off[t]);
          }
        }
        const uint32_t hm = __ballot_sync(0xffffffffu, hit);
        if (hit) out[nout + __popc(hm & lt_mask)] = make_uint2(key, ps);
        nout += __popc(hm);
      }
      __syncwarp();
      {
        const int32_t nrel = c0 + 128 - lead;
        while (tcur + 1 < ntr && ws.off[tcur + 1] <= nrel) ++tcur;
      }
      cur = nxt;
    }
    if (lane == 0) p.tile_cnt[tile] = nout;
    __syncwarp();
  }
}

cudaError_t launch_gather(const GatherParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err =
      cudaFuncSetAttribute(k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  k_gather<<<grid, kGatherThreads, smem, s>>>(p);
  return cudaGetLastError();
}

namespace {

struct LossWarp {
  uint32_t d_key[32];  // deferred events: record
  uint32_t d_ps[32];
  double S[kWarpTrials];
  unsigned long long hits[kWarpTrials];
  unsigned long long hash[kWarpTrials];
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

// Loss after ELT terms of one pair, for the table path; returns false when the
// pair needs the Halley iteration.
__device__ __forceinline__ bool pair_fast(const LossParams& p, const Pair& pr, int64_t trial, uint32_t k, float* out) {
  const uint32_t kind = pair_kind(pr.meta);
  const uint32_t pos = pair_pos(pr.meta);
  float loss = pr.mu;
  if (kind == kKindZero) {
    loss = 0.0f;
  } else if (!p.primary_only && kind == kKindBeta) {
    if (p.newton_only || !pair_tab_exact(pr.meta)) return false;
    const float z = philox_uniform(p.seed_lo, p.seed_hi, trial, k, static_cast<uint32_t>(p.elt_id[pos]));
    loss = pr.max_l * tab_quantile(p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes, z);
  }
  *out = p.t_share[pos] * clamp_terms_f(loss, p.t_ret[pos], p.t_lim[pos]);
  return true;
}

__device__ __noinline__ float pair_slow(const LossParams& p, const Pair& pr, int64_t trial, uint32_t k,
                                        unsigned long long* nc) {
  const uint32_t pos = pair_pos(pr.meta);
  float v;
  if (pair_fast(p, pr, trial, k, &v)) return v;
  const float z = philox_uniform(p.seed_lo, p.seed_hi, trial, k, static_cast<uint32_t>(p.elt_id[pos]));
  const float4* tab = p.tab[pos] + static_cast<size_t>(pair_rec(pr.meta)) * kTabNodes;
  BetaSolveStats st;
  const float x = pair_quantile_newton(pr, z, p.newton_only ? -1.0f : tab_quantile(tab, z), &st);
  if (!st.converged) ++*nc;
  return p.t_share[pos] * clamp_terms_f(pr.max_l * x, p.t_ret[pos], p.t_lim[pos]);
}

// Resolve the deferred events of the warp (all lanes call it): each lane one
// event, then the occurrence losses are added to the trial sums in list order.
__device__ __noinline__ void resolve_deferred(const LossParams& p, LossWarp& ws, int nd, int64_t ta,
                                              unsigned long long* nc, unsigned long long* n_slow) {
  const uint32_t lane = lane_id();
  float O = 0.0f;
  uint32_t tl = 0;
  if (lane < static_cast<uint32_t>(nd)) {
    const uint32_t key = ws.d_key[lane];
    tl = key >> kRecTrialShift;
    const uint32_t k = key & kRecKMask;
    const uint32_t cnt = ((key >> kRecCntShift) & 31u) + 1u;
    float G = 0.0f;
    for (uint32_t j = 0; j < cnt; ++j) G += pair_slow(p, p.pairs[ws.d_ps[lane] + j], ta + tl, k, nc);
    O = clamp_terms_f(G, p.occ_r, p.occ_l);
    ++*n_slow;
  }
  for (int i = 0; i < nd; ++i) {
    const float Oi = __shfl_sync(0xffffffffu, O, i);
    const uint32_t ti = __shfl_sync(0xffffffffu, tl, i);
    if (lane == 0) ws.S[ti] += static_cast<double>(Oi);
  }
  __syncwarp();
}

}  // namespace

__global__ void __launch_bounds__(kLossThreads, 1) k_losses(const LossParams p) {
  __shared__ LossWarp lw[kLossThreads / 32];
  const uint32_t lane = lane_id();
  LossWarp& ws = lw[threadIdx.x >> 5];
  const bool diag = (p.diag_hits != nullptr) || (p.diag_hash != nullptr);
  const uint32_t lt_mask = (1u << lane) - 1u;
  unsigned long long n_nc = 0, n_slow = 0;
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
    const uint32_t n = __ldg(&p.tile_cnt[tile]);
    if (lane < static_cast<uint32_t>(ntr)) {
      ws.S[lane] = 0.0;
      ws.hits[lane] = 0ull;
      ws.hash[lane] = 0ull;
    }
    __syncwarp();
    int nd = 0;
    uint32_t base = 0;
    uint2 rec = make_uint2(0u, 0u);
    if (lane < n) rec = __ldcs(recs + lane);
    while (base < n) {
      const bool valid = base + lane < n;
      const uint32_t cnt = valid ? ((rec.x >> kRecCntShift) & 31u) + 1u : 0u;
      const uint32_t cincl = warp_inclusive_scan(cnt);
      const uint32_t take = __ballot_sync(0xffffffffu, valid && cincl <= 32u);
      const uint32_t n_take = __popc(take);  // a prefix: cincl grows with the lane
      const uint32_t np = __shfl_sync(0xffffffffu, cincl, n_take - 1);
      // lane -> event: event i starts at lane cincl_i - cnt_i
      uint32_t ev = lane;
      if (np != n_take) {
        const uint32_t starts = __reduce_or_sync(0xffffffffu, (lane < n_take) ? (1u << (cincl - cnt)) : 0u);
        ev = static_cast<uint32_t>(__popc(starts & ((lt_mask << 1) | 1u))) - 1u;
      }
      const uint32_t ekey = __shfl_sync(0xffffffffu, rec.x, ev);
      const uint32_t eps = __shfl_sync(0xffffffffu, rec.y, ev);
      const uint32_t estart = __shfl_sync(0xffffffffu, cincl - cnt, ev);
      const uint32_t etl = ekey >> kRecTrialShift, ek = ekey & kRecKMask;
      const bool pv = lane < np;
      float lv = 0.0f;
      bool slow = false;
      if (pv) {
        const Pair pr = p.pairs[eps + (lane - estart)];
        slow = !pair_fast(p, pr, ta + etl, ek, &lv);
        if (diag) {
          const uint32_t elt = static_cast<uint32_t>(p.elt_id[pair_pos(pr.meta)]);
          atomicAdd(&ws.hits[etl], 1ull);
          atomicAdd(&ws.hash[etl], static_cast<unsigned long long>(fmix64((static_cast<uint64_t>(ek) << 32) | elt)));
        }
      }
      n_pairs += pv ? 1u : 0u;
      // next window: starts after the events taken (prefetched now)
      const uint32_t nbase = base + n_take;
      uint2 nrec = make_uint2(0u, 0u);
      if (nbase + lane < n) nrec = __ldcs(recs + nbase + lane);
      // event sums, in lane (= layer) order
      const uint32_t eseg = pv ? ev : 0xFFFFu;
      float G = lv;
      uint32_t any_slow = slow ? 1u : 0u;
      if (np != n_take) {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const float g2 = __shfl_up_sync(0xffffffffu, G, d);
          const uint32_t s2 = __shfl_up_sync(0xffffffffu, eseg, d);
          const uint32_t f2 = __shfl_up_sync(0xffffffffu, any_slow, d);
          if (lane >= static_cast<uint32_t>(d) && s2 == eseg) {
            G += g2;
            any_slow |= f2;
          }
        }
      }
      const uint32_t eseg_next = __shfl_down_sync(0xffffffffu, eseg, 1);
      const bool ev_last = pv && (lane == np - 1 || eseg_next != eseg);
      const bool defer = ev_last && any_slow;
      const float O = (ev_last && !any_slow) ? clamp_terms_f(G, p.occ_r, p.occ_l) : 0.0f;
      const uint32_t dmask = __ballot_sync(0xffffffffu, defer);
      if (dmask) {
        if (nd + __popc(dmask) > 32) {
          resolve_deferred(p, ws, nd, ta, &n_nc, &n_slow);
          nd = 0;
        }
        if (defer) {
          const int at = nd + __popc(dmask & lt_mask);
          ws.d_key[at] = ekey;
          ws.d_ps[at] = eps;
        }
        nd += __popc(dmask);
        __syncwarp();
      }
      // trial sums: segmented double-float reduction by trial, one FP64 add per trial
      {
        float hi = O, lo = 0.0f;
        const uint32_t tseg = pv ? etl : 0xFFFFu;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const float h2 = __shfl_up_sync(0xffffffffu, hi, d);
          const float l2 = __shfl_up_sync(0xffffffffu, lo, d);
          const uint32_t s2 = __shfl_up_sync(0xffffffffu, tseg, d);
          if (lane >= static_cast<uint32_t>(d) && s2 == tseg) df_add(hi, lo, h2, l2);
        }
        const uint32_t tseg_next = __shfl_down_sync(0xffffffffu, tseg, 1);
        if (pv && (lane == np - 1 || tseg_next != tseg)) ws.S[etl] += static_cast<double>(hi) + static_cast<double>(lo);
        __syncwarp();
      }
      base = nbase;
      rec = nrec;
    }
    if (nd > 0) resolve_deferred(p, ws, nd, ta, &n_nc, &n_slow);
    if (lane < static_cast<uint32_t>(ntr)) {
      const int64_t o = ta + lane - p.t_begin;
      p.ylt[o] = clamp_terms_d(ws.S[lane], p.agg_r, p.agg_l);
      if (p.diag_hits) p.diag_hits[o] = static_cast<int64_t>(ws.hits[lane]);
      if (p.diag_hash) p.diag_hash[o] = ws.hash[lane];
    }
    __syncwarp();
  }
  n_pairs = __reduce_add_sync(0xffffffffu, n_pairs);
  for (int d = 16; d > 0; d >>= 1) {
    n_nc += __shfl_xor_sync(0xffffffffu, n_nc, d);
    n_slow += __shfl_xor_sync(0xffffffffu, n_slow, d);
  }
  if (lane == 0) {
    if (n_pairs) atomicAdd(&p.counters[1], static_cast<unsigned long long>(n_pairs));
    if (n_nc) atomicAdd(&p.counters[2], n_nc);
    if (n_slow) atomicAdd(&p.counters[3], n_slow);
  }
}

cudaError_t launch_losses(const LossParams& p, int grid, cudaStream_t s) {
  k_losses<<<grid, kLossThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ara
