// Kernels of the ARA engine outside the layer's hot loop: input checks and
// per-record preparation at load time, the quantile tables, the check kernels,
// the scan and the per-layer event index.  The two layer kernels are in
// ara_layer.cu.
#include <cuda_runtime.h>

#include <cstdint>

#include "ara_df.cuh"
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

// The YET upload from pinned host memory: each thread moves int4 groups of
// ids (four groups in flight) when the source is 16-byte aligned, single ids
// otherwise, and flags any id outside [0, catalogue).  A few blocks keep
// enough reads in flight to fill the host link.
constexpr int kUploadBlocks = 32;
constexpr int kUploadThreads = 512;

__device__ __forceinline__ bool id_bad(int32_t e, uint32_t cat) { return static_cast<uint32_t>(e) >= cat; }

__global__ void __launch_bounds__(kUploadThreads) k_upload_ids(const int32_t* __restrict__ src,
                                                               int32_t* __restrict__ dst, int64_t n,
                                                               int32_t catalogue, uint32_t* flags) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint32_t cat = static_cast<uint32_t>(catalogue);
  bool bad = false;
  int64_t k0 = 0;  // first id of the single-id tail
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    const int4* s4 = reinterpret_cast<const int4*>(src);
    int4* d4 = reinterpret_cast<int4*>(dst);
    const int64_t n4 = n >> 2;
    int64_t i = tid;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      int4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = s4[i + j * stride];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        d4[i + j * stride] = v[j];
        bad |= id_bad(v[j].x, cat) | id_bad(v[j].y, cat) | id_bad(v[j].z, cat) | id_bad(v[j].w, cat);
      }
    }
    for (; i < n4; i += stride) {
      const int4 v = s4[i];
      d4[i] = v;
      bad |= id_bad(v.x, cat) | id_bad(v.y, cat) | id_bad(v.z, cat) | id_bad(v.w, cat);
    }
    k0 = 4 * n4;
  }
  for (int64_t k = k0 + tid; k < n; k += stride) {
    const int32_t e = src[k];
    dst[k] = e;
    bad |= id_bad(e, cat);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kBadEventId);
}

cudaError_t launch_upload_ids(const int32_t* src, int32_t* dst, int64_t n, int32_t catalogue, uint32_t* flags,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_upload_ids<<<kUploadBlocks, kUploadThreads, 0, s>>>(src, dst, n, catalogue, flags);
  return cudaGetLastError();
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
__device__ double beta_cf_f64_ref(double a, double b, double x) {
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

// The continued fraction of beta_cf_f64_ref in double-float arithmetic, two
// terms (the odd and the even one of each m) per iteration: FP64 runs at a
// small fraction of the FP32 rate on this GPU, and 48 bits carry the value to
// the 1e-13 relative tolerance used here (the table nodes are FP32; their
// polish and check need the CDF to about 1e-10).  FP32's exponent range is
// kept by rescaling the four convergents by a power of two each iteration
// (exact; the ratio is unchanged).  Returns NaN when a value leaves the FP32
// range or the iteration does not converge, for the FP64 fallback.
__device__ double beta_cf_df(double a, double b, double x) {
  const DF X = df_of(x);
  DF v = df_of(a);          // a + m
  DF w = df_of(a + b);      // a + b + m
  DF y = df_of(b - 1.0);    // b - m - 1
  DF u = df_of(a);          // a + 2m
  DF A2{1.0f, 0.0f}, B2{0.0f, 0.0f}, A1{1.0f, 0.0f}, B1{1.0f, 0.0f};
  DF q_prev{1.0f, 0.0f};
  double f_prev = 1.0;
  for (int m = 0; m < 20000; ++m) {
    const DF u1 = df_add_f(u, 1.0f), u2 = df_add_f(u, 2.0f);
    // odd term n = 2m + 1: p = -(a + m)(a + b + m) x, q = (a + 2m)(a + 2m + 1)
    const DF qo = df_mul(u, u1);
    const DF ao = df_mul(q_prev, df_neg(df_mul(df_mul(v, w), X)));
    DF A0 = df_add(df_mul(qo, A1), df_mul(ao, A2));
    DF B0 = df_add(df_mul(qo, B1), df_mul(ao, B2));
    // even term n = 2m + 2: p = (m + 1)(b - m - 1) x, q = (a + 2m + 1)(a + 2m + 2)
    const DF qe = df_mul(u1, u2);
    const DF ae = df_mul(qo, df_mul(df_mul(DF{static_cast<float>(m + 1), 0.0f}, y), X));
    const DF Ae = df_add(df_mul(qe, A0), df_mul(ae, A1));
    const DF Be = df_add(df_mul(qe, B0), df_mul(ae, B1));
    A2 = A0;
    B2 = B0;
    A1 = Ae;
    B1 = Be;
    q_prev = qe;
    v = df_add_f(v, 1.0f);
    w = df_add_f(w, 1.0f);
    y = df_add_f(y, -1.0f);
    u = u2;
    const float big = fmaxf(fabsf(A1.hi), fabsf(B1.hi));
    if (!(big < 3.0e38f) || !(big > 0.0f)) return __longlong_as_double(0x7ff8000000000000ll);
    const int k = -f_exponent(big);
    A1 = df_scale(A1, k);
    A2 = df_scale(A2, k);
    B1 = df_scale(B1, k);
    B2 = df_scale(B2, k);
    if ((m & 3) == 3) {
      const double f = df_val(A1) / df_val(B1);
      if (fabs(f - f_prev) <= 1e-13 * fabs(f)) return df_val(B1) / df_val(A1);
      f_prev = f;
    }
  }
  return __longlong_as_double(0x7ff8000000000000ll);
}

// The continued fraction of I_x(a, b): double-float, else FP64.
__device__ double beta_cf_f64(double a, double b, double x) {
  const double r = beta_cf_df(a, b, x);
  return isfinite(r) ? r : beta_cf_f64_ref(a, b, x);
}

}  // namespace

// Section 3.3 per record: sigma_b = sigma / max_l, mu_b = mu / max_l,
// sigma_bmax = sqrt(mu_b (1 - mu_b)), sigma_b clipped to (1 - 1e-6) sigma_bmax,
// alpha = mu_b ((sigma_bmax / sigma_b)^2 - 1), beta = (1 - mu_b)(...).  With a
// correlated part sigma_C (Section 3.1), sigma = sigma_I + sigma_C
// (Section 3.2 step i) and a record with sigma_C > 0 is of kind kKindBetaC,
// with weights (sigma_I, sigma_C) / sqrt(sigma_I^2 + sigma_C^2) for the
// combination of its two normal variables.
__global__ void k_prepare_records(const int32_t* events, const float* mean, const float* sigma,
                                  const float* exposure, int64_t n, Pair* out, BetaShape* shapes, uint32_t* flags,
                                  int32_t* max_event, uint32_t* max_loss, const float* sigma_c, float2* weights) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t f = 0;
  int32_t emax = -1;
  float lmax = 0.0f;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int32_t e = events[i];
    emax = max(emax, e);
    if (e < 0) f |= kBadEventId;
    if (i > 0 && events[i - 1] >= e) f |= kBadOrder;
    const double mu = mean[i], si = sigma[i], ex = exposure[i];
    const double sc = sigma_c ? static_cast<double>(sigma_c[i]) : 0.0;
    const double sg = si + sc;
    Pair p;
    p.a = p.b = p.m0 = p.c = p.p_half = 0.0f;
    p.max_l = static_cast<float>(ex);
    p.mu = static_cast<float>(mu);
    uint32_t kind = kKindBeta;
    double sa = 0.0, sb_ = 0.0, slnb = 0.0;
    float2 w = make_float2(1.0f, 0.0f);
    if (!(mu >= 0.0) || !(si >= 0.0) || !(sc >= 0.0) || !isfinite(mu) || !isfinite(sg) || !isfinite(ex)) {
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
      slnb = lnB;
      p.m0 = (x0 <= y0) ? -static_cast<float>(x0) : static_cast<float>(y0);
      p.c = static_cast<float>(c);
      p.p_half = static_cast<float>(ph);
      if (sc > 0.0) {
        kind = kKindBetaC;
        f |= kHasCorrelated;
        const double nrm = sqrt(si * si + sc * sc);
        w = make_float2(static_cast<float>(si / nrm), static_cast<float>(sc / nrm));
      }
    }
    p.meta = (kind << kMetaKindShift) | (static_cast<uint32_t>(i) << kMetaRecShift);
    if (kind != kKindZero) lmax = fmaxf(lmax, fmaxf(p.max_l, p.mu));
    out[i] = p;
    if (shapes) shapes[i] = BetaShape{sa, sb_, slnb, 0.0};
    if (weights) weights[i] = w;
  }
  if (f) atomicOr(flags, f);
  // block max of event ids, then one atomic per warp
  for (int d = 16; d > 0; d >>= 1) {
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, d));
    lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, d));
  }
  if ((threadIdx.x & 31) == 0 && emax >= 0) atomicMax(max_event, emax);
  // non-negative floats order as their bit patterns
  if ((threadIdx.x & 31) == 0 && max_loss && lmax > 0.0f) atomicMax(max_loss, __float_as_uint(lmax));
}

cudaError_t launch_prepare_records(const int32_t* events, const float* mean, const float* sigma,
                                   const float* exposure, int64_t n, Pair* out, BetaShape* shapes, uint32_t* flags,
                                   int32_t* max_event, uint32_t* max_loss, cudaStream_t s, const float* sigma_c,
                                   float2* weights) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 127) / 128;
  k_prepare_records<<<static_cast<int>(blocks < 65535 ? blocks : 65535), 128, 0, s>>>(
      events, mean, sigma, exposure, n, out, shapes, flags, max_event, max_loss, sigma_c, weights);
  return cudaGetLastError();
}

// =============================================================== quantile tables (FP64, load time)
namespace {

// I_x(a, b) and 1 - I_x(a, b), each without cancellation (A&S 26.5.8 with
// symmetry).  *front_out (optional) receives x^a (1-x)^b / B(a, b), which is
// x (1 - x) f(x) for the Beta density f.
__device__ void beta_inc_pair_f64(double x, double a, double b, double lnB, double* I, double* Ic,
                                  double* front_out = nullptr) {
  if (!(x > 0.0)) {
    *I = 0.0;
    *Ic = 1.0;
    if (front_out) *front_out = 0.0;
    return;
  }
  if (!(x < 1.0)) {
    *I = 1.0;
    *Ic = 0.0;
    if (front_out) *front_out = 0.0;
    return;
  }
  const double front = exp(a * log(x) + b * log1p(-x) - lnB);
  if (front_out) *front_out = front;
  // the fraction on the side where it converges fast: the side is chosen per
  // lane and the fraction called once, so that the lanes of a warp do not
  // run it twice
  const bool lower = x < (a + 1.0) / (a + b + 2.0);
  const double p = lower ? a : b, q = lower ? b : a, y = lower ? x : 1.0 - x;
  const double v = front * beta_cf_f64(p, q, y) / p;
  *I = lower ? v : 1.0 - v;
  *Ic = lower ? 1.0 - v : v;
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
// FP64, where I ~ r^A near 0 makes the step almost exact.  The seed is good to
// ~1e-6, so a step |du| < 1e-5 leaves an error of order du^2 (~1e-10, below
// the FP32 resolution of the stored node) and ends the iteration; at most 3
// steps.  A seed that does not converge goes to the bracketed solver.
__device__ double beta_polish_f64(double p, double A, double B, double lnB, double seed) {
  double r = seed;
  if (!(r > 0.0 && r < 1.0)) return beta_root_f64(p, A, B, lnB, -1.0);
  for (int it = 0; it < 3; ++it) {
    double I, Ic, front;
    beta_inc_pair_f64(r, A, B, lnB, &I, &Ic, &front);
    if (!(I > 0.0) || !(front > 0.0)) return beta_root_f64(p, A, B, lnB, seed);
    const double g = front / ((1.0 - r) * I);  // d ln I / d ln r = r f(r) / I
    const double du = -log1p((I - p) / p) / g;
    if (!(fabs(du) < 0.5)) return beta_root_f64(p, A, B, lnB, seed);
    const double rn = fma(r, expm1(du), r);
    if (!(rn > 0.0 && rn < 1.0)) return beta_root_f64(p, A, B, lnB, seed);
    r = rn;
    if (fabs(du) < 1e-5) return r;
  }
  return beta_root_f64(p, A, B, lnB, r);
}

}  // namespace

// One node of a record's quantile table at t: the FP64 root x (seeded by the
// FP32 Halley solver), w = ln x, and the derivatives in t, w' = phi(t) / (x f(x))
// and w'' = w' (-t - w' (a - (b-1) x/(1-x))).  Returns {x, 0, h w', h^2 w''}
// (the caller fills in w_{j+1} - w_j) and w.
__device__ float4 table_node(const Pair& pr, double a, double b, double lnB, double t, double h, double* w_out) {
  const double zl = normcdf(-fabs(t));  // the smaller tail probability
  // FP32 seed, then FP64 polish on the side where the root keeps relative precision
  BetaSolveStats st;
  const float zf = (t <= 0.0) ? static_cast<float>(zl) : static_cast<float>(1.0 - zl);
  const float seed = pair_quantile_newton(pr, fminf(fmaxf(zf, 5.9604645e-08f), 0.99999994f), -1.0f, &st);
  // the root x (t <= 0) or y = 1 - x (t > 0): the shapes are swapped per lane
  // and the polish called once (ln B is symmetric), so that the two halves of
  // the warp do not run it in turn
  const bool lo = t <= 0.0;
  const double r = beta_polish_f64(zl, lo ? a : b, lo ? b : a, lnB,
                                   lo ? static_cast<double>(seed) : 1.0 - static_cast<double>(seed));
  const double l_r = log(r), l_1mr = log1p(-r);
  const double w = lo ? l_r : l_1mr;
  const double lny = lo ? l_1mr : l_r;
  const double lpdf = (a - 1.0) * w + (b - 1.0) * lny - lnB;
  const double lphi = -0.5 * t * t - 0.91893853320467274178;
  const double D = exp(lphi - w - lpdf);
  const double E = D * (-t - D * (a - (b - 1.0) * exp(w - lny)));
  *w_out = w;
  return make_float4(static_cast<float>(exp(w)), 0.0f, static_cast<float>(h * D), static_cast<float>(h * h * E));
}

// Accuracy of the segment [t, t + h] of a table (node nd = {x, dw, h w', h^2 w''}
// at t; d1, e1 the derivative terms of the next node), checked at the midpoint,
// where the error kernel s^3 (1-s)^3 of quintic Hermite interpolation peaks:
// the FP32 interpolant (as the hot path evaluates it) against the FP64 CDF.
// True when the implied relative error of x there is within kTabTol (a bound
// set by the FP32 evaluation of the interpolant, ~2e-7, more than by the
// interpolation error, which elsewhere in the segment is below its midpoint
// value), or x < 1e-30 (negligible losses).
__device__ bool table_segment_ok(float4 nd, float d1, float e1, double t, double h, double a, double b, double lnB) {
  if (!(isfinite(nd.x) && isfinite(nd.y) && isfinite(nd.z) && isfinite(nd.w))) return false;
  const float xq = (nd.x > 0.0f) ? nd.x * expf(tab_increment(0.5f, nd.y, nd.z, nd.w, d1, e1)) : 0.0f;
  if (!(xq >= 1e-30f)) return true;
  const double tq = t + 0.5 * h;
  const double zq = normcdf(-fabs(tq));
  double I, Ic, front, rel;
  if (xq >= 1.0f) {
    // the FP32 ceiling: fine iff the quantile itself is within 2^-24 of 1
    beta_inc_pair_f64(1.0 - 5.9604644775390625e-08, a, b, lnB, &I, &Ic);
    rel = (tq > 0.0 && Ic >= zq) ? 0.0 : INFINITY;
  } else {
    const double xd = static_cast<double>(xq);
    beta_inc_pair_f64(xd, a, b, lnB, &I, &Ic, &front);
    const double err_z = (tq <= 0.0) ? (I - zq) : (Ic - zq);
    rel = fabs(err_z) * (1.0 - xd) / front;  // |dz| / (x f(x))
  }
  return (rel <= kTabTol) && isfinite(rel);
}

// Coarse tables, one warp per record, lane j = node j at t_j = -T1 + j h.  The
// stored float4 is {x_j, w_{j+1} - w_j, h w'_j, h^2 w''_j}.  need[rec] = 1 for
// a Beta record whose coarse table is not exact (a candidate for a fine table).
__global__ void __launch_bounds__(256, 2) k_build_tables(Pair* recs, const BetaShape* shapes, int64_t n, float4* tab,
                                                        uint32_t* need) {
  const int lane = threadIdx.x & 31;
  const int64_t rec = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (rec >= n) return;
  const Pair pr = recs[rec];
  float4* out = tab + rec * kTabNodes;
  if (!kind_is_beta(pair_kind(pr.meta))) {
    out[lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (lane == 0) need[rec] = 0u;
    return;
  }
  const double a = shapes[rec].a, b = shapes[rec].b, lnB = shapes[rec].lnB;
  const double h = 2.0 * kTabT1 / (kTabNodes - 1);
  const double t = -kTabT1 + h * lane;
  double w;
  float4 node = table_node(pr, a, b, lnB, t, h, &w);
  const double w_next = __shfl_down_sync(0xffffffffu, w, 1);
  if (lane < kTabNodes - 1) node.y = static_cast<float>(w_next - w);
  out[lane] = node;
  const float d1 = __shfl_down_sync(0xffffffffu, node.z, 1);
  const float e1 = __shfl_down_sync(0xffffffffu, node.w, 1);
  const bool ok = (lane < kTabNodes - 1) ? table_segment_ok(node, d1, e1, t, h, a, b, lnB)
                                         : (isfinite(node.x) && isfinite(node.z) && isfinite(node.w));
  const bool all_ok = __all_sync(0xffffffffu, ok);
  if (lane == 0) {
    if (all_ok) recs[rec].meta = pr.meta | (1u << kMetaExactBit);
    need[rec] = all_ok ? 0u : 1u;
  }
}

// Fine tables: global block b is slot b - slot_begin of the job (ELT) whose
// slot range holds b, for that job's (b - slot_begin)-th candidate in record
// order (slot = exclusive prefix of its need flags); thread j = node j at
// t_j = -T1 + j h / kTabRefine.  The record's meta then addresses its fine
// table (by the ELT-local slot); it is table-exact if the fine table passes
// the check.
__global__ void __launch_bounds__(kTabFineStride) k_build_fine(Pair* recs, const BetaShape* shapes,
                                                              const FineJob* jobs, int n_jobs, float4* tabf) {
  __shared__ double s_w[kTabFineStride];
  __shared__ float4 s_node[kTabFineStride];
  __shared__ int64_t s_rec;
  __shared__ uint32_t s_ls;
  const int64_t gb = blockIdx.x;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n_jobs - 1;  // the last job with slot_begin <= gb
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].slot_begin <= gb) lo = mid; else hi = mid - 1;
    }
    const FineJob jb = jobs[lo];
    const uint32_t ls = static_cast<uint32_t>(gb - jb.slot_begin);
    int64_t rec = -1;
    if (jb.n > 0 && ls < jb.cap && ls < jb.slot[jb.n]) {
      int64_t l = 0, h = jb.n - 1;  // the first r with slot[r + 1] > ls
      while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (jb.slot[mid + 1] > ls) h = mid; else l = mid + 1;
      }
      rec = jb.rec_begin + l;
    }
    s_rec = rec;
    s_ls = ls;
  }
  __syncthreads();
  const int64_t rec = s_rec;
  if (rec < 0) return;
  const uint32_t ls = s_ls;
  const Pair pr = recs[rec];
  const double a = shapes[rec].a, b = shapes[rec].b, lnB = shapes[rec].lnB;
  const double h = 2.0 * kTabT1 / (kTabFineNodes - 1);
  const int j = threadIdx.x;
  const double t = -kTabT1 + h * (j < kTabFineNodes ? j : kTabFineNodes - 1);
  double w = 0.0;
  float4 node = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (j < kTabFineNodes) node = table_node(pr, a, b, lnB, t, h, &w);
  s_w[j] = w;
  s_node[j] = node;
  __syncthreads();
  bool ok = true;
  if (j < kTabFineNodes - 1) {
    node.y = static_cast<float>(s_w[j + 1] - w);
    ok = table_segment_ok(node, s_node[j + 1].z, s_node[j + 1].w, t, h, a, b, lnB);
  } else if (j == kTabFineNodes - 1) {
    ok = isfinite(node.x) && isfinite(node.z) && isfinite(node.w);
  }
  if (j < kTabFineNodes) tabf[gb * kTabFineStride + j] = node;
  const bool all_ok = __syncthreads_and(ok) != 0;
  if (j == 0)
    recs[rec].meta = (pr.meta & ((1u << kMetaFineBit) - 1u)) | (1u << kMetaFineBit) |
                     (all_ok ? (1u << kMetaExactBit) : 0u) | (ls << kMetaRecShift);
}

size_t build_tables_work_words(int64_t n) {
  // need/slot (n + 1), scan scratch, then room for one 16-byte aligned FineJob
  return static_cast<size_t>(n) + 1 + scan_tmp_words(n + 1) + (sizeof(FineJob) + 16) / sizeof(uint32_t);
}

uint32_t fine_table_cap(int64_t n) {
  const int64_t cap = n / 16 + 16;
  return static_cast<uint32_t>(cap < n ? cap : n);
}

cudaError_t launch_build_coarse(Pair* recs, const BetaShape* shapes, int64_t n, float4* tab, uint32_t* need,
                                cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 7) / 8;  // 8 warps (records) per block
  k_build_tables<<<static_cast<int>(blocks < 2147483647 ? blocks : 2147483647), 256, 0, s>>>(recs, shapes, n, tab,
                                                                                          need);
  return cudaGetLastError();
}

cudaError_t launch_build_fine_jobs(Pair* recs, const BetaShape* shapes, const FineJob* jobs, int n_jobs,
                                   int64_t total_slots, float4* tabf, cudaStream_t s) {
  if (n_jobs == 0 || total_slots == 0) return cudaSuccess;
  k_build_fine<<<static_cast<int>(total_slots), kTabFineStride, 0, s>>>(recs, shapes, jobs, n_jobs, tabf);
  return cudaGetLastError();
}

// One ELT: its scan, then its fine tables (a one-job launch; the job record
// sits after the scan's scratch in `work`).
cudaError_t launch_build_fine(Pair* recs, const BetaShape* shapes, int64_t n, const uint32_t* need, float4* tabf,
                              uint32_t* work, cudaStream_t s, int* n_launch) {
  if (n == 0) return cudaSuccess;
  int launched = 0;
  cudaError_t err = scan_exclusive_u32(need, work, n, work + n + 1, s, &launched);
  if (err != cudaSuccess) return err;
  FineJob jb{0, n, work, 0, fine_table_cap(n), 0};
  FineJob* d_job = reinterpret_cast<FineJob*>(
      (reinterpret_cast<uintptr_t>(work + n + 1 + scan_tmp_words(n + 1)) + 15) & ~uintptr_t(15));
  if ((err = cudaMemcpyAsync(d_job, &jb, sizeof(FineJob), cudaMemcpyHostToDevice, s)) != cudaSuccess) return err;
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;  // jb lives on this stack frame
  if ((err = launch_build_fine_jobs(recs, shapes, d_job, 1, jb.cap, tabf, s)) != cudaSuccess) return err;
  if (n_launch) *n_launch += launched + 1;
  return cudaSuccess;
}

cudaError_t launch_build_tables(Pair* recs, const BetaShape* shapes, int64_t n, float4* tab, float4* tabf,
                                uint32_t* work, cudaStream_t s, int* n_launch) {
  if (n == 0) return cudaSuccess;
  cudaError_t err = launch_build_coarse(recs, shapes, n, tab, work, s);
  if (err != cudaSuccess) return err;
  if (n_launch) *n_launch += 1;
  return launch_build_fine(recs, shapes, n, work, tabf, work, s, n_launch);
}

// =============================================================== check kernels
__global__ void k_debug_uniforms(uint32_t seed_lo, uint32_t seed_hi, int64_t n, const int64_t* trials,
                                 const int32_t* ks, const int32_t* elts, float* out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    out[i] = philox_uniform(seed_lo, seed_hi, trials[i], static_cast<uint32_t>(ks[i]), static_cast<uint32_t>(elts[i]));
}

__global__ void k_debug_losses(const Pair* recs, const float4* tab, const float4* tabf, const float* z, int64_t n,
                               int newton_only, float* out, int32_t* iters) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    BetaSolveStats st;
    const Pair pr = recs[i];
    const int64_t r = pair_rec(pr.meta);
    const float4* tb = pair_fine(pr.meta) ? tabf + r * kTabFineStride : tab + r * kTabNodes;
    out[i] = pair_loss(pr, z[i], false, tb, newton_only != 0, &st);
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

cudaError_t launch_debug_losses(const Pair* recs, const float4* tab, const float4* tabf, const float* z, int64_t n,
                                int newton_only, float* out, int32_t* iters, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t b = (n + 127) / 128;
  k_debug_losses<<<static_cast<int>(b < 65535 ? b : 65535), 128, 0, s>>>(recs, tab, tabf, z, n, newton_only, out,
                                                                         iters);
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

__global__ void k_mark_positions(LayerEltRefs r, const uint32_t* bits, const uint32_t* slot_base,
                                 unsigned long long* mask) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int32_t e = r.events[p][i - r.rec_begin[p]];
    atomicOr(&mask[rank_of(bits, slot_base, e)], 1ull << p);
  }
}

__global__ void k_slot_counts(const unsigned long long* mask, int64_t n, uint32_t* cnt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
    cnt[i] = __popcll(mask[i]);
}

__global__ void k_fill_pairs(LayerEltRefs r, const uint32_t* bits, const uint32_t* slot_base,
                             const unsigned long long* mask,
                             const uint32_t* slot_start, Pair* pairs, PairHot* hot, float2* pw, int32_t* pev) {
  const int64_t n = r.rec_begin[r.n_elts];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const int p = find_pos(r, i);
    const int64_t j = i - r.rec_begin[p];
    const int32_t e = r.events[p][j];
    const uint32_t slot = rank_of(bits, slot_base, e);
    const uint32_t within = __popcll(mask[slot] & ((1ull << p) - 1ull));
    Pair q = r.recs[p][j];
    q.meta = (q.meta & ~kMetaPosMask) | static_cast<uint32_t>(p);
    const uint32_t at = slot_start[slot] + within;
    pairs[at] = q;
    PairHot hq;
    hq.max_l = q.max_l;
    hq.mu = q.mu;
    hq.meta = q.meta;
    hq.node = pair_rec(q.meta) * (pair_fine(q.meta) ? kTabFineStride : kTabNodes);
    hot[at] = hq;
    if (pw && r.wts[p]) pw[at] = r.wts[p][j];
    if (pev) pev[at] = e;
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
  if ((err = cudaMemsetAsync(ix.mask, 0, sizeof(unsigned long long) * (n_recs > 0 ? n_recs : 1), s)) !=
      cudaSuccess)
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
    k_fill_pairs<<<grid_for(n_recs, 256), 256, 0, s>>>(refs, ix.bits, ix.word_cnt, ix.mask, ix.slot_cnt, ix.pairs, ix.hot,
                                                        ix.pw, ix.pev);
    launched += 3;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  } else {
    if ((err = cudaMemsetAsync(ix.slot_cnt, 0, sizeof(uint32_t), s)) != cudaSuccess) return err;
  }
  if (n_launch) *n_launch += launched;
  return cudaSuccess;
}

}  // namespace ara
