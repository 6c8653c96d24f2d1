// Device arithmetic of the ARA hot path: the Philox uniform, the FP32
// inverse of the regularised incomplete Beta function, and the financial
// terms.  Everything here runs per (trial, event, ELT) pair on the GPU.
//
// Inverse Beta (Section 3.4: Loss = max_l * InvCDF_beta(z; alpha, beta)).
// The root x of I_x(a, b) = z is found in FP32 as the smaller of x and 1 - x
// (the side is chosen with the per-record value I_{1/2}(a, b)), so both ends
// keep relative precision.  Writing (A, B, P) for the oriented problem and r
// for its root, the iteration runs on u = ln r:
//   F(u)  = ln I_r(A, B) - ln P,
//   F'(u) = r pdf(r) / I = g,
//   F''/F' = A - (B - 1) r / (1 - r) - g,
// with Halley's correction and a bracket on r that falls back to geometric
// bisection.  ln of the front factor r^A (1-r)^B / B(A, B) is evaluated in the
// cancellation-free form C - A phi(t) - B phi(s), t = r/x0 - 1,
// s = (1-r)/y0 - 1, phi(t) = t - ln(1 + t), x0 = A/(A+B), y0 = B/(A+B), with
// the per-record constant C = A ln x0 + B ln y0 - ln B(A, B) precomputed in
// FP64 at load time.  I_r itself comes from the continued fraction of
// Abramowitz & Stegun 26.5.8 (modified Lentz), with the symmetry
// I_r(A, B) = 1 - I_{1-r}(B, A) past r = (A + 1)/(A + B + 2).  The starting
// point is Carter's normal approximation (Abramowitz & Stegun 26.5.22) for
// A, B >= 1 and the small-x / small-(1-x) power laws otherwise.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ara {

// ------------------------------------------------------------------ records
// One (event, ELT) pair of a layer, 32 bytes (one L2 sector).
enum : uint32_t {
  kKindBeta = 0u,  // Beta secondary uncertainty
  kKindMean = 1u,  // sigma == 0: the loss is the mean
  kKindZero = 2u,  // mean == 0: no loss
};

struct __align__(16) Pair {
  float a, b;     // Beta shapes (kKindBeta)
  float m0;       // min(x0, y0), x0 = a / (a + b), y0 = b / (a + b)
  float c;        // a ln x0 + b ln y0 - ln B(a, b)
  float max_l;    // exposure (maximum loss)
  float mu;       // mean loss
  float p_half;   // I_{1/2}(a, b)
  uint32_t meta;  // bits 0-4 layer position, 5-6 kind, 7: m0 is x0
};
static_assert(sizeof(Pair) == 32, "Pair must be one 32-byte sector");

__host__ __device__ inline uint32_t pair_pos(uint32_t meta) { return meta & 31u; }
__host__ __device__ inline uint32_t pair_kind(uint32_t meta) { return (meta >> 5) & 3u; }
__host__ __device__ inline bool pair_m0_is_x0(uint32_t meta) { return (meta >> 7) & 1u; }

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Uniform of (trial, event index k, ELT pool id): word 0 of the block with
// counter (trial mod 2^32, k, elt, trial >> 32) under key (seed_lo, seed_hi),
// mapped to ((w >> 9) + 1/2) 2^-23, a value in [2^-24, 1 - 2^-24] whose FP32
// representation and complement are exact.
__device__ __forceinline__ float philox_uniform(uint32_t seed_lo, uint32_t seed_hi, int64_t trial,
                                                uint32_t k, uint32_t elt) {
  const uint64_t t = static_cast<uint64_t>(trial);
  const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(t), k, elt, static_cast<uint32_t>(t >> 32)),
                                make_uint2(seed_lo, seed_hi));
  return (static_cast<float>(w.x >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
}

// ------------------------------------------------------------------ terms
__device__ __forceinline__ float clamp_terms_f(float l, float retention, float limit) {
  return fminf(fmaxf(l - retention, 0.0f), limit);
}
__device__ __forceinline__ double clamp_terms_d(double l, double retention, double limit) {
  return fmin(fmax(l - retention, 0.0), limit);
}

// ------------------------------------------------------------------ Beta
// phi(t) = t - ln(1 + t) for |t| <= 1/2, from ln(1 + t) = 2 atanh(q),
// q = t / (2 + t): phi = t^2 / (2 + t) - 2 q^3 (1/3 + q^2/5 + q^4/7 + ...).
__device__ __forceinline__ float phi_small(float t) {
  const float q = t / (2.0f + t);
  const float q2 = q * q;
  float s = 1.0f / 17.0f;
  s = fmaf(s, q2, 1.0f / 15.0f);
  s = fmaf(s, q2, 1.0f / 13.0f);
  s = fmaf(s, q2, 1.0f / 11.0f);
  s = fmaf(s, q2, 1.0f / 9.0f);
  s = fmaf(s, q2, 1.0f / 7.0f);
  s = fmaf(s, q2, 1.0f / 5.0f);
  s = fmaf(s, q2, 1.0f / 3.0f);
  return t * t / (2.0f + t) - 2.0f * q * q2 * s;
}

// ln(r^A (1 - r)^B / B(A, B)) = C - A phi(r/x0 - 1) - B phi((1-r)/y0 - 1).
__device__ __forceinline__ float beta_log_front(float r, float A, float B, float x0, float y0, float C) {
  const float d = r - x0;
  const float t = d / x0;
  const float s = -d / y0;
  const float pt = (fabsf(t) <= 0.5f) ? phi_small(t) : (t - logf(r / x0));
  const float ps = (fabsf(s) <= 0.5f) ? phi_small(s) : (s - logf((1.0f - r) / y0));
  return C - A * pt - B * ps;
}

// 1 / K with K = 1 + d1/(1 + d2/(1 + ...)), the continued fraction of
// I_x(A, B) = x^A (1-x)^B / (A B(A, B)) / K (A&S 26.5.8), modified Lentz.
// Returns the number of partial fractions used through *terms.
__device__ __forceinline__ float beta_cf(float A, float B, float x, int max_terms, int* terms) {
  const float tiny = 1e-30f;
  float K = 1.0f, Cl = 1.0f, D = 0.0f;
  int m = 1;
  for (; m <= max_terms; ++m) {
    const float h = static_cast<float>(m >> 1);
    float num;
    if (m & 1) {
      num = -(A + h) * (A + B + h) * x / ((A + 2.0f * h) * (A + 2.0f * h + 1.0f));
    } else {
      num = h * (B - h) * x / ((A + 2.0f * h - 1.0f) * (A + 2.0f * h));
    }
    D = fmaf(num, D, 1.0f);
    if (fabsf(D) < tiny) D = tiny;
    Cl = 1.0f + num / Cl;
    if (fabsf(Cl) < tiny) Cl = tiny;
    D = 1.0f / D;
    const float delta = Cl * D;
    K *= delta;
    if (fabsf(delta - 1.0f) < 2.4e-7f) break;
  }
  *terms = m;
  return 1.0f / K;
}

struct BetaSolveStats {
  int iters;
  int cf_terms;
  bool converged;
};

// Root r of I_r(A, B) = P, r expected in (0, ~1/2].  lnA = ln A,
// lnP = ln P; x0 = A/(A+B), y0 = B/(A+B); C as above.
__device__ __forceinline__ float beta_solve_oriented(float A, float B, float x0, float y0, float C, float P,
                                                     BetaSolveStats* st) {
  const float lnP = logf(P);
  const float lnA = logf(A);
  // ------------------------------------------------------------ start point
  float r;
  if (A >= 1.0f && B >= 1.0f) {
    // Carter (A&S 26.5.22): y is the upper-tail normal deviate of P
    const float y = -normcdfinvf(P);
    const float lam = (y * y - 3.0f) * (1.0f / 6.0f);
    const float ia = 1.0f / (2.0f * A - 1.0f), ib = 1.0f / (2.0f * B - 1.0f);
    const float h = 2.0f / (ia + ib);
    const float w = y * sqrtf(h + lam) / h - (ib - ia) * (lam + 5.0f / 6.0f - 2.0f / (3.0f * h));
    r = A / (A + B * expf(2.0f * w));
  } else {
    // power laws at the two ends: I ~ r^A / (A B(A,B)) and 1 - I ~ (1-r)^B / (B B(A,B))
    const float lnB = A * logf(x0) + B * logf(y0) - C;
    const float rl = expf((lnP + lnA + lnB) / A);
    if (rl < x0) {
      r = rl;
    } else {
      const float ru = 1.0f - expf((log1pf(-P) + logf(B) + lnB) / B);
      r = (ru > x0 && ru < 1.0f) ? ru : x0;
    }
  }
  if (!(r > 0.0f) || !(r < 1.0f)) r = x0;
  if (r < 1e-37f) r = 1e-37f;
  // ------------------------------------------------------------ Halley on ln r
  float rlo = 0.0f, rhi = 1.0f;
  const float switch_x = (A + 1.0f) / (A + B + 2.0f);
  int it = 0, cf_total = 0;
  bool done = false;
  for (; it < 48; ++it) {
    const float L = beta_log_front(r, A, B, x0, y0, C);
    int terms = 0;
    float F, g;
    if (r < switch_x) {
      const float cf = beta_cf(A, B, r, 256, &terms);
      F = L - lnA + logf(cf) - lnP;
      g = A / ((1.0f - r) * cf);
    } else {
      const float cf = beta_cf(B, A, 1.0f - r, 256, &terms);
      const float eL = expf(L);
      const float J = eL * cf / B;  // 1 - I
      F = log1pf(-J) - lnP;
      g = eL / ((1.0f - r) * (1.0f - J));
    }
    cf_total += terms;
    if (F < 0.0f) rlo = r; else rhi = r;
    if (F == 0.0f) { done = true; ++it; break; }
    const float newton = -F / g;
    const float curv = A - (B - 1.0f) * r / (1.0f - r) - g;
    const float denom = fmaf(0.5f * newton, curv, 1.0f);
    float du = (denom > 0.5f && denom < 2.0f) ? newton / denom : newton;
    du = fminf(fmaxf(du, -80.0f), 80.0f);
    float rn = r * expf(du);
    bool bisect = false;
    if (!(rn > rlo && rn < rhi)) {
      const float lo = fmaxf(rlo, 1e-37f);
      rn = (rhi > 4.0f * lo) ? sqrtf(lo) * sqrtf(rhi) : 0.5f * (rlo + rhi);
      bisect = true;
    }
    if (!bisect && fabsf(du) < 4e-4f) { r = rn; done = true; ++it; break; }
    if (rn == r) { done = true; ++it; break; }
    r = rn;
    if (rhi <= 1e-37f) { done = true; ++it; break; }  // root below the FP32 normal range
  }
  st->iters = it;
  st->cf_terms = cf_total;
  st->converged = done;
  return r;
}

// Loss of one pair: max_l * InvCDF(z; a, b) for Beta records, the mean for
// sigma == 0 records (and for every record when primary_only), 0 for
// mean == 0 records.
__device__ __forceinline__ float pair_loss(const Pair& p, float z, bool primary_only, BetaSolveStats* st) {
  const uint32_t kind = pair_kind(p.meta);
  st->iters = 0;
  st->cf_terms = 0;
  st->converged = true;
  if (kind == kKindZero) return 0.0f;
  if (primary_only || kind == kKindMean) return p.mu;
  const bool m0x = pair_m0_is_x0(p.meta);
  const float x0 = m0x ? p.m0 : 1.0f - p.m0;
  const float y0 = m0x ? 1.0f - p.m0 : p.m0;
  if (z <= p.p_half) {
    const float r = beta_solve_oriented(p.a, p.b, x0, y0, p.c, z, st);
    return p.max_l * r;
  }
  // root above 1/2: 1 - x solves I_{1-x}(b, a) = 1 - z (exact in FP32)
  const float r = beta_solve_oriented(p.b, p.a, y0, x0, p.c, 1.0f - z, st);
  return p.max_l * (1.0f - r);
}

// fmix64 finaliser (MurmurHash3), for the order-free hit-list checksum.
__device__ __forceinline__ uint64_t fmix64(uint64_t v) {
  v ^= v >> 33;
  v *= 0xff51afd7ed558ccdull;
  v ^= v >> 33;
  v *= 0xc4ceb9fe1a85ec53ull;
  v ^= v >> 33;
  return v;
}

}  // namespace ara
