// Device arithmetic of the ARA hot path: the Philox uniform, the FP32
// inverse of the regularised incomplete Beta function, and the financial
// terms.  Everything here runs per (trial, event, ELT) pair on the GPU.
//
// Inverse Beta (Section 3.3: Loss = max_l * InvCDF_beta(z; alpha, beta)).
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
//
// Quantile tables.  Each record also carries a table of its quantile built in
// FP64 at load time: kTabNodes nodes uniform in t = Phi^-1(z) over
// [Phi^-1(2^-24), Phi^-1(1 - 2^-24)] (the whole range of the uniform grid),
// with w = ln x, dw/dt and d2w/dt2 at each node.  Between nodes w follows the
// quintic Hermite interpolant, evaluated as x = x_i exp(w - w_i) so that x
// keeps FP32 relative precision.  Records whose table reproduces the FP64
// quantile to kTabTol (checked at load at three points per segment) use the
// table alone; the others start the Halley iteration from the table's value.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ara {

// ------------------------------------------------------------------ records
// One (event, ELT) pair of a layer, 32 bytes (one L2 sector).
enum : uint32_t {
  kKindBeta = 0u,   // Beta secondary uncertainty, uniform z_(Prog,E)
  kKindBetaC = 1u,  // Beta secondary uncertainty with a correlated sigma_C > 0 (Section 3.2 uniform)
  kKindMean = 2u,   // sigma == 0: the loss is the mean
  kKindZero = 3u,   // mean == 0: no loss
};

struct __align__(16) Pair {
  float a, b;     // Beta shapes (kKindBeta)
  float m0;       // min(x0, y0), x0 = a / (a + b), y0 = b / (a + b); negative when it is x0
  float c;        // a ln x0 + b ln y0 - ln B(a, b)
  float max_l;    // exposure (maximum loss)
  float mu;       // mean loss
  float p_half;   // I_{1/2}(a, b)
  uint32_t meta;  // bits 0-5 position in the layer (or batch), 6-7 kind, 8: fine table, 9: table exact,
                  // 10-31 record index (the fine-table slot when bit 8 is set)
};
static_assert(sizeof(Pair) == 32, "Pair must be one 32-byte sector");

// What the table path reads of a pair (the layer keeps it beside the full
// Pair, which only the Halley iteration needs).
struct __align__(16) PairHot {
  float max_l;    // exposure (maximum loss)
  float mu;       // mean loss
  uint32_t meta;  // as Pair::meta
  uint32_t node;  // first node of the record's quantile table (coarse or fine table of its ELT)
};

constexpr uint32_t kMaxEltRecords = 1u << 22;  // record index field of meta
constexpr uint32_t kMetaPosMask = 63u;          // positions 0..63
constexpr uint32_t kMetaKindShift = 6, kMetaFineBit = 8, kMetaExactBit = 9, kMetaRecShift = 10;

__host__ __device__ inline uint32_t pair_pos(uint32_t meta) { return meta & kMetaPosMask; }
__host__ __device__ inline uint32_t pair_kind(uint32_t meta) { return (meta >> kMetaKindShift) & 3u; }
__host__ __device__ inline bool pair_fine(uint32_t meta) { return (meta >> kMetaFineBit) & 1u; }
__host__ __device__ inline bool pair_tab_exact(uint32_t meta) { return (meta >> kMetaExactBit) & 1u; }
__host__ __device__ inline uint32_t pair_rec(uint32_t meta) { return meta >> kMetaRecShift; }
// Beta and BetaC are the two kinds below kKindMean.
__host__ __device__ inline bool kind_is_beta(uint32_t kind) { return kind < kKindMean; }

// ------------------------------------------------------------------ tables
constexpr int kTabNodes = 32;
constexpr double kTabT1 = 5.294704084854597;  // Phi^-1(1 - 2^-24)
constexpr float kTabT1f = 5.294704f;
constexpr float kTabInvH = static_cast<float>((kTabNodes - 1) / (2.0 * kTabT1));
constexpr float kTabTol = 5e-7f;  // relative error allowed to the table alone
// Fine tables: the same t range at 1/8 of the spacing, 8 * 31 + 1 nodes padded
// to 256, for records whose quantile has features narrower than the coarse
// spacing (U-shaped Betas, a and b well below 1).
constexpr int kTabRefine = 8;
constexpr int kTabFineNodes = kTabRefine * (kTabNodes - 1) + 1;
constexpr int kTabFineStride = 256;

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

// Philox4x32-10 with the ten round keys precomputed (k_r = k_0 + r W): the
// same function, without the key schedule in the loop.
__device__ __forceinline__ uint32_t philox4x32_10_w0(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk[2 * i], lo1, hi0 ^ c.w ^ rk[2 * i + 1], lo0);
  }
  return c.x;
}

__device__ __forceinline__ float philox_uniform_rk(const uint32_t (&rk)[20], int64_t trial, uint32_t k, uint32_t elt) {
  const uint64_t t = static_cast<uint64_t>(trial);
  const uint32_t w = philox4x32_10_w0(make_uint4(static_cast<uint32_t>(t), k, elt, static_cast<uint32_t>(t >> 32)), rk);
  return (static_cast<float>(w >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
}

// The event-occurrence uniform z_(E) (Section 3.1 (ii)): one per (trial,
// event index), shared by every ELT; the same stream with the ELT word
// 0xFFFFFFFF, which no pool id takes.
__device__ __forceinline__ float philox_uniform_event_rk(const uint32_t (&rk)[20], int64_t trial, uint32_t k) {
  return philox_uniform_rk(rk, trial, k, 0xFFFFFFFFu);
}

// Section 3.2 for a record with a correlated sigma: the normal variable
// v = (sigma_I Phi^-1(z_(Prog,E)) + sigma_C Phi^-1(z_(E))) / sqrt(sigma_I^2 +
// sigma_C^2), with w = (sigma_I, sigma_C) / sqrt(sigma_I^2 + sigma_C^2).  Its
// uniform is z = Phi(v); a record's table is a function of t = Phi^-1(z) = v.
__device__ __forceinline__ float correlated_normal(const uint32_t (&rk)[20], int64_t trial, uint32_t k, uint32_t elt,
                                                   float2 w) {
  const float zp = philox_uniform_rk(rk, trial, k, elt);
  const float ze = philox_uniform_event_rk(rk, trial, k);
  return w.x * normcdfinvf(zp) + w.y * normcdfinvf(ze);
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

// Quintic Hermite weights on [0, 1] for the increment w(s) - w_0 given the
// node data (x_i, w_{i+1} - w_i, h w'_i, h^2 w''_i) and (h w'_{i+1}, h^2 w''_{i+1}).
__device__ __forceinline__ float tab_increment(float s, float dw, float d0, float e0, float d1, float e1) {
  const float s2 = s * s, s3 = s2 * s;
  const float g0 = s3 * fmaf(s, fmaf(6.0f, s, -15.0f), 10.0f);                // 10s^3 - 15s^4 + 6s^5
  const float h1 = s * fmaf(s2, fmaf(s, fmaf(-3.0f, s, 8.0f), -6.0f), 1.0f);  // s - 6s^3 + 8s^4 - 3s^5
  const float g1 = s3 * fmaf(s, fmaf(-3.0f, s, 7.0f), -4.0f);                 // -4s^3 + 7s^4 - 3s^5
  const float h2 = 0.5f * s2 * fmaf(s, fmaf(s, 3.0f - s, -3.0f), 1.0f);       // (s^2 - 3s^3 + 3s^4 - s^5)/2
  const float g2 = 0.5f * s3 * fmaf(s, s - 2.0f, 1.0f);                       // (s^3 - 2s^4 + s^5)/2
  return fmaf(dw, g0, fmaf(d0, h1, fmaf(d1, g1, fmaf(e0, h2, e1 * g2))));
}

// x = InvCDF_beta(Phi(t)) from a record's table (nodes are float4 {x_i,
// w_{i+1} - w_i, h w'_i, h^2 w''_i} on a grid in t); `fine` selects the 8x
// refined grid.  t outside the grid's range [-T1, T1] is clamped to it.
__device__ __forceinline__ float tab_quantile_t(const float4* __restrict__ tab, float t, bool fine) {
  const int nseg = fine ? kTabFineNodes - 1 : kTabNodes - 1;
  float u = (t + kTabT1f) * (fine ? kTabInvH * kTabRefine : kTabInvH);
  u = fminf(fmaxf(u, 0.0f), static_cast<float>(nseg));
  int i = static_cast<int>(u);
  if (i > nseg - 1) i = nseg - 1;
  const float s = u - static_cast<float>(i);
  const float4 n0 = __ldg(tab + i);
  if (!(n0.x > 0.0f)) return 0.0f;  // below the FP32 range
  const float2 n1 = __ldg(reinterpret_cast<const float2*>(tab + i + 1) + 1);
  return n0.x * expf(tab_increment(s, n0.y, n0.z, n0.w, n1.x, n1.y));
}

// x = InvCDF_beta(z) from a record's table.
__device__ __forceinline__ float tab_quantile(const float4* __restrict__ tab, float z, bool fine) {
  return tab_quantile_t(tab, normcdfinvf(z), fine);
}

struct BetaSolveStats {
  int iters;
  int cf_terms;
  bool converged;
};

// Root r of I_r(A, B) = P, r expected in (0, ~1/2].  The caller passes
// lnP = ln P and ln1mP = ln(1 - P), each computed from the uniform itself so
// that neither loses the precision of a small P or a small 1 - P;
// x0 = A/(A+B), y0 = B/(A+B); C as above.
__device__ __forceinline__ float beta_solve_oriented(float A, float B, float x0, float y0, float C, float lnP,
                                                     float ln1mP, float r_start, BetaSolveStats* st) {
  const float P = expf(lnP);
  const float lnA = logf(A);
  // ------------------------------------------------------------ start point
  float r;
  if (r_start > 0.0f && r_start < 1.0f) {
    r = r_start;
  } else if (A >= 1.0f && B >= 1.0f) {
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
      const float ru = 1.0f - expf((ln1mP + logf(B) + lnB) / B);
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
    if (fabsf(du) < 4e-4f) {
      // converged (Halley: the remaining error is O(du^3)); near the root F
      // carries FP32 rounding noise, so the bracket no longer decides
      r = fmaf(r, expm1f(du), r);
      done = true;
      ++it;
      break;
    }
    du = fminf(fmaxf(du, -80.0f), 80.0f);
    float rn = r * expf(du);
    if (!(rn > rlo && rn < rhi)) {
      const float lo = fmaxf(rlo, 1e-37f);
      rn = (rhi > 4.0f * lo) ? sqrtf(lo) * sqrtf(rhi) : 0.5f * (rlo + rhi);
    }
    if (rn == r) { done = true; ++it; break; }
    r = rn;
    if (rhi <= 1e-37f) { done = true; ++it; break; }  // root below the FP32 normal range
  }
  st->iters = it;
  st->cf_terms = cf_total;
  st->converged = done;
  return r;
}

// InvCDF_beta(z; a, b) from z and its complement zc = 1 - z, each computed
// directly (so that neither loses the precision of a value near 0).
__device__ __forceinline__ float pair_quantile_newton_zc(const Pair& p, float z, float zc, float x_start,
                                                         BetaSolveStats* st) {
  const bool m0x = signbit(p.m0);
  const float m0 = fabsf(p.m0);
  const float x0 = m0x ? m0 : 1.0f - m0;
  const float y0 = m0x ? 1.0f - m0 : m0;
  const float lnz = logf(z), ln1mz = logf(zc);
  if (z <= p.p_half) return beta_solve_oriented(p.a, p.b, x0, y0, p.c, lnz, ln1mz, x_start, st);
  const float y_start = (x_start > 0.0f && x_start < 1.0f) ? 1.0f - x_start : -1.0f;
  return 1.0f - beta_solve_oriented(p.b, p.a, y0, x0, p.c, ln1mz, lnz, y_start, st);
}

// InvCDF_beta(z; a, b) of a Beta record by the FP32 Halley iteration; x_start
// in (0, 1) seeds it (otherwise the analytic start point is used).
__device__ __forceinline__ float pair_quantile_newton(const Pair& p, float z, float x_start, BetaSolveStats* st) {
  const bool m0x = signbit(p.m0);
  const float m0 = fabsf(p.m0);
  const float x0 = m0x ? m0 : 1.0f - m0;
  const float y0 = m0x ? 1.0f - m0 : m0;
  const float lnz = logf(z), ln1mz = log1pf(-z);
  if (z <= p.p_half) return beta_solve_oriented(p.a, p.b, x0, y0, p.c, lnz, ln1mz, x_start, st);
  // root above 1/2: 1 - x solves I_{1-x}(b, a) = 1 - z
  const float y_start = (x_start > 0.0f && x_start < 1.0f) ? 1.0f - x_start : -1.0f;
  return 1.0f - beta_solve_oriented(p.b, p.a, y0, x0, p.c, ln1mz, lnz, y_start, st);
}

// Loss of one pair: max_l * InvCDF(z; a, b) for Beta records, the mean for
// sigma == 0 records (and for every record when primary_only), 0 for
// mean == 0 records.  `tab` (may be null) is the record's quantile table (the
// fine one when meta bit 7 is set); newton_only forces the Halley iteration
// for every Beta record.
__device__ __forceinline__ float pair_loss(const Pair& p, float z, bool primary_only, const float4* tab,
                                           bool newton_only, BetaSolveStats* st) {
  const uint32_t kind = pair_kind(p.meta);
  st->iters = 0;
  st->cf_terms = 0;
  st->converged = true;
  if (kind == kKindZero) return 0.0f;
  if (primary_only || !kind_is_beta(kind)) return p.mu;
  if (tab != nullptr && !newton_only) {
    const float x = tab_quantile(tab, z, pair_fine(p.meta));
    if (pair_tab_exact(p.meta)) return p.max_l * x;
    return p.max_l * pair_quantile_newton(p, z, x, st);
  }
  return p.max_l * pair_quantile_newton(p, z, -1.0f, st);
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
