/*
 * FP64 CPU oracle for Aggregate Risk Analysis (ARA) with secondary
 * uncertainty -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct statement of what the
 * CUDA path computes.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it; the product path never links or calls it, and it
 * shares no code, header or constant table with the CUDA sources.
 *
 * Method (B. Varghese, "The GPU vs Phi Debate: Risk Analytics Using
 * Many-Core Computing"):
 *   Algorithm 1 (Section 2.2): for each trial of the YET, for each event in
 *   time order, for each ELT of the layer: look up the event's loss, apply
 *   the ELT financial terms, sum over ELTs; apply the occurrence terms
 *   l = min(max(l - OccR, 0), OccL); accumulate the occurrence losses and
 *   apply the aggregate terms l = min(max(S - AggR, 0), AggL) to the
 *   cumulative sum.  The trial's final aggregate loss is its YLT entry.
 *   Section 3.3: secondary uncertainty is applied to each looked-up loss,
 *   after the lookup and before the financial terms: with
 *   sigma_b = sigma / max_l, mu_b = mu / max_l,
 *   sigma_bmax = sqrt(mu_b (1 - mu_b)) (sigma_b clipped just below it),
 *   alpha = mu_b ((sigma_bmax / sigma_b)^2 - 1),
 *   beta  = (1 - mu_b) ((sigma_bmax / sigma_b)^2 - 1),
 *   Loss  = max_l * InvCDF_beta(z; alpha, beta).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   - occurrence terms act on the event loss combined over ELTs, aggregate
 *     terms on the running sum of occurrence losses (Section 2.2 text);
 *   - ELT financial terms are (retention R, limit L, share s):
 *     l' = s * min(max(l - R, 0), L); the identity is (0, +inf, 1);
 *   - "a value very close to sigma_bmax" is (1 - 1e-6) * sigma_bmax, applied
 *     when sigma_b >= (1 - 1e-6) * sigma_bmax;
 *   - z is one Philox4x32-10 draw per (trial, event index, ELT pool id):
 *     counter (trial mod 2^32, k, elt_id, trial >> 32), key (seed mod 2^32,
 *     seed >> 32), word 0 mapped to ((w >> 9) + 0.5) * 2^-23, which lies in
 *     [2^-24, 1 - 2^-24], is exact in both FP32 and FP64 and has an exact
 *     complement 1 - z on the same grid; with sigma_C = 0 the
 *     five-step combination of Section 3.2 returns z unchanged;
 *   - records may carry a correlated standard deviation sigma_C (Section
 *     3.1): the Beta then uses sigma = sigma_I + sigma_C (Section 3.2 step
 *     i), and its uniform combines z_(Prog,E) with the event-occurrence
 *     uniform z_(E), one draw per (trial, event index) shared by every ELT,
 *     taken from the same Philox stream with the ELT word 0xFFFFFFFF; the
 *     transform of step ii, written as the CDF integral, is the quantile;
 *   - a record with mu = 0 contributes nothing; a record with sigma = 0 has
 *     no secondary uncertainty and contributes mu;
 *   - PML(RP) is the m-th largest year loss, m = ceil(N / RP), and TVaR(RP)
 *     the mean of the m largest (ties broken by trial index).
 *
 * Parity pins: see tests/test_oracle_*.py (closed forms of the Beta quantile,
 * binomial sums, SciPy, cuRAND's Philox generator run as a library,
 * hand-summed tiny YETs, monotonicity and permutation invariants, Monte Carlo
 * moments, brute-force sort).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror and Shaw, "Parallel random      */
/* numbers: as easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 round  */
/* function with two multipliers and a Weyl-sequence key schedule.     */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t a_hi = (uint32_t)(prod_a >> 32), a_lo = (uint32_t)prod_a;
        uint32_t b_hi = (uint32_t)(prod_b >> 32), b_lo = (uint32_t)prod_b;
        uint32_t y0 = b_hi ^ x1 ^ k0;
        uint32_t y1 = b_lo;
        uint32_t y2 = a_hi ^ x3 ^ k1;
        uint32_t y3 = a_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;  /* golden ratio */
        k1 += 0xBB67AE85u;  /* sqrt(3) - 1 */
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The uniform z_(Prog,E) of one (trial, event index, ELT) triple. */
double or_uniform(uint64_t seed, int64_t trial, int32_t k, int32_t elt_id)
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = (uint32_t)((uint64_t)trial & 0xffffffffu);
    ctr[1] = (uint32_t)k;
    ctr[2] = (uint32_t)elt_id;
    ctr[3] = (uint32_t)((uint64_t)trial >> 32);
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, w);
    return ((double)(w[0] >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* The event-occurrence uniform z_(E) of Section 3.1 (ii), shared by all  */
/* ELTs (and layers) for one occurrence: the same stream with the ELT      */
/* word of the counter set to 0xFFFFFFFF, which no pool id takes.          */
double or_uniform_event(uint64_t seed, int64_t trial, int32_t k)
{
    return or_uniform(seed, trial, k, (int32_t)-1);
}

/* ------------------------------------------------------------------ */
/* Standard normal CDF and quantile (Section 3.2 steps ii and v; the   */
/* transform written as the CDF integral is read as the quantile).     */
/* ------------------------------------------------------------------ */
double or_normcdf(double v)
{
    return 0.5 * erfc(-v / sqrt(2.0));
}

/* The v with Phi(v) = p, by bisection on Phi (each halving keeps the root */
/* bracketed) down to adjacent doubles; the upper half by symmetry.        */
double or_normcdfinv(double p)
{
    double lo = -40.0, hi = 0.0;
    int it;
    if (!(p > 0.0)) return -INFINITY;
    if (!(p < 1.0)) return INFINITY;
    if (p > 0.5) return -or_normcdfinv(1.0 - p);
    for (it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (or_normcdf(mid) < p) lo = mid; else hi = mid;
    }
    return (p - or_normcdf(lo) <= or_normcdf(hi) - p) ? lo : hi;
}

/* Section 3.2: the uniform fed to the Beta quantile from z_(Prog,E) = zp  */
/* and z_(E) = ze: sigma = sI + sC, v_P = Phi^-1(zp), v_E = Phi^-1(ze),    */
/* LC = v_P sI / sigma + v_E sC / sigma, v = LC / sqrt((sI/sigma)^2 +      */
/* (sC/sigma)^2), z = Phi(v).  The two extreme cases the model names are   */
/* exact: sC = 0 gives zp, sI = 0 gives ze.  Returns v; *z and *zc receive  */
/* Phi(v) and 1 - Phi(v), each computed directly.                           */
double or_combined_normal(double zp, double ze, double s_i, double s_c, double *z, double *zc)
{
    double s, vp, ve, lc, v;
    if (s_c == 0.0) { *z = zp; *zc = 1.0 - zp; return or_normcdfinv(zp); }
    if (s_i == 0.0) { *z = ze; *zc = 1.0 - ze; return or_normcdfinv(ze); }
    s = s_i + s_c;
    vp = or_normcdfinv(zp);
    ve = or_normcdfinv(ze);
    lc = vp * (s_i / s) + ve * (s_c / s);
    v = lc / sqrt((s_i / s) * (s_i / s) + (s_c / s) * (s_c / s));
    *z = or_normcdf(v);
    *zc = or_normcdf(-v);
    return v;
}

/* ------------------------------------------------------------------ */
/* Regularised incomplete Beta I_x(a, b) = B(x; a, b) / B(a, b)         */
/* (Section 3.3) by its continued fraction (Abramowitz & Stegun 26.5.8)*/
/* evaluated with the modified Lentz method, using the symmetry         */
/* I_x(a, b) = 1 - I_{1-x}(b, a) on the side where the fraction        */
/* converges fast, x > (a + 1) / (a + b + 2).                           */
/* ------------------------------------------------------------------ */
static double log_beta_fn(double a, double b)
{
    return lgamma(a) + lgamma(b) - lgamma(a + b);
}

/* 1 / (1 + d1 / (1 + d2 / (1 + ...))) with
 *   d_{2m+1} = -(a + m)(a + b + m) x / ((a + 2m)(a + 2m + 1)),
 *   d_{2m}   =  m (b - m) x / ((a + 2m - 1)(a + 2m)).              */
static double beta_cont_frac(double a, double b, double x, int *n_terms)
{
    /* Modified Lentz evaluation of K = 1 + d1/(1 + d2/(1 + ...)); returns 1/K. */
    const double tiny = 1e-300, eps = 1e-16;
    double K = 1.0, C = 1.0, D = 0.0, delta, num;
    int m;
    for (m = 1; m <= 100000; ++m) {
        int h = m / 2;
        if (m & 1)
            num = -(a + h) * (a + b + h) * x / ((a + 2.0 * h) * (a + 2.0 * h + 1.0));
        else
            num = h * (b - h) * x / ((a + 2.0 * h - 1.0) * (a + 2.0 * h));
        D = 1.0 + num * D;
        if (fabs(D) < tiny) D = tiny;
        C = 1.0 + num / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        delta = C * D;
        K *= delta;
        if (fabs(delta - 1.0) < eps) break;
    }
    if (n_terms) *n_terms = m;
    return 1.0 / K;
}

double or_betainc(double x, double a, double b)
{
    double lfront;
    if (!(x > 0.0)) return 0.0;
    if (!(x < 1.0)) return 1.0;
    lfront = a * log(x) + b * log1p(-x) - log_beta_fn(a, b);
    if (x < (a + 1.0) / (a + b + 2.0))
        return exp(lfront) * beta_cont_frac(a, b, x, NULL) / a;
    return 1.0 - exp(lfront) * beta_cont_frac(b, a, 1.0 - x, NULL) / b;
}

/* Beta density x^(a-1) (1-x)^(b-1) / B(a, b). */
static double beta_pdf(double x, double a, double b, double lbeta)
{
    return exp((a - 1.0) * log(x) + (b - 1.0) * log1p(-x) - lbeta);
}

/* The root x of I_x(a, b) = p on (0, 1/2], given that I_{1/2}(a, b) >= p.
 * Bracketed Newton: the bracket [lo, hi] always satisfies
 * I_lo <= p <= I_hi; a Newton step that leaves it is replaced by a
 * bisection step (geometric while the bracket spans more than a factor of
 * two, so that roots near 1e-300 are reached in a few dozen steps). */
static double betaincinv_small_root(double p, double a, double b)
{
    const double floor_x = 1e-300;
    double lbeta = log_beta_fn(a, b);
    double lo = 0.0, hi = 0.5, x, xn;
    int it;
    /* initial point: the small-x form I_x ~ x^a / (a B(a,b)) */
    x = exp((log(p) + log(a) + lbeta) / a);
    if (!(x > floor_x) || !(x < hi)) x = 0.25;
    for (it = 0; it < 2000; ++it) {
        double f = or_betainc(x, a, b) - p;
        if (f == 0.0) return x;
        if (f < 0.0) lo = x; else hi = x;
        xn = x - f / beta_pdf(x, a, b, lbeta);
        if (!(xn > lo && xn < hi)) {
            double l = lo > floor_x ? lo : floor_x;
            if (lo == 0.0 && hi <= floor_x) return hi; /* root below the double range */
            if (hi > 2.0 * l) xn = sqrt(l * hi);
            else xn = 0.5 * (lo + hi);
        }
        if (fabs(xn - x) <= 1e-15 * xn || xn == lo || xn == hi) { x = xn; break; }
        x = xn;
    }
    return x;
}

/* InvCDF_beta(p; a, b) of Section 3.3: the x in (0, 1) with I_x(a, b) = p.
 * The root is computed as the smaller of x and 1 - x, so that both ends
 * keep full relative precision: when I_{1/2}(a, b) < p the root lies above
 * 1/2 and 1 - x solves I_{1-x}(b, a) = 1 - p. */
double or_betaincinv(double p, double a, double b)
{
    if (!(p > 0.0)) return 0.0;
    if (!(p < 1.0)) return 1.0;
    if (p <= or_betainc(0.5, a, b)) return betaincinv_small_root(p, a, b);
    return 1.0 - betaincinv_small_root(1.0 - p, b, a);
}

/* 1 - InvCDF_beta(p; a, b), accurate when the root is close to 1. */
double or_betaincinv_complement(double p, double a, double b)
{
    if (!(p > 0.0)) return 1.0;
    if (!(p < 1.0)) return 0.0;
    if (p <= or_betainc(0.5, a, b)) return 1.0 - betaincinv_small_root(p, a, b);
    return betaincinv_small_root(1.0 - p, b, a);
}

/* InvCDF_beta(1 - q; a, b): the x with 1 - I_x(a, b) = q, from the upper-  */
/* tail probability q itself (so that a q far below 1 keeps its precision). */
/* When the root lies above 1/2 (q <= I_{1/2}(b, a)) its complement y = 1 - x */
/* is the small root of I_y(b, a) = q.                                       */
double or_betaincinv_upper(double q, double a, double b)
{
    if (!(q > 0.0)) return 1.0;
    if (!(q < 1.0)) return 0.0;
    if (q <= or_betainc(0.5, b, a)) return 1.0 - betaincinv_small_root(q, b, a);
    return betaincinv_small_root(1.0 - q, a, b);
}

/* Beta shape parameters of one XELT record (Section 3.3).  Returns 0 when
 * the record carries secondary uncertainty (alpha, beta set), 1 when it is
 * deterministic (sigma == 0 or mu == 0), -1 when it is invalid
 * (mu_b outside (0, 1) with mu > 0, or a negative/non-finite value). */
int or_beta_params(double mu, double sigma, double max_l, double *alpha, double *beta)
{
    const double delta = 1e-6;
    double mu_b, s_b, s_max, k;
    if (!(mu >= 0.0) || !(sigma >= 0.0) || !isfinite(mu) || !isfinite(sigma) || !isfinite(max_l))
        return -1;
    if (mu == 0.0 || sigma == 0.0) return 1;
    if (!(max_l > mu)) return -1;
    mu_b = mu / max_l;
    s_b = sigma / max_l;
    s_max = sqrt(mu_b * (1.0 - mu_b));
    if (s_b >= (1.0 - delta) * s_max) s_b = (1.0 - delta) * s_max;
    k = (s_max / s_b) * (s_max / s_b) - 1.0;
    *alpha = mu_b * k;
    *beta = (1.0 - mu_b) * k;
    return 0;
}

/* One record's loss with or without secondary uncertainty.  sigma_c is the */
/* record's correlated standard deviation (Section 3.1): the Beta uses      */
/* sigma = sigma_I + sigma_C (Section 3.2 step i), and its uniform is the   */
/* combination of z_(Prog,E) and z_(E).                                      */
static double record_loss(double mu, double sigma, double sigma_c, double max_l, int primary_only,
                          uint64_t seed, int64_t trial, int32_t k, int32_t elt_id)
{
    double a, b, zp, z, zc;
    int kind;
    if (primary_only) return mu;
    kind = or_beta_params(mu, sigma + sigma_c, max_l, &a, &b);
    if (kind != 0) return mu; /* mu == 0 or sigma == 0 (invalid records are rejected at load) */
    zp = or_uniform(seed, trial, k, elt_id);
    if (sigma_c == 0.0) return max_l * or_betaincinv(zp, a, b);
    or_combined_normal(zp, or_uniform_event(seed, trial, k), sigma, sigma_c, &z, &zc);
    /* z above 1/2 is solved from 1 - z = Phi(-v), which keeps its precision */
    return max_l * ((z <= 0.5) ? or_betaincinv(z, a, b) : or_betaincinv_upper(zc, a, b));
}

static double clamp_terms(double l, double retention, double limit)
{
    double v = l - retention;
    if (v < 0.0) v = 0.0;
    if (v > limit) v = limit;
    return v;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 with secondary uncertainty for one layer.               */
/*   yet: offsets[n_trials + 1], ids[offsets[n_trials]]                */
/*   elts: the layer's ELTs, each a sorted list of (event id, mu,      */
/*         sigma, max_l) with per-ELT terms (ret, lim, share) and pool */
/*         id (the Philox key component)                               */
/*   trials: n_list trial indices to evaluate (NULL: all trials)       */
/* Outputs per listed trial: year loss, gross loss sum_k G_k (before    */
/* any terms), hit count (number of (event, ELT) pairs with a record), */
/* and a hash of the hit list (sum over hits of a 64-bit mix of        */
/* (k, elt_id)), all optional.                                          */
/* ------------------------------------------------------------------ */
static uint64_t mix64(uint64_t v)
{
    v ^= v >> 33; v *= 0xff51afd7ed558ccdull;
    v ^= v >> 33; v *= 0xc4ceb9fe1a85ec53ull;
    v ^= v >> 33;
    return v;
}

/* The layer's records as a direct-access table, row_of[j * C + e] = the  */
/* record of event e in the layer's j-th ELT, or -1 (Section 4.2 keeps the  */
/* ELTs as direct-access tables too).  NULL on a bad event id or no memory. */
static int32_t *direct_access_rows(int32_t catalogue, int32_t n_elts, const int64_t *rec_offsets,
                                   const int32_t *rec_events, int *status)
{
    int32_t *row_of;
    int64_t j, e;
    row_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)catalogue * (size_t)(n_elts > 0 ? n_elts : 1));
    if (!row_of) { *status = -2; return NULL; }
    for (j = 0; j < (int64_t)catalogue * n_elts; ++j) row_of[j] = -1;
    for (j = 0; j < n_elts; ++j)
        for (e = rec_offsets[j]; e < rec_offsets[j + 1]; ++e) {
            int32_t ev = rec_events[e];
            if (ev < 0 || ev >= catalogue) { free(row_of); *status = -3; return NULL; }
            row_of[j * (int64_t)catalogue + ev] = (int32_t)e;
        }
    *status = 0;
    return row_of;
}

/* What one trial's year loss depends on: the layer (its ELT records and   */
/* terms) and the draw (seed, primary-only switch).                         */
typedef struct {
    int32_t catalogue, n_elts;
    const int32_t *row_of, *elt_pool_ids;
    const float *mean, *sigma, *sigma_c, *exposure, *elt_terms;
    double occ_ret, occ_lim, agg_ret, agg_lim;
    uint64_t seed;
    int primary_only;
} layer_def;

/* Per-trial by-products: the gross loss (sum of the sampled record losses  */
/* before any terms), the number of (event occurrence, ELT record) pairs   */
/* and an order-free hash of them.                                          */
typedef struct {
    double gross;
    int64_t hits;
    uint64_t hash;
} trial_extras;

/* The loss of event occurrence k (event id ev) of trial t combined over    */
/* the layer's ELTs, before the occurrence terms.  Section 2.2: each ELT's   */
/* loss for the event, after that ELT's financial terms, summed over the     */
/* ELTs of the layer; an ELT without a record for the event contributes     */
/* nothing.  Section 3.3: the loss of a record is the secondary-uncertainty */
/* draw, taken before the financial terms act on it.                         */
static double combined_event_loss(const layer_def *L, int64_t t, int32_t k, int32_t ev, trial_extras *x)
{
    double combined = 0.0;
    int32_t j;
    for (j = 0; j < L->n_elts; ++j) {
        int32_t r = L->row_of[(int64_t)j * L->catalogue + ev];
        double sampled;
        if (r < 0) continue;
        sampled = record_loss(L->mean[r], L->sigma[r], L->sigma_c ? L->sigma_c[r] : 0.0f, L->exposure[r],
                              L->primary_only, L->seed, t, k, L->elt_pool_ids[j]);
        x->gross += sampled;
        x->hits += 1;
        x->hash += mix64(((uint64_t)(uint32_t)k << 32) | (uint32_t)L->elt_pool_ids[j]);
        combined += L->elt_terms
                        ? (double)L->elt_terms[3 * j + 2] *
                              clamp_terms(sampled, L->elt_terms[3 * j + 0], L->elt_terms[3 * j + 1])
                        : sampled;
    }
    return combined;
}

/* The year loss of trial t (Section 2.2 and the YLT of Section 2.3): the    */
/* occurrence terms act on each event's combined loss; the aggregate terms   */
/* act on the running total of the occurrence losses, taken in the trial's  */
/* event (time) order; the value after the last event is the year loss, 0   */
/* for a trial without events.                                               */
static double trial_year_loss(const layer_def *L, const int64_t *offsets, const int32_t *ids, int64_t t,
                              trial_extras *x)
{
    double running = 0.0, after_aggregate = 0.0;
    int64_t pos;
    x->gross = 0.0;
    x->hits = 0;
    x->hash = 0;
    for (pos = offsets[t]; pos < offsets[t + 1]; ++pos) {
        int32_t k = (int32_t)(pos - offsets[t]);
        double occurrence = clamp_terms(combined_event_loss(L, t, k, ids[pos], x), L->occ_ret, L->occ_lim);
        running += occurrence;
        after_aggregate = clamp_terms(running, L->agg_ret, L->agg_lim);
    }
    return after_aggregate;
}

static void set_layer_def(layer_def *L, const int32_t *row_of, int32_t catalogue, int32_t n_elts,
                          const int32_t *elt_pool_ids, const float *mean, const float *sigma, const float *sigma_c,
                          const float *exposure, const float *elt_terms, double occ_ret, double occ_lim,
                          double agg_ret, double agg_lim, uint64_t seed, int primary_only)
{
    L->row_of = row_of;
    L->catalogue = catalogue;
    L->n_elts = n_elts;
    L->elt_pool_ids = elt_pool_ids;
    L->mean = mean;
    L->sigma = sigma;
    L->sigma_c = sigma_c;
    L->exposure = exposure;
    L->elt_terms = elt_terms;
    L->occ_ret = occ_ret;
    L->occ_lim = occ_lim;
    L->agg_ret = agg_ret;
    L->agg_lim = agg_lim;
    L->seed = seed;
    L->primary_only = primary_only;
}

/* The YLT of one layer over a list of trials (all trials when `trials` is */
/* NULL), with the per-trial by-products above (each output optional).     */
int or_run_layer(int64_t n_trials, const int64_t *offsets, const int32_t *ids, int32_t catalogue,
                 int32_t n_elts, const int32_t *elt_pool_ids, const int64_t *rec_offsets,
                 const int32_t *rec_events, const float *rec_mean, const float *rec_sigma,
                 const float *rec_sigma_c /* or NULL: all zero */,
                 const float *rec_exposure, const float *elt_terms /* [n_elts*3] or NULL */,
                 double occ_ret, double occ_lim, double agg_ret, double agg_lim,
                 uint64_t seed, int primary_only,
                 int64_t n_list, const int64_t *trials,
                 double *ylt, double *gross, int64_t *n_hits, uint64_t *hit_hash, int n_threads)
{
    layer_def L;
    int status;
    int32_t *row_of;
    int64_t n_eval;
    if (catalogue <= 0 || n_elts < 0) return -1;
    row_of = direct_access_rows(catalogue, n_elts, rec_offsets, rec_events, &status);
    if (!row_of) return status;
    set_layer_def(&L, row_of, catalogue, n_elts, elt_pool_ids, rec_mean, rec_sigma, rec_sigma_c, rec_exposure,
                  elt_terms, occ_ret, occ_lim, agg_ret, agg_lim, seed, primary_only);
    n_eval = trials ? n_list : n_trials;
    {
        int64_t i;
#ifdef _OPENMP
        /* n_threads > 0: that many threads for this call only */
        const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#else
        (void)n_threads;
#endif
        for (i = 0; i < n_eval; ++i) {
            trial_extras x;
            double y = trial_year_loss(&L, offsets, ids, trials ? trials[i] : i, &x);
            ylt[i] = y;
            if (gross) gross[i] = x.gross;
            if (n_hits) n_hits[i] = x.hits;
            if (hit_hash) hit_hash[i] = x.hash;
        }
    }
    free(row_of);
    return 0;
}

/* Per-event output of one layer: the Algorithm 1 loop over trials        */
/* t_begin .. t_end-1 in order, emitting one row per event occurrence that  */
/* at least one of the layer's ELTs holds a record for, in (trial, event    */
/* index) order: the trial, the event index k, the event id, the event's     */
/* occurrence loss O_k (after the occurrence terms) and the increment        */
/* inc_k = A_k - A_{k-1} of the loss after aggregate terms (A before the     */
/* first event is 0), so that a trial's increments add up to its year loss. */
/* max_occ (optional) receives each trial's largest O_k, 0 without rows.    */
/* Returns the number of rows, or -1 when cap is too small (-2: no memory). */
int64_t or_run_layer_events(const int64_t *offsets, const int32_t *ids, int32_t catalogue,
                            int32_t n_elts, const int32_t *elt_pool_ids, const int64_t *rec_offsets,
                            const int32_t *rec_events, const float *rec_mean, const float *rec_sigma,
                            const float *rec_sigma_c, const float *rec_exposure, const float *elt_terms,
                            double occ_ret, double occ_lim, double agg_ret, double agg_lim,
                            uint64_t seed, int primary_only, int64_t t_begin, int64_t t_end,
                            int64_t *row_trial, int32_t *row_k, int32_t *row_event, double *row_occ,
                            double *row_inc, int64_t cap, double *max_occ)
{
    layer_def L;
    int status;
    int32_t *row_of;
    int64_t t, n = 0;
    if (catalogue <= 0 || n_elts < 0) return -3;
    row_of = direct_access_rows(catalogue, n_elts, rec_offsets, rec_events, &status);
    if (!row_of) return status == -2 ? -2 : -3;
    set_layer_def(&L, row_of, catalogue, n_elts, elt_pool_ids, rec_mean, rec_sigma, rec_sigma_c, rec_exposure,
                  elt_terms, occ_ret, occ_lim, agg_ret, agg_lim, seed, primary_only);
    for (t = t_begin; t < t_end; ++t) {
        double running = 0.0, before = 0.0, O_max = 0.0;
        int64_t pos;
        for (pos = offsets[t]; pos < offsets[t + 1]; ++pos) {
            int32_t k = (int32_t)(pos - offsets[t]);
            trial_extras x = {0.0, 0, 0};
            double occurrence = clamp_terms(combined_event_loss(&L, t, k, ids[pos], &x), occ_ret, occ_lim);
            double after;
            if (x.hits == 0) continue; /* no ELT of the layer holds the event: no row */
            running += occurrence;
            after = clamp_terms(running, agg_ret, agg_lim);
            if (n >= cap) { free(row_of); return -1; }
            row_trial[n] = t;
            row_k[n] = k;
            row_event[n] = ids[pos];
            row_occ[n] = occurrence;
            row_inc[n] = after - before;
            ++n;
            before = after;
            if (occurrence > O_max) O_max = occurrence;
        }
        if (max_occ) max_occ[t - t_begin] = O_max;
    }
    free(row_of);
    return n;
}

/* Per-occurrence combined event losses l_T (after ELT terms, before the
 * occurrence terms) of the listed trials, for the percentile calibration of
 * layer terms.  Writes the nonzero values into out (capacity cap) and
 * returns their count (or -1 when cap is too small). */
int64_t or_event_losses(const int64_t *offsets, const int32_t *ids, int32_t catalogue,
                        int32_t n_elts, const int32_t *elt_pool_ids, const int64_t *rec_offsets,
                        const int32_t *rec_events, const float *rec_mean, const float *rec_sigma,
                        const float *rec_sigma_c, const float *rec_exposure, const float *elt_terms,
                        uint64_t seed, int primary_only, int64_t t_begin, int64_t t_end,
                        double *out, int64_t cap)
{
    layer_def L;
    int status;
    int32_t *row_of;
    int64_t t, n = 0;
    if (catalogue <= 0 || n_elts < 0) return -3;
    row_of = direct_access_rows(catalogue, n_elts, rec_offsets, rec_events, &status);
    if (!row_of) return status == -2 ? -2 : -3;
    set_layer_def(&L, row_of, catalogue, n_elts, elt_pool_ids, rec_mean, rec_sigma, rec_sigma_c, rec_exposure,
                  elt_terms, 0.0, 0.0, 0.0, 0.0, seed, primary_only);
    for (t = t_begin; t < t_end; ++t) {
        int64_t pos;
        for (pos = offsets[t]; pos < offsets[t + 1]; ++pos) {
            trial_extras x = {0.0, 0, 0};
            double combined = combined_event_loss(&L, t, (int32_t)(pos - offsets[t]), ids[pos], &x);
            if (combined != 0.0) {
                if (n >= cap) { free(row_of); return -1; }
                out[n++] = combined;
            }
        }
    }
    free(row_of);
    return n;
}

/* ------------------------------------------------------------------ */
/* PML and TVaR from the YLT (Section 2.3): order the trials by year   */
/* loss, largest first, ties by trial index; PML(RP) is the m-th       */
/* value, m = ceil(N / RP); TVaR(RP) is the mean of the first m.        */
/* ------------------------------------------------------------------ */
static const double *g_sort_keys;
static int cmp_desc(const void *pa, const void *pb)
{
    int64_t ia = *(const int64_t *)pa, ib = *(const int64_t *)pb;
    double va = g_sort_keys[ia], vb = g_sort_keys[ib];
    if (va > vb) return -1;
    if (va < vb) return 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

int or_sort_desc(const double *ylt, int64_t n, int64_t *order)
{
    int64_t i;
    for (i = 0; i < n; ++i) order[i] = i;
    g_sort_keys = ylt;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_desc);
    return 0;
}

int or_pml_tvar(const double *ylt, int64_t n, const double *rps, int32_t n_rp,
                double *pml, double *tvar)
{
    int64_t *order;
    int32_t r;
    if (n <= 0) return -1;
    order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!order) return -2;
    or_sort_desc(ylt, n, order);
    for (r = 0; r < n_rp; ++r) {
        int64_t m = (int64_t)ceil((double)n / rps[r]), i;
        long double acc = 0.0L;
        if (m < 1) m = 1;
        if (m > n) m = n;
        for (i = 0; i < m; ++i) acc += (long double)ylt[order[i]];
        pml[r] = ylt[order[m - 1]];
        tvar[r] = (double)(acc / (long double)m);
    }
    free(order);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Batched forms of the scalar functions above, for the tests.         */
/* ------------------------------------------------------------------ */
void or_uniform_batch(uint64_t seed, int64_t n, const int64_t *trials, const int32_t *ks,
                      const int32_t *elts, double *out)
{
    int64_t i;
    for (i = 0; i < n; ++i) out[i] = or_uniform(seed, trials[i], ks[i], elts[i]);
}

void or_combined_normal_batch(uint64_t seed, int64_t n, const int64_t *trials, const int32_t *ks,
                              const int32_t *elts, double s_i, double s_c, double *v_out, double *z_out)
{
    int64_t i;
    for (i = 0; i < n; ++i) {
        double z, zc;
        v_out[i] = or_combined_normal(or_uniform(seed, trials[i], ks[i], elts[i]),
                                      or_uniform_event(seed, trials[i], ks[i]), s_i, s_c, &z, &zc);
        if (z_out) z_out[i] = z;
    }
}

void or_normcdfinv_batch(int64_t n, const double *p, double *out)
{
    int64_t i;
    for (i = 0; i < n; ++i) out[i] = or_normcdfinv(p[i]);
}

void or_betaincinv_batch(int64_t n, const double *p, const double *a, const double *b, double *out)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < n; ++i) out[i] = or_betaincinv(p[i], a[i], b[i]);
}

void or_betainc_batch(int64_t n, const double *x, const double *a, const double *b, double *out)
{
    int64_t i;
    for (i = 0; i < n; ++i) out[i] = or_betainc(x[i], a[i], b[i]);
}
