/*
 * ara.h -- C ABI of the GB300 (sm_103a) Aggregate Risk Analysis engine.
 *
 * The engine runs the data-parallel hot path of Aggregate Risk Analysis (ARA)
 * with secondary uncertainty (B. Varghese, "The GPU vs Phi Debate: Risk
 * Analytics Using Many-Core Computing"): for each trial of a Year Event Table
 * (YET), for each event in time order, for each Event Loss Table (ELT) of a
 * layer, look up the event's loss record, draw a loss from the record's Beta
 * distribution (Section 3.3), apply the ELT financial terms, sum over the
 * layer's ELTs, apply the occurrence terms, and apply the aggregate terms to
 * the running sum of occurrence losses (Algorithm 1, Section 2.2).  The result
 * is the Year Loss Table (YLT), from which PML and TVaR are read (Section 2.3).
 *
 * Conventions for every entry point:
 *   - Return value: ARA_OK (0) on success, a negative ARA_E* code on failure.
 *     On failure ara_last_error() describes the cause.  No entry point aborts,
 *     traps on the device or throws across this boundary.
 *   - Pointers: input arrays may be host or device memory (the kind is
 *     detected per pointer).  Inputs are read during the call only; the
 *     library copies what it keeps into device memory that it owns and frees
 *     in ara_destroy().  Output arrays are owned by the caller and may be host
 *     or device memory.
 *   - Ordering: all device work is issued on the context's CUDA stream.  A call
 *     whose outputs are all device memory returns without synchronising; a
 *     call with a host output synchronises the stream before returning.
 *   - Threading: a context is used by one host thread at a time.
 *   - Device: a context binds one CUDA device (chosen at ara_create) and makes
 *     it current on every call.
 */
#ifndef ARA_H
#define ARA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ARA_API __attribute__((visibility("default")))
#else
#define ARA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define ARA_OK 0
#define ARA_EINVAL (-1)     /* invalid argument or input data */
#define ARA_ENOMEM (-2)     /* device allocation failed or over the HBM budget */
#define ARA_ENOTLOADED (-3) /* the YET or a referenced ELT is not loaded */
#define ARA_ECUDA (-4)      /* a CUDA runtime call failed */
#define ARA_ETIMEOUT (-5)   /* a bounded wait gave up (ara_wait) */
#define ARA_EAGAIN (-6)     /* a served request has not finished yet */

/* Largest number of ELTs in one layer.  The paper's layers cover 3 to 30
 * ELTs (Section 2.1 (iii)). */
#define ARA_MAX_LAYER_ELTS 32

/* Relative gap below sigma_bmax used when sigma_b is clipped: the paper
 * clips sigma_b to "a value very close to sigma_bmax" (Section 3.3); this
 * library uses (1 - ARA_SIGMA_CLIP) * sigma_bmax whenever
 * sigma_b >= (1 - ARA_SIGMA_CLIP) * sigma_bmax. */
#define ARA_SIGMA_CLIP 1e-6

/* Layer flags */
#define ARA_PRIMARY_ONLY 1u /* no secondary uncertainty: every record's loss is its mean */
#define ARA_NEWTON_ONLY 2u  /* invert every Beta by the FP32 Halley iteration, not the record's quantile table */
/* The uniform z_(Prog,E) per event occurrence, shared by the layer's ELTs
 * (Section 3.1 keys it by the YET entry): every pair of an occurrence draws
 * word 0 of the Philox block with the ELT word of the counter set to
 * 0xFFFFFFFE (no pool id takes it) in place of its ELT pool id, which also
 * stands for the pool id in the hit hash of ara_run_layer_diag.  Without it,
 * each (trial, event index, ELT pool id) has its own draw. */
#define ARA_SHARED_Z 4u
/* ara_run_layers: pick the losses kernel's configuration (its work item, see
 * ara_set_batch_config; CTAs per SM) by measurement.  The first pass
 * of a batch shape (layers, ELTs of the union, trials, hit records per trial)
 * runs every candidate once, timed with CUDA events, and keeps the fastest
 * for later passes of that shape; all candidates give the same bits.  Without
 * the flag a pass uses the cached choice for its shape if there is one, else
 * the default rule. */
#define ARA_AUTOTUNE 16u

typedef struct ara_ctx ara_ctx;

/* Per-ELT financial terms I (Section 2.1 (ii)), read as retention R, limit L
 * and share s: l' = s * min(max(l - R, 0), L).  Identity: {0, +INF, 1}. */
typedef struct {
    float retention;
    float limit;
    float share;
} ara_elt_terms;

/* A layer (Section 2.1 (iii)): a set of ELTs from the resident pool and the
 * layer terms T = (OccR, OccL, AggR, AggL).  Occurrence terms apply to the
 * event loss combined over the layer's ELTs, l = min(max(l - OccR, 0), OccL);
 * aggregate terms to the running sum S of occurrence losses,
 * l = min(max(S - AggR, 0), AggL) (Section 2.2).  Retentions are >= 0, limits
 * > 0 and may be +INF. */
typedef struct {
    int32_t n_elts;         /* 1 .. ARA_MAX_LAYER_ELTS */
    const int32_t *elt_ids; /* host array of n_elts distinct pool ids */
    double occ_retention;
    double occ_limit;
    double agg_retention;
    double agg_limit;
    uint32_t flags; /* ARA_PRIMARY_ONLY, ARA_NEWTON_ONLY, ARA_SHARED_Z, or 0 */
} ara_layer;

/* Optional per-trial diagnostics of ara_run_layer_diag(); any pointer may be
 * NULL.  Arrays have trial_end - trial_begin entries, host or device. */
typedef struct {
    int64_t *hits;      /* number of (event, ELT) lookups that found a record */
    uint64_t *hit_hash; /* sum over hits of fmix64((k << 32) | elt_id), k = event index in the trial */
} ara_diag;

/* Per-event output of ara_run_layer_events() (the Year Event Loss Table).
 * One row per event occurrence of the trial range that at least one of the
 * layer's ELTs holds a record for, in (trial, event index) order.  Every
 * pointer may be NULL (not written) and may be host or device memory; row
 * arrays hold `capacity` entries and only the first min(capacity, n_rows)
 * rows are written. */
typedef struct {
    int64_t capacity;     /* rows the arrays below hold */
    int64_t *trial;       /* trial index */
    int32_t *event_index; /* k: position of the event in the trial, from 0 */
    int32_t *event_id;    /* the event's id in the catalogue */
    double *occ_loss;     /* O_k: the event's loss after ELT and occurrence terms */
    double *agg_inc;      /* inc_k = A_k - A_(k-1), A the loss after aggregate terms */
    double *max_occ;      /* trial_end - trial_begin entries: each trial's largest O_k (0 without rows) */
    int64_t n_rows;       /* out: rows of the trial range (may exceed capacity) */
} ara_event_rows;

/* Counters of the last ara_run_layer* call (read back with ara_get_stats). */
typedef struct {
    int64_t n_events;        /* YET entries scanned */
    int64_t n_evals;         /* n_events x n_elts: trial-event-ELT evaluations */
    int64_t n_pairs_hit;     /* (event, ELT) lookups that found a record */
    int64_t n_nonconverged;  /* Beta inversions that hit the iteration cap */
    int64_t n_newton;        /* pairs inverted by the Halley iteration (not the table alone) */
    float index_ms;          /* per-layer index build, device time */
    float kernel_ms;         /* layer kernels (gather + losses), device time */
    int32_t grid;            /* CTAs of the main kernel */
    int32_t block;           /* threads per CTA */
    int32_t smem_bytes;      /* dynamic shared memory per CTA */
    int32_t filter_bits;     /* shared-memory membership filter size in bits */
    /* ara_run_layers: the losses kernel's configuration (the last pass) */
    int32_t batch_item;          /* the work item: an ARA_BATCH_ITEM_* value */
    int32_t batch_blocks_per_sm; /* resident CTAs per SM of the persistent grid */
    int32_t batch_tuned;         /* 1: chosen by the autotuner (measured), 0: by the default rule */
    int32_t reserved;
} ara_stats;

/* Device time accumulated over the ara_run_layer* and ara_pml_tvar calls
 * since the last reset (CUDA events recorded on the context's stream around
 * each launch group). */
typedef struct {
    int64_t layer_calls;     /* ara_run_layer* calls */
    double kernel_ms;        /* sum of the layer kernels' durations (gather + losses) */
    double gather_ms;        /* of which the gather kernel (YET stream, filter, hit records) */
    double losses_ms;        /* of which the losses kernel (Beta inversion, terms, trial sums) */
    double index_ms;         /* sum of the per-layer index builds */
    int64_t pml_calls;       /* ara_pml_tvar calls */
    double pml_ms;           /* sum of the PML/TVaR selections */
    int64_t kernel_launches; /* kernels this library launched (all calls) */
} ara_timing;

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the
 * device memory the library allocates (0: no cap).  `cuda_stream` is a
 * cudaStream_t to issue work on (NULL: the legacy default stream).
 * Errors: ARA_EINVAL (bad device), ARA_ECUDA. */
ARA_API int ara_create(ara_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Switch the stream used by later calls.  Synchronises the previous stream. */
ARA_API int ara_set_stream(ara_ctx *ctx, void *cuda_stream);

/* Load (replace) the Year Event Table (Section 2.1 (i)).  Trial t owns
 * event_ids[offsets[t] .. offsets[t+1]), in time order.  offsets has
 * n_trials + 1 entries, offsets[0] == 0 and non-decreasing; every id lies in
 * [0, catalogue_size); a trial holds fewer than 2^22 events.  Time stamps
 * are not needed: they only fix the order.
 * Errors: ARA_EINVAL (bad sizes, offsets or ids), ARA_ENOMEM, ARA_ECUDA. */
ARA_API int ara_load_yet(ara_ctx *ctx, int64_t n_trials, const int64_t *offsets, const int32_t *event_ids,
                 int32_t catalogue_size);

/* ara_load_yet without waiting for the upload: the offsets are read and the
 * sizes checked during the call (the call first waits for the work already on
 * the context's stream); the offsets and ids are then copied to the device
 * and checked on an internal stream, beside later work on the context's
 * stream, so that an ELT load (its table build) overlaps the copy.  Ids in
 * pinned host memory are read by a kernel over the host link, which leaves
 * the copy engine to the other streams' copies; other ids are copied by the
 * copy engine.  offsets and event_ids stay owned by the caller and must stay
 * valid and unchanged until the upload is finished: by ara_finish_yet or by
 * the next call that uses the YET (ara_run_layer*, ara_submit,
 * ara_serve_step, ...), which waits for it.  Errors in the offsets or ids are returned by that call (ARA_EINVAL,
 * with no YET loaded); errors in the arguments by this one.  A second upload
 * replaces one still in flight. */
ARA_API int ara_load_yet_async(ara_ctx *ctx, int64_t n_trials, const int64_t *offsets, const int32_t *event_ids,
                               int32_t catalogue_size);

/* Waits for an ara_load_yet_async upload and returns its result (ARA_OK when
 * none is in flight). */
ARA_API int ara_finish_yet(ara_ctx *ctx);

/* Load ELTs into the resident pool (Sections 2.1 (ii), 3.1): ELT i has pool id
 * elt_ids[i] (>= 0) and records rec_offsets[i] .. rec_offsets[i+1] of
 * (event_ids, mean, sigma, exposure), with strictly increasing event ids.
 * `exposure` is the maximum loss max_l; a record with mean > 0 and sigma > 0
 * needs exposure > mean.  mean == 0 gives no loss; sigma == 0 gives the mean
 * (no secondary uncertainty).  `terms` (n_elts entries, NULL: identity) are
 * the ELT financial terms.  Loading a pool id that is already resident
 * replaces it.  The Beta shapes of every record are derived here (Section
 * 3.3), once per record, together with a 32-node quantile table of each
 * record's Beta built in FP64 (512 bytes per record).  At most 2^22 - 1
 * records per ELT.
 * Errors: ARA_EINVAL (unsorted or duplicate ids, negative or non-finite
 * values, exposure <= mean), ARA_ENOMEM, ARA_ECUDA. */
ARA_API int ara_load_elts(ara_ctx *ctx, int32_t n_elts, const int32_t *elt_ids, const int64_t *rec_offsets,
                  const int32_t *event_ids, const float *mean, const float *sigma,
                  const float *exposure, const ara_elt_terms *terms);

/* ara_load_elts with the two-part secondary uncertainty of Sections 3.1 and
 * 3.2: each record's standard deviation is split into an independent part
 * sigma_i and a correlated part sigma_c (both >= 0, finite).  The Beta of
 * Section 3.3 takes sigma = sigma_i + sigma_c.  A record with sigma_c == 0
 * draws its uniform z_(Prog,E) as in ara_load_elts; one with sigma_c > 0 uses
 * z = Phi(v), v = (sigma_i Phi^-1(z_(Prog,E)) + sigma_c Phi^-1(z_(E))) /
 * sqrt(sigma_i^2 + sigma_c^2), where z_(E) is the occurrence's uniform, shared
 * by every ELT and layer: word 0 of the Philox block of ara_run_layer with the
 * ELT word of the counter set to 0xFFFFFFFF (no pool id takes that value).
 * sigma_i == 0 makes every ELT of an occurrence use z = z_(E).  Such ELTs keep
 * 8 more bytes per record (the two weights).  sigma_c must not be NULL when
 * there are records; the other arguments, ownership and errors are those of
 * ara_load_elts. */
ARA_API int ara_load_xelts(ara_ctx *ctx, int32_t n_elts, const int32_t *elt_ids, const int64_t *rec_offsets,
                   const int32_t *event_ids, const float *mean, const float *sigma_i, const float *sigma_c,
                   const float *exposure, const ara_elt_terms *terms);

/* Run one layer over trials [trial_begin, trial_end) (Algorithm 1 with the
 * secondary uncertainty of Section 3.3) and write one year loss per trial to
 * ylt_out (FP64, trial_end - trial_begin entries).  The uniform of trial t,
 * event index k (position in the trial, from 0) and ELT pool id j is word 0
 * of Philox4x32-10 with counter (t mod 2^32, k, j, t >> 32) and key
 * (seed mod 2^32, seed >> 32), mapped to ((w >> 9) + 0.5) * 2^-23.
 * Working memory: 8 bytes per YET entry of the trial range (hit-event
 * records), kept by the context between calls.
 * The loss arithmetic is FP32; each trial's running sum of occurrence losses
 * is FP64.  Event ids outside the catalogue were rejected at load.
 * Errors: ARA_EINVAL (bad layer or range), ARA_ENOTLOADED, ARA_ENOMEM,
 * ARA_ECUDA. */
ARA_API int ara_run_layer(ara_ctx *ctx, const ara_layer *layer, uint64_t seed, int64_t trial_begin,
                  int64_t trial_end, double *ylt_out);

/* ara_run_layer plus the per-trial diagnostics of ara_diag (hit counts and
 * an order-free hash of the hit list), used to check event indexing. */
ARA_API int ara_run_layer_diag(ara_ctx *ctx, const ara_layer *layer, uint64_t seed, int64_t trial_begin,
                       int64_t trial_end, double *ylt_out, const ara_diag *diag);

/* ara_run_layer plus its per-event output (Algorithm 1, Section 2.2, read
 * per event): for each held event occurrence, O_k is the combined loss of the
 * layer's ELTs after the occurrence terms; S_k is the sum of O_1..O_k in
 * event order (FP64), A_k = min(max(S_k - AggR, 0), AggL) the loss after the
 * aggregate terms, and inc_k = A_k - A_(k-1) with A_0 = 0, so that a trial's
 * increments add up to its year loss.  max_occ holds each trial's largest
 * O_k, the input of occurrence exceedance: ara_pml_tvar over max_occ gives the
 * OEP loss and its tail mean at the return periods (the year losses give the
 * aggregate ones).  O_k is the FP32 value the year loss sums; ylt_out is
 * written as by ara_run_layer.  rows->n_rows receives the row count.  Limit:
 * the trial range holds fewer than 2^32 YET entries.  Extra device memory: 4
 * bytes per YET entry of the range, and the rows when the arrays are host
 * memory.
 * Errors: those of ara_run_layer; ARA_EINVAL for a NULL rows or a negative
 * capacity. */
ARA_API int ara_run_layer_events(ara_ctx *ctx, const ara_layer *layer, uint64_t seed, int64_t trial_begin,
                         int64_t trial_end, double *ylt_out, ara_event_rows *rows);

/* Several layers over the same trials in one pass (a batch): the YET of the
 * trial range is read once for all the layers, and the loss after ELT terms
 * of each (event occurrence, ELT) is computed once for every layer of the
 * batch that holds the ELT.  Algorithm 1 runs per layer over a portfolio's
 * layers (Section 2.1 (iii)); each layer's year losses are those of
 * ara_run_layer with the same seed, up to FP32 rounding of the per-event sums
 * (the uniforms depend on the trial, event index and ELT pool id only).
 * layers: n_layers (1..ARA_MAX_BATCH_LAYERS) layers, each as for
 * ara_run_layer, all with the same flags; their ELTs together (the union)
 * number at most ARA_MAX_BATCH_ELTS.
 * ylt_out: n_layers * (trial_end - trial_begin) doubles, layer-major (layer l's
 * year losses start at l * (trial_end - trial_begin)); host or device memory.
 * Each trial's sum of occurrence losses is accumulated per layer as a 64-bit
 * fixed-point integer (a power-of-two scale per layer, chosen from the layer's
 * largest possible occurrence loss and the longest trial of the YET), so the
 * result does not depend on the order of the additions.
 * Errors: ARA_EINVAL (bad layers, mixed flags, union too large, bad range),
 * ARA_ENOTLOADED, ARA_ENOMEM, ARA_ECUDA. */
#define ARA_MAX_BATCH_LAYERS 32
#define ARA_MAX_BATCH_ELTS 64
ARA_API int ara_run_layers(ara_ctx *ctx, int32_t n_layers, const ara_layer *layers, uint64_t seed,
                   int64_t trial_begin, int64_t trial_end, double *ylt_out);

/* The losses kernel of ara_run_layers (and of the serving loop's passes) has
 * three work items, which add the same fixed-point numbers and so give the
 * same bits:
 *   ARA_BATCH_ITEM_TILE   one warp per tile of 8 trials, a lane per hit record;
 *   ARA_BATCH_ITEM_TRIAL  one warp per trial, a lane per hit record;
 *   ARA_BATCH_ITEM_DENSE  one warp per tile of 8 trials, a lane per (event, ELT)
 *                         pair: each pair's loss once, then each record's
 *                         per-layer occurrence losses;
 *   ARA_BATCH_ITEM_INDEXED  (once ara_build_yet_index has run) a warp per
 *                         event of the pass's ELTs, over that event's
 *                         occurrences in the pass's trials, from the YET's
 *                         event-major index: the YET is not streamed.
 * ara_set_batch_config pins the work item and the CTAs per SM of the
 * persistent grid (blocks_per_sm 0: as many as an SM holds; a larger number is
 * cut to that) for later passes; item ARA_BATCH_AUTO returns to the cached
 * autotuner choice for the pass's shape, else the default rule (the indexed
 * item when the YET's index is built, else the dense item, with as many CTAs
 * as an SM holds).
 * Errors: ARA_EINVAL (unknown item, blocks_per_sm outside 0..16). */
#define ARA_BATCH_AUTO (-1)
#define ARA_BATCH_ITEM_TILE 0
#define ARA_BATCH_ITEM_TRIAL 1
#define ARA_BATCH_ITEM_DENSE 2
#define ARA_BATCH_ITEM_INDEXED 3
ARA_API int ara_set_batch_config(ara_ctx *ctx, int32_t item, int32_t blocks_per_sm);

/* The event-major index of the loaded YET (Section 2.1's lookup taken from the
 * ELT side): for each catalogue event, its occurrences (trial, event index) in
 * trial order, built on the device: each occurrence is counted into and placed
 * in a bucket per (event, 262,144-trial cell), and each bucket sorted; where a
 * bucket would hold more than 2,048 occurrences, by a stable radix sort of the
 * YET's events by id instead (the same index).  Once built, batched passes (ara_run_layers and the serving loop)
 * default to ARA_BATCH_ITEM_INDEXED, which reaches a pass's hit events through
 * its ELTs' events instead of streaming every trial's events; the year losses
 * are the same bits as the other work items'.  ara_run_layer (one layer, with
 * its double-float sums and hit diagnostics) keeps streaming the YET.
 * With each event's occurrences the index keeps their offsets at every
 * 262,144 trials (the serving chunk), so that a pass's slices of trials find
 * their occurrences without a search.  It takes 8 bytes per YET event and
 * 4 * (ceil(n_trials / 262144) + 1) per catalogue id, and lasts until the next
 * YET load; the bucket build needs 4 bytes per (catalogue id, cell) of
 * scratch besides, the radix sort about 24 bytes per event.  Errors: ARA_ENOTLOADED; ARA_EINVAL (served requests queued or
 * running, or 2^32 or more events); ARA_ENOMEM; ARA_ECUDA.
 * ara_yet_index_info reports whether the index is built, its bytes, the
 * device time of its build and how it was built (0 buckets, 1 radix sort, -1
 * not built); any pointer may be NULL. */
ARA_API int ara_build_yet_index(ara_ctx *ctx);
ARA_API int ara_yet_index_info(const ara_ctx *ctx, int32_t *built, int64_t *bytes, float *build_ms, int32_t *method);

/* Serving: layer requests against the resident YET and ELT pool, with
 * continuous batching.  The paper has no serving system; a portfolio's
 * layers (Section 2.1 (iii)) are its natural requests, and the chunked,
 * asynchronous hand-off of trials follows the hybrid offload of Section 4.
 *
 * ara_submit queues one request: a layer (as for ara_run_layer), its seed, the
 * trial prefix [0, trial_end) to simulate, and n_rp (1..ARA_SERVE_MAX_RP)
 * return periods (host memory, each >= 1) for PML/TVaR of the prefix's YLT.
 * The layer's ELTs must be loaded.  *ticket receives the request's handle.
 * Errors: ARA_EINVAL, ARA_ENOTLOADED, ARA_ENOMEM (the request's year losses,
 * 8 * trial_end bytes, exceed the serving arena, which the HBM budget bounds:
 * it would never be admitted).
 *
 * The prefix is cut into chunks of trials (ara_serve_info.chunk_trials).
 * ara_serve_step does not wait for the device.  It (1) finishes the requests
 * whose work the device has completed; (2) admits queued requests, in arrival
 * order, whose year losses fit the serving arena (one that does not fit yet
 * stays queued and a later, smaller one may go first); (3) when fewer than two
 * rounds are in flight, launches one round on the context's stream: batched
 * passes over one chunk each (one seed and flags per pass, at most
 * ARA_MAX_BATCH_LAYERS requests with at most ARA_MAX_BATCH_ELTS ELTs
 * together), and, behind each request's last chunk, its PML/TVaR over its own
 * prefix.  Requests submitted while a round runs join the next round, so a
 * short request overtakes a long one admitted before it.  *n_done (may be
 * NULL) receives the number of requests finished in this call.  A request's
 * result does not depend on the requests it shared rounds with.
 * Errors: ARA_ENOMEM (the serving workspace), ARA_ECUDA.  The YET cannot be
 * replaced while requests are queued or running, nor an ELT that a running
 * request uses (ARA_EINVAL).
 *
 * ara_poll returns ARA_EAGAIN while the request is not finished; once
 * finished, it copies its PML and TVaR (n_rp doubles each, host memory) and
 * releases the ticket, returning the request's own status (ARA_OK, or the
 * error its pass met).  Errors: ARA_EINVAL (unknown ticket).
 *
 * ara_wait runs serve steps, and waits on the host for the oldest round when a
 * step finishes nothing, until the request is finished; then it returns as
 * ara_poll does.  It returns ARA_ETIMEOUT, with the request still pending,
 * when timeout_ns (nanoseconds of host time, 0: no limit) has passed at the
 * end of a step or a wait.
 *
 * ara_serve_stats reports the queue: requests queued (not admitted), active
 * (admitted, not finished), rounds in flight, and totals since the context
 * was created. */
typedef struct {
    int64_t queued;            /* submitted, not yet admitted */
    int64_t active;            /* admitted, not finished */
    int64_t rounds_in_flight;  /* launched, not yet retired */
    int64_t rounds_launched;   /* totals since the context was created */
    int64_t passes_launched;
    int64_t requests_finished;
    int64_t chunk_trials;      /* trials per chunk */
    int64_t arena_bytes;       /* device memory for the year losses of admitted requests */
} ara_serve_info;
#define ARA_SERVE_MAX_RP 16
ARA_API int ara_submit(ara_ctx *ctx, const ara_layer *layer, uint64_t seed, int64_t trial_end,
               const double *return_periods, int32_t n_rp, int64_t *ticket);
ARA_API int ara_serve_step(ara_ctx *ctx, int32_t *n_done);
ARA_API int ara_poll(ara_ctx *ctx, int64_t ticket, double *pml_out, double *tvar_out);
ARA_API int ara_wait(ara_ctx *ctx, int64_t ticket, double *pml_out, double *tvar_out, uint64_t timeout_ns);
ARA_API int ara_serve_stats(ara_ctx *ctx, ara_serve_info *out);

/* PML and TVaR of a YLT (Section 2.3) at n_rp return periods (each >= 1):
 * with m = ceil(n / RP), PML is the m-th largest year loss and TVaR the mean
 * of the m largest (FP64).  Computed on the device by a radix select over
 * order-preserving 64-bit keys.  ylt may be host or device memory; pml_out
 * and tvar_out have n_rp entries.
 * Errors: ARA_EINVAL (n < 1, RP < 1), ARA_ENOMEM, ARA_ECUDA. */
ARA_API int ara_pml_tvar(ara_ctx *ctx, const double *ylt, int64_t n, const double *return_periods,
                 int32_t n_rp, double *pml_out, double *tvar_out);

/* Trial order of a YLT, largest year loss first, ties by ascending trial
 * index, by an on-device LSD radix sort of 64-bit keys.  order_out has n
 * entries (host or device).  Errors: ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA. */
ARA_API int ara_sort_ylt(ara_ctx *ctx, const double *ylt, int64_t n, int64_t *order_out);

/* Check entry points: the hot path's own device functions on caller-chosen
 * inputs, for parity tests against an independent implementation.
 *
 * ara_debug_uniforms: out[i] = the uniform of (trials[i], ks[i], elts[i])
 * under `seed`, exactly as ara_run_layer draws it (FP32 values; n entries).
 *
 * ara_debug_record_losses: for n XELT records (mean, sigma, exposure) and
 * uniforms z (FP32, in (0, 1)), out[i] = the secondary-uncertainty loss
 * max_l * InvCDF_beta(z[i]; alpha_i, beta_i) (Section 3.3) computed with the
 * same record preparation, quantile table and FP32 inverse as
 * ara_run_layer (the mean for sigma == 0, 0 for mean == 0); newton_only != 0
 * uses the Halley iteration for every record, as ARA_NEWTON_ONLY does.
 * iters_out (NULL allowed) receives the Halley iteration count of each
 * inversion (0: the table alone; negative: hit the iteration cap).
 * All arrays may be host or device memory.  Errors: ARA_EINVAL, ARA_ENOMEM,
 * ARA_ECUDA. */
ARA_API int ara_debug_uniforms(ara_ctx *ctx, uint64_t seed, int64_t n, const int64_t *trials, const int32_t *ks,
                               const int32_t *elts, float *out);
ARA_API int ara_debug_record_losses(ara_ctx *ctx, int64_t n, const float *mean, const float *sigma,
                                    const float *exposure, const float *z, int32_t newton_only, float *out,
                                    int32_t *iters_out);

/* Trial shards across GPUs (Section 5 treats trials as independent): a rank
 * that holds the YLT of trials [trial_offset, trial_offset + n) needs to send
 * only its m largest year losses for the PML and TVaR of the whole YLT at
 * return periods of at least N_total / m.
 *
 * ara_top_m writes the m largest year losses of ylt (host or device, n >= 1
 * doubles) in descending order, ties by trial index, to values_out, and their
 * global trial indices (trial_offset + local index) to trials_out (m entries
 * each, host or device memory).  When m > n the last m - n entries are
 * (-INFINITY, -1).  Runs the device radix sort of the YLT.
 * Errors: ARA_EINVAL (n < 1 or >= 2^31, m < 1, trial_offset < 0), ARA_ENOMEM,
 * ARA_ECUDA.
 *
 * ara_merge_top (host memory only, no context, no GPU) takes the ranks'
 * lists concatenated (count entries; -INFINITY entries are ignored), orders
 * them by year loss, largest first, ties by global trial index, and writes
 * for each of the n_rp return periods (each >= 1) PML = the m-th value and
 * TVaR = the mean of the first m (m = ceil(n_total / RP), at least 1 and at
 * most n_total), the TVaR sum compensated (Neumaier) in that order: the
 * definitions of ara_pml_tvar over the whole YLT.
 * Errors: ARA_EINVAL (bad arguments, or fewer than m finite values). */
ARA_API int ara_top_m(ara_ctx *ctx, const double *ylt, int64_t n, int64_t m, int64_t trial_offset,
                      double *values_out, int64_t *trials_out);
ARA_API int ara_merge_top(const double *values, const int64_t *trials, int64_t count, int64_t n_total,
                          const double *return_periods, int32_t n_rp, double *pml_out, double *tvar_out);

/* PML and TVaR without any device allocation.
 *
 * Same result as ara_pml_tvar, for callers that may not allocate device
 * memory: code running under a framework's caching allocator, which owns the
 * device memory budget, or in a latency-critical loop where cudaMalloc and
 * cudaFree, which can synchronise the whole device, are not acceptable.  It
 * needs no context (creating one allocates).  The paper has no counterpart.
 *
 * The select state lives in a fixed block of device memory that belongs to
 * the library (ARA_NOALLOC_SCRATCH_BYTES per GPU, held from the library's
 * first use on that GPU until the process exits).  Every call on a GPU
 * reuses that one block: calls that may overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 *
 *   ylt          device (or managed) memory, n >= 1 year losses
 *   return_periods, n_rp
 *                host array, 1 <= n_rp <= ARA_NOALLOC_MAX_RP, each RP >= 1
 *   pml_out, tvar_out
 *                n_rp doubles each, host or device memory
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream);
 *                the current device must be the device that holds ylt and
 *                any device output
 *
 * The first call on each device looks up the device address of the fixed
 * block (cudaGetSymbolAddress); make that first call before any stream
 * capture begins.  With host outputs the call synchronises the stream.
 * Returns ARA_OK, ARA_EINVAL (NULL or host ylt, ylt or a device output on
 * another device than the current one, n < 1, n_rp outside
 * 1..ARA_NOALLOC_MAX_RP, RP < 1) or ARA_ECUDA.  It never calls cudaMalloc,
 * cudaFree or any allocating routine. */
#define ARA_NOALLOC_MAX_RP 64
#define ARA_NOALLOC_SCRATCH_BYTES 16384
ARA_API int ara_pml_tvar_noalloc(const double *ylt, int64_t n, const double *return_periods, int32_t n_rp,
                                 double *pml_out, double *tvar_out, void *cuda_stream);

/* Counters of the last ara_run_layer* call. */
ARA_API int ara_get_stats(const ara_ctx *ctx, ara_stats *out);

/* Accumulated device times since the last reset; waits for the recorded
 * events.  reset != 0 clears the accumulators after reading. */
ARA_API int ara_get_timing(ara_ctx *ctx, ara_timing *out, int reset);

/* Message of the last failed call on this context (never NULL). */
ARA_API const char *ara_last_error(const ara_ctx *ctx);

/* Release every device buffer and the context.  NULL is ignored. */
ARA_API void ara_destroy(ara_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ARA_H */
