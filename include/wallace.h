/*
 * wallace.h -- C ABI of a GB300 (sm_103a) implementation of Wallace's normal
 * random number generator in the vectorised form of Brent's RANN4
 * (R. P. Brent, "A fast vectorised implementation of Wallace's normal random
 * number generator", 1997).
 *
 * One generator ("handle") keeps a pool of nu = n*N binary32 normal variates
 * in device memory, viewed as n sub-vectors of length N (Section 2).  A pass
 * (Section 2, footnote: "the process of regenerating the pool") replaces the
 * pool with
 *     x'_i[j] = c * ((2/n) * sum_k g_k - g_i),   g_k = x_k[(alpha_k j + gamma_k) mod N]
 * for j = 0..N-1 (Eq. 1 with A = (2/n)J - I, n in {4, 8}), where the strides
 * alpha_k and offsets gamma_k are redrawn every pass from the generator's own
 * uniform source (Sections 3, 7, 8; gcd rule Eq. 2) and c rescales the pool's
 * sum of squares to a chi-squared sample (Section 4, Eq. 3).  Of each new pool
 * the first R = min(floor(frac*nu), nu-1) values are returned to the user
 * (Section 6, throw-away factor f = 1/frac); the last value is never returned.
 *
 * Conventions for every call:
 *   - All compute runs in CUDA kernels on the handle's stream (default: the
 *     legacy default stream; see wallace_set_stream).  Calls are asynchronous
 *     unless stated otherwise.
 *   - Pointers documented as "device" must point to device memory of the
 *     device that was current when the handle was created, be aligned to
 *     their element size, and stay valid until the work on the handle's
 *     stream that uses them has completed.  The caller owns them.
 *   - Return value: WALLACE_OK (0) or a positive status.  Status bits found on
 *     the device (WALLACE_ECORRUPT) are sticky and surface at the next call
 *     that synchronises (wallace_sync, wallace_stats, wallace_get_pool*);
 *     they stay set until wallace_clear_error.  A failed CUDA call sets
 *     WALLACE_ECUDA, also sticky.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef WALLACE_H
#define WALLACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wallace wallace_t;

/* status codes (bit flags; a call may return several OR-ed together) */
#define WALLACE_OK        0
#define WALLACE_EINVAL    1   /* an argument is out of range                      */
#define WALLACE_ENOMEM    2   /* device or host allocation failed                 */
#define WALLACE_ECORRUPT  4   /* sum-of-squares monitor tripped (Section 8)       */
#define WALLACE_ECUDA     8   /* a CUDA runtime call failed                       */
#define WALLACE_ETIMEOUT 16   /* a bounded device-side wait gave up               */
#define WALLACE_ESTATE   32   /* call not valid in the handle's current mode      */

/* pool precision */
#define WALLACE_FP32      0   /* binary32 pool; exact integer sum of squares, binary64 scale */
#define WALLACE_FP64POOL  1   /* binary64 pool (reference mode for precision studies)        */
/* mode flag, OR-ed into either precision: the chi-squared sample of Section 4
 * by Wilson and Hilferty's cube (Abramowitz and Stegun 26.4.17),
 * S = nu (1 - a + x sqrt(a))^3 with a = 2/(9 nu), instead of Eq. 3's
 * (x + sqrt(2 nu - 1))^2 / 2 -- closer to chi-squared for small pools.  A
 * sample that is not positive marks the pool corrupt (c stays 1). */
#define WALLACE_CHI_WH    0x100
/* mode flag: a different orthogonal matrix at each pass (Section 3 prefers
 * it to a fixed A): pass k uses A D_k with D_k = diag(+-1), its pattern the
 * top n bits of one more uniform drawn after the pass's strides and offsets.
 * Breaks the fixed matrix's invariant sum(pool)/sqrt(Q) (A 1 = 1).
 * Single-generator handles only. */
#define WALLACE_MATRIX_SIGNS 0x200

/* pass kernel selection (wallace_set_variant) */
#define WALLACE_VARIANT_AUTO    0  /* pick by pool size: whole pool in shared memory when
                                      it fits; else binary32 pools (n = 4, 8) of at most
                                      2^22 values take WALLACE_VARIANT_L2RUN; else the
                                      lane-tiled (or two-phase) pass, one per launch     */
#define WALLACE_VARIANT_GATHER  1  /* direct strided gather from HBM, one pass/launch   */
#define WALLACE_VARIANT_TILED   2  /* lane-tiled gather staged in shared memory: the
                                      bulk-copy (TMA) pipeline when N % 4 == 0 and
                                      N is coprime to 15 (n = 4) or 105 (n = 8: 315
                                      lanes; pools over 64 MB take the two-CTA
                                      cluster form and write the returned values in
                                      a second, streaming kernel), else per-thread
                                      16-byte async copies (n = 4)                  */
#define WALLACE_VARIANT_FUSED   3  /* whole pool in shared memory, many passes/launch   */
#define WALLACE_VARIANT_TILED_ASYNC 4 /* lane-tiled, per-thread 16-byte async copies      */
#define WALLACE_VARIANT_TILED_TMA   5 /* lane-tiled, warp-specialised bulk (TMA) copies
                                         into a stage ring, one CTA per tile; needs
                                         N % 4 == 0 and N coprime to 15 (n = 4; else the
                                         per-thread-copy kernel runs) or to 105 (n = 8) */
#define WALLACE_VARIANT_TWOPHASE    6 /* binary32 pools the lane-tiled kernels cannot
                                         tile (n = 8 with N a multiple of 3, 5 or 7, or
                                         N % 4 != 0; n = 4 with 15 dividing N), and any
                                         n = 8 pool on request: every
                                         sub-vector un-strided into a j-ordered copy,
                                         then the transform streamed over it (2
                                         launches per pass; a third pool-sized buffer
                                         held from creation when every stride N can
                                         draw is at most 16384)                       */

#define WALLACE_VARIANT_L2RUN       7 /* binary32 pools of at most 2^23 values (n = 4 or
                                         8; (alpha + 1) N < 2^32 for every stride the
                                         pool can draw): every pass of a fill in ONE
                                         cooperative launch (up to 2^20 passes), each
                                         thread gathering its tuples straight from L2,
                                         CTAs meeting at a grid barrier after each pass,
                                         where each CTA runs the end of pass (Eq. 3)
                                         itself; for pools that stay in L2 between
                                         passes                                        */
#define WALLACE_VARIANT_TILED_CLUSTER 8 /* n = 8, the pools of the n = 8 bulk-copy pass
                                         (binary32, N % 4 == 0, N coprime to 105) on
                                         clusters of two CTAs: each holds four of the
                                         eight sub-vectors of a 315-lane x 16-lane-time
                                         tile and they exchange each tuple's half-sum
                                         through distributed shared memory; rejected
                                         (WALLACE_EINVAL) where the device cannot hold
                                         a cluster of two such CTAs                    */

/* Scalars of the most recent pass (or of the initial pool after create). */
typedef struct {
    uint64_t q_lo, q_hi;  /* exact sum-of-squares integer Q (128-bit): sum floor(y^2 2^32)
                             (FP32) or sum floor(fl(y*y) 2^64) (FP64POOL)                */
    double q;             /* Q as a real sum of squares                                  */
    double S;             /* chi-squared target from the withheld value (Eq. 3)          */
    double c;             /* scale the next pass applies, sqrt(S/q)                      */
    float c32;            /* c rounded to binary32                                       */
    double drift;         /* q_k / S_{k-1} - 1 (0 for the initial pool)                  */
    int64_t passes;       /* passes completed                                            */
    int32_t status;       /* sticky WALLACE_* bits                                       */
    int32_t bad;          /* a pool value was non-finite or |y| >= 256                   */
    uint64_t lcg;         /* uniform generator state after the strides of the most recent
                             pass were drawn (after the initial pool before any pass)    */
    int32_t alpha[8];     /* strides of the most recent pass                             */
    int64_t gamma[8];     /* offsets of the most recent pass                             */
    int64_t R;            /* values returned per pass                                    */
    int64_t cursor;       /* index in the current pool of the next value to return       */
    double kernel_ms;     /* summed pass-kernel time when timing is on                   */
    int64_t kernel_launches; /* pass kernels timed                                       */
    int64_t launches;     /* kernels launched by passes and fills (pass and drain kernels),
                             counted whether or not timing is on                         */
    uint32_t signs;       /* sign pattern of the most recent pass (WALLACE_MATRIX_SIGNS;
                             bit i: sub-vector i negated before A)                        */
    double rot_c, rot_s;  /* n = 2: cos and sin of the most recent pass's rotation        */
} wallace_stats_t;

/*
 * wallace_create -- make a generator and its initial pool.
 *   n      sub-vectors per pool, 4 or 8 (A = (2/n)J - I; Section 2, Section 9)
 *   N      sub-vector length, 4 <= N and n*N <= 2^30 (Section 2: pool of nN)
 *   seed   32-bit seed of the uniform source (Section 8)
 *   frac   returned fraction 1/f, 0 < frac <= 1 (Section 6); R must be >= 1
 *   out    receives the handle
 * The initial pool is filled on the device by Box-Muller from the uniform
 * source (Sections 5 and 8) and is not itself returned; its last value sets
 * the first chi-squared target (Eq. 3).  Allocates 2*n*round_up(N,64)
 * elements of device memory plus a small state block.
 * Errors: WALLACE_EINVAL (bad n, N, frac), WALLACE_ENOMEM, WALLACE_ECUDA.
 */
int wallace_create(int n, int64_t N, uint32_t seed, double frac, wallace_t **out);

/*
 * wallace_create_ex -- as wallace_create, plus:
 *   stream_id  appended to the seed (Section 8: DP_VRANU4 appends the
 *              processor number so that processors get different sequences)
 *   mode       WALLACE_FP32 or WALLACE_FP64POOL, optionally OR-ed with
 *              WALLACE_CHI_WH and/or WALLACE_MATRIX_SIGNS
 *   cuda_stream  cudaStream_t to run on (NULL: legacy default stream)
 */
int wallace_create_ex(int n, int64_t N, uint32_t seed, uint32_t stream_id, double frac,
                      int mode, void *cuda_stream, wallace_t **out);

/* wallace_destroy -- synchronise the handle's stream and free everything. NULL-safe. */
void wallace_destroy(wallace_t *h);

/*
 * wallace_pass -- advance one pass (Section 2, Eq. 1; Section 4, Eq. 3).
 * The R returned values of the new pool become the next values that
 * wallace_fill hands out; any values of the previous pool not yet handed
 * out are skipped.  Asynchronous.
 */
int wallace_pass(wallace_t *h);

/*
 * wallace_fill -- write the next `count` values of the returned stream,
 * mapped to N(mu, sigma^2) as mu + sigma*y (binary32 multiply, then add;
 * Section 7 and Section 8: size, mean and variance may change every call).
 *   out    device pointer to `count` floats (caller-owned)
 * Runs as many passes as needed; each pass writes its returned prefix
 * straight into `out` from the pass kernel.  Splitting a request into several
 * calls yields the same stream.  FP32 mode only (WALLACE_ESTATE otherwise).
 * Asynchronous.
 */
int wallace_fill(wallace_t *h, float *out, int64_t count, float mu, float sigma);

/* wallace_fill64 -- as wallace_fill for a WALLACE_FP64POOL handle; binary64 out. */
int wallace_fill64(wallace_t *h, double *out, int64_t count, double mu, double sigma);

/*
 * wallace_fill_host -- as wallace_fill, but `host_out` is a HOST pointer to
 * `count` floats.  The values are produced on the device in chunks and
 * copied back while the next chunk is generated.  Page-locked memory gives
 * asynchronous copies; pageable memory works but is slower.  Synchronous:
 * returns when all values are in host memory.
 */
int wallace_fill_host(wallace_t *h, float *host_out, int64_t count, float mu, float sigma);

/* wallace_set_stream -- run subsequent work on `cuda_stream` (a cudaStream_t). */
int wallace_set_stream(wallace_t *h, void *cuda_stream);

/* wallace_set_variant -- choose the pass kernel (WALLACE_VARIANT_*); all
 * variants produce bit-identical pools.  EINVAL for an unknown variant or a
 * FUSED request on a pool too large for shared memory. */
int wallace_set_variant(wallace_t *h, int variant);

/*
 * wallace_set_restart -- Section 5 (restarting): refill the pool by
 * Box-Muller from the uniform source before every pass that follows a
 * multiple of `interval` passes (counted from creation), and take the
 * chi-squared sample, scale and drift history afresh from the new pool, as at
 * creation.  Restart r = 1, 2, ... takes the uniforms at positions
 * [r 2^40, r 2^40 + n*N) of the generator's sequence, apart from the initial
 * pool and the per-pass draws, which are unchanged.  The paper suggests a
 * restart after about 1000 N returned numbers (interval ~ 1000 N / R).  The
 * refilled pool is not returned.  interval = 0 (the default) never restarts.
 * Returns WALLACE_OK or WALLACE_EINVAL (NULL handle, interval < 0).
 */
int wallace_set_restart(wallace_t *h, int64_t interval);

/*
 * wallace_set_l2_grid -- CTAs of WALLACE_VARIANT_L2RUN's launch (not part of
 * the paper's method): 0 (the default) is two per SM; larger values are
 * capped at what the device can keep resident.  Results do not depend on it.
 * Returns WALLACE_OK or WALLACE_EINVAL (NULL handle, grid < 0).
 */
int wallace_set_l2_grid(wallace_t *h, int grid);

/* wallace_set_timing -- when on, every pass kernel is bracketed by CUDA
 * events on the handle's stream; the summed time appears in kernel_ms. */
int wallace_set_timing(wallace_t *h, int on);

/* wallace_sync -- wait for the handle's stream; returns the sticky status. */
int wallace_sync(wallace_t *h);

/* wallace_stats -- synchronise and copy the scalars of the last pass. */
int wallace_stats(wallace_t *h, wallace_stats_t *out);

/*
 * wallace_get_pool -- synchronise and copy the current pool to HOST memory
 * `host_out` (nu floats, sub-vector-major: x_0[0..N-1], x_1[0..N-1], ...).
 * In FP64POOL mode each value is rounded to binary32.
 */
int wallace_get_pool(wallace_t *h, float *host_out);

/* wallace_get_pool64 -- as wallace_get_pool into nu doubles (exact in both modes). */
int wallace_get_pool64(wallace_t *h, double *host_out);

/*
 * wallace_set_pool -- overwrite the current pool from HOST memory (nu floats,
 * same layout).  Models a caller who writes over the work area; the next
 * pass's sum-of-squares check (Section 8) then reports WALLACE_ECORRUPT.
 */
int wallace_set_pool(wallace_t *h, const float *host_in);

/* wallace_clear_error -- reset the sticky status bits. */
int wallace_clear_error(wallace_t *h);

/* wallace_returned_per_pass -- R for the handle (host value, no sync). */
int64_t wallace_returned_per_pass(const wallace_t *h);

/* ---- many generators in one launch ------------------------------------ */
/*
 * A batch holds `count` independent generators (Section 9: independent
 * streams need no communication after initialisation) with their own pool
 * sizes and seeds, in one device arena.  wallace_batch_run advances every
 * generator by the same number of passes in ONE persistent kernel launch
 * (a CUDA graph: work-counter reset + kernel).  CTAs take whole generators,
 * largest pool first; small pools stay in shared memory across all passes.
 * Each generator produces exactly the values a handle made by
 * wallace_create_ex(n, N[s], seed[s], 0, frac, WALLACE_FP32, ...) would:
 * run(P1) then run(P2) equals run(P1 + P2), and both equal P passes of
 * wallace_fill with count R_s per pass.
 */
typedef struct wallace_batch wallace_batch_t;

/*
 * wallace_batch_create -- `count` >= 1 generators; N and seed are host
 * arrays of `count` values (4 <= N[s], n*N[s] <= 2^30); n in {4, 8} and
 * frac as in wallace_create.  Initial pools are made here (synchronous).
 * Errors: WALLACE_EINVAL, WALLACE_ENOMEM, WALLACE_ECUDA.
 */
int wallace_batch_create(int count, int n, const int64_t *N, const uint32_t *seed, double frac,
                         void *cuda_stream, wallace_batch_t **out);

/*
 * wallace_batch_create_ex -- as wallace_batch_create, with a mode for every
 * generator: WALLACE_FP32 optionally OR-ed with WALLACE_CHI_WH (Wilson and
 * Hilferty's chi-squared sample) and/or WALLACE_MATRIX_SIGNS (a different
 * orthogonal matrix A D_k each pass, Section 3).  Each generator then
 * produces exactly what wallace_create_ex(n, N[s], seed[s], 0, frac, mode,
 * ...) would.  WALLACE_EINVAL for any other mode.
 */
int wallace_batch_create_ex(int count, int n, const int64_t *N, const uint32_t *seed, double frac, int mode,
                            void *cuda_stream, wallace_batch_t **out);

/*
 * wallace_batch_set_restart -- Section 5 (restarting) for every generator:
 * before the pass that follows each multiple of `interval` passes (counted
 * from creation; all generators advance together), every pool is refilled
 * by Box-Muller from the uniforms its restart takes (as wallace_set_restart
 * describes) and the scale and drift history start afresh.  A run that
 * crosses restart points is split into several launches around the refills
 * (one refill launch per generator, after reading back which buffer holds
 * each pool: synchronous), with the output laid out as for one launch.
 * interval = 0 (the default) never restarts.  WALLACE_EINVAL on a NULL batch
 * or interval < 0.
 */
int wallace_batch_set_restart(wallace_batch_t *b, int64_t interval);

/* wallace_batch_destroy -- synchronise and free everything.  NULL-safe. */
void wallace_batch_destroy(wallace_batch_t *b);

/*
 * wallace_batch_run -- `passes` passes of every generator, one launch.
 *   out   device buffer, or NULL to discard the returned values.  Generator s
 *         writes its passes*R_s returned values (mu + sigma*y, pass-major) to
 *         out + wallace_batch_out_offset(b, s, passes); the total size is
 *         wallace_batch_out_offset(b, count, passes).
 * Asynchronous on the batch's stream.
 */
int wallace_batch_run(wallace_batch_t *b, int64_t passes, float *out, float mu, float sigma);

/* wallace_batch_out_offset -- passes * (sum of R over generators before s);
 * s == count gives the total.  -1 on bad arguments. */
int64_t wallace_batch_out_offset(const wallace_batch_t *b, int s, int64_t passes);

/* wallace_batch_returned_per_pass -- R_s; -1 on bad arguments. */
int64_t wallace_batch_returned_per_pass(const wallace_batch_t *b, int s);

/* wallace_batch_sync -- wait; returns the OR of every generator's status. */
int wallace_batch_sync(wallace_batch_t *b);

/* wallace_batch_stats -- synchronise and copy generator s's scalars. */
int wallace_batch_stats(wallace_batch_t *b, int s, wallace_stats_t *out);

/* wallace_batch_get_pool -- synchronise and copy generator s's pool to HOST
 * memory (n*N[s] floats, sub-vector-major). */
int wallace_batch_get_pool(wallace_batch_t *b, int s, float *host_out);

/*
 * wallace_batch_set_tuning / wallace_batch_get_tuning -- launch shape: CTAs
 * per SM (capped by occupancy), lane-times per tile of the tiled gather
 * (4 <= etarget <= 2560), and the largest pool (n*N values) kept in shared
 * memory across passes (at most ~8400 values fit; ~24500 with the bulk-copy
 * runner).  ctas_per_sm = 0 selects
 * the bulk-copy runner instead: one CTA of 608 threads per SM, pools with
 * n = 4 and 16384 <= N <= 2^28 regenerated through a warp-specialised stage
 * ring fed by bulk (TMA) copies, the others as before (etarget and fused_max
 * apply to them).
 */
int wallace_batch_set_tuning(wallace_batch_t *b, int ctas_per_sm, int etarget, int64_t fused_max);
int wallace_batch_get_tuning(const wallace_batch_t *b, int *ctas_per_sm, int *etarget,
                             int64_t *fused_max);

/*
 * wallace_batch_autotune -- pick the launch shape.  If `cache_path` (may be
 * NULL) holds an entry for this device and batch shape (count, n, frac and
 * the histogram of pool sizes), use it.  Otherwise time `trial_passes`
 * passes for each candidate (CTAs/SM in {1,2,3} or the bulk-copy runner,
 * tile in {1280,1920,2560}, shared-memory pool limit in {2048,4096,8192}) on a snapshot of the
 * generators -- the generators themselves do not advance -- keep the fastest
 * and append it to `cache_path` as one JSON object per line.  Synchronous.
 */
int wallace_batch_autotune(wallace_batch_t *b, const char *cache_path, int trial_passes);

/* ---- serving many clients by continuous batching ---------------------- */
/*
 * A server holds one generator per client (pool resident in device memory)
 * and answers fill requests (client, count, mu, sigma).  A request is
 * admitted when its client has no request in flight (each client's stream
 * stays in order) and its output buffer -- plus a second pool buffer for
 * pools too large for shared memory -- fits in the device-memory budget
 * given at creation, which also holds every client's pool.  Each scheduler
 * tick launches one persistent kernel over all admitted requests (each gets
 * the values left in its client's current pool, then up to
 * passes_per_tick passes whose returned prefixes go straight into its
 * output); requests that arrive meanwhile join at the next tick.  The values
 * a client receives do not depend on what other clients ask for: they are
 * exactly those of a handle with the same n, N, seed and frac.
 */
typedef struct wallace_server wallace_server_t;

typedef struct {
    int64_t submitted, admitted, completed, queued, active, ticks;
    int64_t values_delivered;   /* sum of the counts of completed requests     */
    int64_t hbm_budget, hbm_in_use, hbm_peak;   /* bytes                      */
    double p50_ms, p99_ms, mean_ms;   /* request latency: submit to completion */
    double elapsed_s;           /* first submit to last completion            */
    int32_t status;
    int32_t pad_;
    double host_tick_s;         /* host time spent building and enqueueing ticks */
    double host_wait_s;         /* host time blocked waiting for a tick         */
    int64_t items;              /* requests summed over ticks (work items)      */
    double mean_admit_wait_ms;  /* mean time from submit to admission           */
} wallace_server_stats_t;

/*
 * wallace_server_create -- n_clients generators (host arrays N, seed); n and
 * frac as in wallace_create.  hbm_budget_bytes bounds all device memory the
 * server uses (pools, states, request buffers); WALLACE_ENOMEM if the pools
 * alone do not fit.  Initial pools are made here (synchronous).
 */
int wallace_server_create(int n_clients, int n, const int64_t *N, const uint32_t *seed, double frac,
                          int64_t hbm_budget_bytes, void *cuda_stream, wallace_server_t **out);

/*
 * wallace_server_create_ex -- as wallace_server_create, with a mode for every
 * client's generator: WALLACE_FP32 optionally OR-ed with WALLACE_CHI_WH and/or
 * WALLACE_MATRIX_SIGNS (as for wallace_create_ex).  A client then receives
 * exactly the values of wallace_create_ex(n, N[c], seed[c], 0, frac, mode, ...).
 */
int wallace_server_create_ex(int n_clients, int n, const int64_t *N, const uint32_t *seed, double frac,
                             int mode, int64_t hbm_budget_bytes, void *cuda_stream, wallace_server_t **out);

/*
 * wallace_server_set_restart -- Section 5 (restarting) for every client, as
 * wallace_set_restart for a handle: before the pass that follows each
 * multiple of `interval` of a client's passes, its pool is refilled (on the
 * tick's stream, before the tick's kernels) after any values of its current
 * pool still owed to the request have been handed out.  interval = 0 (the
 * default) never restarts.  Only while idle; WALLACE_EINVAL otherwise.
 */
int wallace_server_set_restart(wallace_server_t *s, int64_t interval);

/* wallace_server_destroy -- synchronise and free everything.  NULL-safe. */
void wallace_server_destroy(wallace_server_t *s);

/* wallace_server_set_tuning -- passes per request per tick (>= 1), the
 * largest pool kept in shared memory across passes, CTAs per SM.
 * ctas_per_sm = 0: three CTAs per SM as before, and the requests one CTA
 * serves whose pools have n = 4 and 16384 <= N <= 2^28 run the bulk-copy
 * (TMA) runner instead, one 608-thread CTA per SM on a second stream beside
 * the others.  Only while idle. */
int wallace_server_set_tuning(wallace_server_t *s, int passes_per_tick, int64_t fused_max,
                              int ctas_per_sm);

/* wallace_server_set_tick -- what one scheduler tick gives a request (not
 * part of the paper's method): pools of up to one_cta_max_values values run on
 * one CTA per request, for up to values_per_tick / (n N) passes a tick (at
 * least one); larger pools run pass-major over all CTAs, passes_per_tick
 * passes a tick.  Defaults 2^22 and 2^20.  Only while idle; WALLACE_EINVAL
 * otherwise or on a negative value. */
int wallace_server_set_tick(wallace_server_t *s, int64_t one_cta_max_values, int64_t values_per_tick);

/* wallace_server_submit -- queue a request; returns its id (host, no GPU work). */
int wallace_server_submit(wallace_server_t *s, int client, int64_t count, float mu, float sigma,
                          int64_t *request_id);

/* wallace_server_progress -- reap finished ticks, admit, enqueue one tick.
 * Non-blocking unless every tick slot is busy. */
int wallace_server_progress(wallace_server_t *s);

/* wallace_server_drain -- progress until no request is queued or active, then
 * synchronise. */
int wallace_server_drain(wallace_server_t *s);

/* wallace_server_poll -- ids (up to max_ids) of requests completed since the
 * last poll. */
int wallace_server_poll(wallace_server_t *s, int64_t *ids, int max_ids, int *n_out);

/* wallace_server_result -- a completed request's DEVICE output (count floats,
 * owned by the server until released), count and latency in ms;
 * WALLACE_ESTATE if not completed. */
int wallace_server_result(wallace_server_t *s, int64_t id, float **dev_out, int64_t *count,
                          double *latency_ms);

/* wallace_server_release -- return a completed request's output buffer to
 * the budget. */
int wallace_server_release(wallace_server_t *s, int64_t id);

/*
 * wallace_server_run_trace -- replay n requests in real time: request k is
 * submitted at arrival_s[k] seconds after the call starts (ascending), and
 * its output is released as soon as it completes.  latency_ms (may be NULL)
 * receives each request's time from its scheduled arrival to completion.
 * Returns when all are done.
 */
int wallace_server_run_trace(wallace_server_t *s, int64_t n, const double *arrival_s,
                             const int32_t *client, const int64_t *count, const float *mu,
                             const float *sigma, double *latency_ms);

/* wallace_server_stats -- counters, memory and latency percentiles. */
int wallace_server_stats(wallace_server_t *s, wallace_server_stats_t *out);

/*
 * wallace_pass_static -- one pass that allocates nothing.  The paper has no
 * counterpart: this is a deployment entry point.
 *
 * For callers that cannot allocate device memory -- for example a plug-in
 * whose host application hands it fixed buffers and a fixed memory budget
 * and does not allow cudaMalloc, or a path where cudaMalloc's implicit
 * device-wide synchronisation is not acceptable.  Such a caller cannot
 * create a handle (wallace_create allocates the double buffer and state), so
 * here the caller keeps the pool and the per-pass parameters itself, and the
 * pass's scratch (the second pool buffer and the reduction/finaliser block)
 * lives in one fixed array of 4 * WALLACE_STATIC_MAX_VALUES + 1024 bytes
 * inside the library, present on every device that loads the library until
 * the process exits.  Neither this call nor anything it calls allocates.
 *
 *   n, N        sub-vectors and their length as in wallace_create;
 *               n*N <= WALLACE_STATIC_MAX_VALUES, else WALLACE_EINVAL
 *   pool        device, n*N floats, sub-vector-major, rows of exactly N
 *               values (no padding); read, then overwritten with the new pool
 *   alpha, gamma  host arrays of n strides and offsets for this pass
 *               (0 <= gamma < N); results match wallace_pass only when they
 *               are coprime to N as Eq. 2 requires
 *   c32         scale of this pass (the c32 a previous pass reported)
 *   out         device, receives mu + sigma*y for the first out_count values
 *               of the new pool (0 <= out_count <= n*N - 1, as a handle's R:
 *               the last value sets the next scale and is never returned;
 *               NULL if 0).  Must not overlap `pool`.
 *   result      host; receives Q, q, S and the next pass's c and c32
 *   cuda_stream stream to run on (NULL: legacy default stream)
 * The next scale comes from Eq. 3's sample only (no WALLACE_CHI_WH option),
 * and there is no drift check (Section 8): the caller keeps the previous S.
 * With the strides and offsets a handle drew, the results equal that
 * handle's pass when it uses the default chi-squared sample.
 * Synchronous: every call waits on `cuda_stream` until the pass, the copy
 * back into `pool` and the result copy have finished.  Returns WALLACE_OK,
 * WALLACE_EINVAL, WALLACE_ECUDA, or WALLACE_ECORRUPT (bad value, Q = 0 or
 * Q >= 2^64).
 *
 * The scratch array is shared by every call: calls that overlap on the GPU
 * (in flight at the same time on any streams) race and give wrong results.
 * The block that must start at zero is cleared at the start of each call.
 * The first call on a device looks up the array's device address with that
 * device current; make it before any stream capture begins.
 */
#define WALLACE_STATIC_MAX_VALUES (1 << 20)

typedef struct {
    uint64_t q_lo, q_hi;  /* exact sum of squares of the new pool (128-bit)   */
    double q;             /* Q * 2^-32                                         */
    double S;             /* chi-squared target from the new pool's last value */
    double c;             /* scale for the next pass, sqrt(S/q)                */
    float c32;            /* c rounded to binary32                             */
    int32_t bad;          /* a value was non-finite or |y| >= 256              */
    int32_t status;       /* WALLACE_* bits found by the pass                  */
} wallace_pass_result_t;

int wallace_pass_static(int n, int64_t N, float *pool, const int32_t *alpha, const int64_t *gamma,
                        float c32, float *out, int64_t out_count, float mu, float sigma,
                        wallace_pass_result_t *result, void *cuda_stream);

/*
 * wallace_boxmuller_fill -- the Box-Muller method as a stand-alone generator,
 * the comparison point of the paper (its abstract and Section 1 measure RANN4
 * against the Box-Muller and Polar methods).  Writes values
 * [offset, offset + count) of the Box-Muller stream of (seed, stream_id):
 * pair p is formed from uniforms 2p and 2p+1 of the generator's uniform
 * source (u1 = (U+1) 2^-32, u2 = U' 2^-32; r = sqrt(-2 ln u1),
 * y = (r cos 2 pi u2, r sin 2 pi u2)), each mapped to mu + sigma*y (binary32
 * multiply, then add).  Values [0, n*N) of a stream are the initial pool of
 * the Wallace generator with the same seed and stream id (Sections 5 and 8).
 *   seed, stream_id as for wallace_create_ex
 *   offset      first value index, >= 0
 *   out         device, count floats, written in order
 *   count       >= 0
 *   exact       1: binary64 arithmetic with the library's own series, bit-
 *               identical to the initial pool; 0: binary32 with CUDA's logf,
 *               log1pf and sincospif (within a few binary32 ulps of exact)
 *   cuda_stream stream to run on (NULL: legacy default stream)
 * Asynchronous on cuda_stream; no state, no allocation.  Returns WALLACE_OK,
 * WALLACE_EINVAL (negative offset or count, NULL out, offset too large) or
 * WALLACE_ECUDA (launch failure).
 */
int wallace_boxmuller_fill(uint32_t seed, uint32_t stream_id, int64_t offset, float *out,
                           int64_t count, float mu, float sigma, int exact, void *cuda_stream);

/*
 * wallace_selftest_bounded_wait -- exercises the bounded device-side wait
 * that every shared-memory barrier wait of the bulk-copy kernels uses (not a
 * part of the paper's method: the library's own failure detection).  One
 * CTA on the current device waits on a barrier that nothing arrives at, which
 * must give up after its cycle budget (about one second), and on a barrier
 * whose phase has completed, which must return at once.  Synchronous.
 * Returns WALLACE_ETIMEOUT when the first wait gave up as designed (the
 * context stays usable), WALLACE_OK if it did not, WALLACE_ECUDA on a CUDA
 * error.  *completed_ok (may be NULL) receives 1 when the second wait
 * returned.
 */
int wallace_selftest_bounded_wait(int *completed_ok);

/* wallace_strerror -- static text for a status code (lowest set bit). */
const char *wallace_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* WALLACE_H */
