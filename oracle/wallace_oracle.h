/*
 * Oracle for Wallace's normal generator in the vectorised form of Brent's RANN4
 * (R. P. Brent, "A fast vectorised implementation of Wallace's normal random
 * number generator", 1997).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, sequential C restatement of
 * what one generator computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * constant table or helper with the CUDA library, and the CUDA library never
 * loads it.
 *
 * Two arithmetic modes:
 *   ORC_FP32  pool in binary32; every floating operation of the pass is one
 *             IEEE round-to-nearest operation in the order written here (the
 *             library must reproduce these values bit for bit);
 *   ORC_FP64  the same algorithm with a binary64 pool (accuracy reference).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared.
 */
#ifndef WALLACE_ORACLE_H
#define WALLACE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FP32 = 0, ORC_FP64 = 1 };
/* mode flag: Wilson-Hilferty chi-squared sample instead of Eq. 3's */
enum { ORC_CHI_WH = 0x100 };
/* mode flag: a random sign pattern per pass, matrix A D_k (Section 3) */
enum { ORC_SIGNS = 0x200 };

enum {
    ORC_OK = 0,
    ORC_EINVAL = 1,
    ORC_ENOMEM = 2,
    ORC_ECORRUPT = 4
};

typedef struct orc_gen orc_gen;

/* Scalars describing the most recent pass (or the initial pool). */
typedef struct {
    uint64_t q_lo, q_hi;   /* exact sum-of-squares integer Q (128-bit)      */
    double q;              /* Q converted to a real sum of squares          */
    double S;              /* chi-squared target drawn from the pool (Eq. 3) */
    double c;              /* scale applied by the NEXT pass, c = sqrt(S/q)  */
    float c32;             /* c rounded to binary32 (FP32 mode)             */
    double drift;          /* q_k / S_{k-1} - 1 (0 for the initial pool)     */
    int64_t passes;        /* passes done                                    */
    int status;            /* sticky ORC_* status                            */
    int bad;               /* a pool value was non-finite or |y| >= 256      */
    uint64_t lcg;          /* uniform generator state                        */
    int32_t alpha[8];      /* strides of the most recent pass                */
    int64_t gamma[8];      /* offsets of the most recent pass                */
    int64_t R;             /* values returned per pass                       */
    int64_t cursor;        /* next returned index in the current pool        */
    uint32_t signs;        /* sign pattern of the most recent pass (ORC_SIGNS) */
    double rot_c, rot_s;   /* cos and sin of the most recent pass's rotation (n = 2) */
} orc_stats;

/* ---- building blocks (exposed so the tests can pin each one) ---------- */
uint64_t orc_splitmix64(uint64_t x);
uint64_t orc_seed_state(uint32_t seed, uint32_t stream);
uint32_t orc_lcg_next(uint64_t *state);
double orc_log_w(uint64_t w);                      /* ln(w * 2^-32), 1 <= w <= 2^32 */
void orc_sincos_quarter(double g, double *s, double *c); /* sin, cos of g*pi/2, 0<=g<=1/2 */
void orc_sincos_2pi(uint32_t u, double *s, double *c);   /* sin, cos of 2*pi*u*2^-32      */
void orc_box_muller(uint32_t u1, uint32_t u2, float *a, float *b);
uint64_t orc_lcg_jump(uint64_t state, uint64_t steps);
void orc_boxmuller_stream(uint32_t seed, uint32_t stream, int64_t offset, int64_t count,
                          float mu, float sigma, float *out);
int orc_stride_candidates(int n, int64_t N, int32_t *cand);
void orc_draw_params(int n, int64_t N, uint64_t *state, int32_t *alpha, int64_t *gamma);
void orc_transform32(int n, const float *g, float c, float *y);
void orc_transform64(int n, const double *g, double c, double *y);
uint64_t orc_term32(float y, int *bad);
/* one pass from explicit parameters (no correction bookkeeping) */
void orc_pass_explicit32(int n, int64_t N, const float *x, float *y,
                         const int32_t *alpha, const int64_t *gamma, float c, uint32_t signs);
void orc_pass_explicit64(int n, int64_t N, const double *x, double *y,
                         const int32_t *alpha, const int64_t *gamma, double c, uint32_t signs);
/* n = 2 (RANN4): the rotation of one pass, and a pass with the scaled rotation */
void orc_draw_rotation(uint64_t *state, double *cs, double *sn);
void orc_pass_rot32(int64_t N, const float *x, float *y, const int32_t *alpha,
                    const int64_t *gamma, float C, float S);
void orc_pass_rot64(int64_t N, const double *x, double *y, const int32_t *alpha,
                    const int64_t *gamma, double C, double S);
/* exact sum of squares of an FP32 pool: returns 0/1 "bad" flag */
int orc_sumsq32(const float *pool, int64_t nu, uint64_t *q_lo, uint64_t *q_hi);
int orc_sumsq64(const double *pool, int64_t nu, uint64_t *q_lo, uint64_t *q_hi);
int64_t orc_returned_count(int64_t nu, double frac);

/* ---- a whole generator ------------------------------------------------- */
orc_gen *orc_create(int n, int64_t N, uint32_t seed, uint32_t stream, double frac, int mode);
/* refill the pool (Section 5, restarting) before every pass that follows a
 * multiple of `interval` passes; 0 turns it off (the default) */
void orc_set_restart(orc_gen *g, int64_t interval);
/* the pool of restart r (nu values): Box-Muller pairs from uniforms
 * [r 2^40, r 2^40 + nu) of the (seed, stream) sequence */
void orc_restart_pool(uint32_t seed, uint32_t stream, int64_t r, int64_t nu, float *pool);
int orc_pass(orc_gen *g);
int orc_fill32(orc_gen *g, float *out, int64_t count, float mu, float sigma);
int orc_fill64(orc_gen *g, double *out, int64_t count, double mu, double sigma);
void orc_get_pool32(const orc_gen *g, float *out);
void orc_get_pool64(const orc_gen *g, double *out);
void orc_get_stats(const orc_gen *g, orc_stats *st);
/* overwrite the current pool, as a user who writes over the work area would
 * (Section 8's corruption check); tests only */
void orc_set_pool32(orc_gen *g, const float *pool);
void orc_destroy(orc_gen *g);

#ifdef __cplusplus
}
#endif
#endif
