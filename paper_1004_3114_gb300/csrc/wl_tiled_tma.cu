// One pass of Wallace's generator (Eq. 1 of Brent's RANN4 paper; n = 4,
// binary32 pool, N a multiple of 4) as a warp-specialised lane-tiled gather.
//
// Lane geometry as in wl_tiled.cu: L = lcm(alpha_i) lanes, lane l starting at
// J_l = ceil(l N / L); a tile of T lane times reads, per sub-vector i,
// m_i = L / alpha_i contiguous spans of alpha_i T values (span p starts at
// ceil(p N / m_i) + alpha_i t0 + gamma_i mod N) and uses every value.  With
// strides drawn from the odd divisors of 45, L = 45 and a tile is 45 lanes by
// T = 64 lane times: at most 32 spans of 0.75 to 11.5 KB.
//
// Pipeline (one CTA per SM, persistent; tiles handed out dynamically from a
// per-generator counter that the end-of-pass finaliser resets):
//   producer warps -- for each span of the tile: its address, its 16-byte
//                     alignment lead (stored for the consumers), its byte
//                     count, and one bulk copy (cp.async.bulk, the TMA engine;
//                     two for a span that wraps past the end of its row) into
//                     a ring of shared-memory stages (3 for n = 4, 2 for n = 2), completing on
//                     the stage's "full" mbarrier.  Span sp belongs to lane
//                     sp / 4 of producer warp sp % 4: a single warp issues
//                     bulk copies too slowly for spans of about 1 KB;
//   consumer warps -- wait for the stage; each warp owns whole lanes (three
//                     of the 45) and walks their lane times 64 at a time (two
//                     independent values per thread), so lane-table reads are
//                     broadcasts done once per lane,
//                     shared-memory gathers have odd stride alpha_i (no bank
//                     conflicts) and every store instruction writes 128
//                     contiguous bytes; transform, store the new pool and the
//                     returned values, accumulate the exact sum of squares,
//                     then release the stage on its "empty" mbarrier.
// Every wait is bounded by a cycle budget; on expiry the CTA records
// WALLACE_ETIMEOUT in the state, stops issuing work, waits (bounded) for its
// copies still in flight, and leaves.
#include <math.h>

#include "wl_common.cuh"
#include "wl_launch.h"
#include "wl_tma_common.cuh"

namespace {

using namespace wl_tma;

// n = 2: also the scaled rotation C = c cos, S = c sin of this pass.
__device__ __forceinline__ float tm_wait_prev(WlDevState *st, volatile float *s_c, float &C, float &S)
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    if (threadIdx.x == 0) {
        s_c[0] = st->next.c32;
        s_c[1] = st->next.rc32;
        s_c[2] = st->next.rs32;
    }
    __syncthreads();
    C = s_c[1];
    S = s_c[2];
    return s_c[0];
}

// SG: the generator draws a sign pattern each pass (matrix A D_k); the
// fixed-matrix kernel has no trace of it.  NSUB: 4 (A = J/2 - I) or 2
// (RANN4's rotation, strides from {3,5} and {7,11}: L = alpha beta <= 55 lanes,
// T = 11520 / L lane times per tile, rounded down to a multiple of 64).
template <bool SG, int NSUB>
__global__ void __launch_bounds__(TM_THREADS, 1) tma_kernel(WlPassArgs a, double rnu)
{
    constexpr int LMAXN = NSUB == 4 ? TM_LMAX : TM_LMAX2;     // lanes, and lane-table row stride
    constexpr int ET = tm_et<NSUB>();          // lane-times per tile, at most
    constexpr int STG = tm_stages<NSUB>();     // ring stages
    constexpr int SW = tm_stage_words<NSUB>(), SDW = tm_stage_data_words<NSUB>();
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_full[STG];
    __shared__ __align__(8) uint64_t bar_empty[STG];
    __shared__ __align__(8) uint64_t bar_tile[STG];   // a stage's tile index is published
    __shared__ volatile int s_stage_tile[STG];
    __shared__ uint64_t red[3 * (TM_THREADS / 32 + 1)];
    __shared__ volatile int s_abort;

    // Launched as a programmatic dependent of the previous pass: the CTAs
    // start while that pass drains.  Everything up to tm_wait_prev() uses only
    // this pass's strides, drawn two finalisers back (slot pass & 1, final
    // since the pass before the previous one completed); the pool and the
    // scale c are read after the wait.
    WlDevState *st = a.st;
    const float *__restrict__ src = (const float *)a.src;
    float *__restrict__ dst = (float *)a.dst;
    const int64_t N = a.N, Np = a.Np;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // one warp per CTA reads the strides and shares them: every CTA starts at
    // once, and 600 threads each loading the same few words would queue on
    // one L2 slice
    __shared__ int64_t s_gam[NSUB];
    __shared__ int s_alpha[NSUB];
    __shared__ uint32_t s_signs;
    __shared__ volatile float s_c[3];
    if (warp == 0) {
        const WlStrides *cur = &st->ahead[a.pass & 1];
        if (lane < NSUB)
            s_alpha[lane] = __ldcg(&cur->alpha[lane]);
        else if (lane < 2 * NSUB)
            s_gam[lane - NSUB] = (int64_t)__ldcg((const long long *)&cur->gamma[lane - NSUB]);
        else if (lane == 2 * NSUB)
            s_signs = SG ? __ldcg(&cur->signs) : 0u;
    }
    __syncthreads();
    const uint32_t signs = SG ? s_signs : 0u;
    int alpha[NSUB];
    int64_t gam[NSUB];
#pragma unroll
    for (int i = 0; i < NSUB; i++) {
        alpha[i] = s_alpha[i];
        gam[i] = s_gam[i];
    }
    float c, rC = 0.f, rS = 0.f;
    float *out = (float *)a.out;
    const float mu = (float)a.mu, sigma = (float)a.sigma;
    const int64_t w0 = a.w0, w1 = a.w1;

    // n = 4: L = lcm of the strides when all divide 45 (3^e3 5^e5).  n = 2:
    // L = alpha beta for alpha in {3, 5}, beta in {7, 11}.  Any other stride
    // sends the pass to the plain gather below (n = 2 with N a multiple of 15
    // or 77; the host sends n = 4 pools with other strides elsewhere).
    int L;
    bool tileable;
    if constexpr (NSUB == 4) {
        int e3 = 0, e5 = 0;
        tileable = true;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int al = alpha[i];
            if (al == 3 || al == 15)
                e3 = max(e3, 1);
            if (al == 9 || al == 45)
                e3 = 2;
            if (al == 5 || al == 15 || al == 45)
                e5 = 1;
            tileable &= al == 3 || al == 5 || al == 9 || al == 15 || al == 45;
        }
        L = tileable ? (e3 == 2 ? 9 : (e3 == 1 ? 3 : 1)) * (e5 ? 5 : 1) : TM_LMAX + 1;
    } else {
        tileable = (alpha[0] == 3 || alpha[0] == 5) && (alpha[1] == 7 || alpha[1] == 11);
        L = tileable ? alpha[0] * alpha[1] : TM_LMAX2 + 1;
    }
    int m[NSUB], sb[NSUB + 1];
    sb[0] = 0;
#pragma unroll
    for (int i = 0; i < NSUB; i++) {
        m[i] = tileable ? tm_divc(L, alpha[i]) : 0;
        sb[i + 1] = sb[i] + m[i];
    }
    const int nspans = sb[NSUB];

    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;

    if (!tileable || nspans > TM_MAXSPANS || N < TM_MIN_N || (N & 3)) {
        // plain strided gather for this pass (strides with a larger lcm)
        c = tm_wait_prev(st, s_c, rC, rS);
        const int64_t G = (int64_t)gridDim.x * blockDim.x;
        int64_t j = (int64_t)blockIdx.x * blockDim.x + tid;
        int64_t idx[NSUB], stp[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            idx[i] = (int64_t)(((uint64_t)alpha[i] * (uint64_t)(j < N ? j : 0) + (uint64_t)gam[i]) % (uint64_t)N);
            stp[i] = (int64_t)(((uint64_t)alpha[i] * (uint64_t)G) % (uint64_t)N);
        }
        for (; j < N; j += G) {
            float g[NSUB], y[NSUB];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                g[i] = wl_sgn(src[i * Np + idx[i]], signs, i);
                idx[i] += stp[i];
                if (idx[i] >= N)
                    idx[i] -= N;
            }
            if constexpr (NSUB == 4)
                wl_xform4(g, c, y);
            else
                wl_xform2(g, rC, rS, y);
#pragma unroll
            for (int k = 0; k < NSUB; k++) {
                dst[k * Np + j] = y[k];
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                int64_t q = k * N + j;
                if (q >= w0 && q < w1)
                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
            }
        }
    } else {
        // n = 2: whole 64-time chunks (a consumer thread takes t and t + 32)
        const int T = NSUB == 4 ? tm_divc(ET, L) : (tm_divc(ET, L) & ~63);
        int SL[NSUB], slot0[NSUB];
        slot0[0] = 0;
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            SL[i] = (alpha[i] * T + 8 + 3) & ~3;   // 16-byte aligned slots; wrap copies need +6
            if (i < NSUB - 1)
                slot0[i + 1] = slot0[i] + m[i] * SL[i];
        }
        float *stage0 = smem;
        int *common = (int *)(smem + STG * SW);
        int *J = common;
        int *lanebase = J + (TM_LMAX2 + 1);
        int *spanC = lanebase + 4 * TM_LMAX;

        // ceil(l N / L) and ceil(p N / m_i) as l (N / L) + ceil(l (N mod L) / L):
        // 32-bit arithmetic (N < 2^31, l (N mod L) < L^2)
        const int N32 = (int)N;
        for (int l = tid; l <= L; l += TM_THREADS) {
            const int qN = tm_divc(N32, L), rN = N32 - qN * L;
            J[l] = l * qN + tm_divc(l * rN + L - 1, L);
        }
        for (int s = tid; s < nspans; s += TM_THREADS) {
            const int i = tm_sub<NSUB>(s, sb);
            const int p = s - sb[i], mi = m[i];
            const int qN = tm_divc(N32, mi), rN = N32 - qN * mi;
            spanC[s] = p * qN + tm_divc(p * rN + mi - 1, mi);
        }
        if (tid == 0) {
            for (int s = 0; s < STG; s++) {
                mbar_init(smem_u32(&bar_full[s]), 32 * TM_PROD_WARPS);
                mbar_init(smem_u32(&bar_empty[s]), TM_CONS_WARPS);
                mbar_init(smem_u32(&bar_tile[s]), 1);
            }
            s_abort = 0;
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        __syncthreads();
        // per lane and sub-vector: slot offset of the lane's first value,
        // packed with the index of the span that holds it (span < 32)
        for (int e = tid; e < NSUB * L; e += TM_THREADS) {
            int i = tm_divc(e, L), l = e - i * L;
            int w = tm_divc(l, m[i]), p = l - w * m[i];
            int64_t r = (int64_t)alpha[i] * J[l] - (int64_t)w * N - spanC[sb[i] + p];
            lanebase[i * LMAXN + l] = ((slot0[i] + p * SL[i] + (int)r) << 5) | (sb[i] + p);
        }
        __syncthreads();
        c = tm_wait_prev(st, s_c, rC, rS);
        const int maxlen = tm_divc(N32 + L - 1, L);
        const int ntiles = (maxlen + T - 1) / T;

        if (warp >= TM_CONS_WARPS) {
            // ---------------- producer warps ----------------
            // span sp belongs to this lane for the whole kernel
            const int sp = (warp - TM_CONS_WARPS) + TM_PROD_WARPS * lane;
            const bool owner = sp < nspans;
            int sp_i = 0, sp_alpha = 0;
            int64_t sp_gam = 0, sp_C = 0;
            uint32_t sp_doff = 0;
            const float *sp_row = src;
            if (owner) {
                sp_i = tm_sub<NSUB>(sp, sb);
                const int sp_p = sp - sb[sp_i];
                sp_alpha = alpha[sp_i];
                sp_gam = gam[sp_i];
                sp_C = spanC[sp];
                sp_doff = 4u * (uint32_t)(slot0[sp_i] + sp_p * SL[sp_i]);
                sp_row = src + (int64_t)sp_i * Np;
            }
            const uint32_t stage_base = smem_u32(stage0);
            int issued[STG];
#pragma unroll
            for (int s = 0; s < STG; s++)
                issued[s] = 0;
            const int pw = warp - TM_CONS_WARPS;
            for (int it = 0;; it++) {
                const int s = it % STG;
                const int k = it / STG;
                if (s_abort)
                    break;
                if (k > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (uint32_t)((k - 1) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                // tiles are handed out dynamically: producer warp 0 takes the
                // next one from the generator's counter and publishes it
                if (pw == 0) {
                    if (lane == 0) {
                        s_stage_tile[s] = (int)atomicAdd(&st->tile_ctr, 1u);
                        mbar_arrive(smem_u32(&bar_tile[s]));
                    }
                    __syncwarp();
                } else if (!mbar_wait(smem_u32(&bar_tile[s]), (uint32_t)(k & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int tile = s_stage_tile[s];
                if (tile >= ntiles) {
                    // no more tiles: release the consumers without data
                    mbar_arrive(smem_u32(&bar_full[s]));
                    issued[s] = k + 1;
                    break;
                }
                const int t0 = tile * T;
                const int Tt = min(T, maxlen - t0);
                int *lead = (int *)(stage0 + s * SW + SDW);
                const uint32_t full = smem_u32(&bar_full[s]);
                const uint32_t d = stage_base + 4u * (uint32_t)(s * SW) + sp_doff;
                int64_t addr = 0;
                int len = 0, as = 0;
                uint32_t bytes = 0;
                bool wrap = false;
                if (owner) {
                    addr = sp_C + (int64_t)sp_alpha * t0 + sp_gam;   // < 3N
                    if (addr >= N)
                        addr -= N;
                    if (addr >= N)
                        addr -= N;
                    len = sp_alpha * Tt;
                    as = (int)addr & ~3;
                    lead[sp] = (int)addr - as;
                    wrap = addr + len > N;
                    bytes = wrap ? 4u * (uint32_t)((int)N - as) +
                                       4u * (uint32_t)(((int)(addr + len - N) + 3) & ~3)
                                 : 16u * (uint32_t)(((int)addr - as + len + 3) >> 2);
                }
                uint32_t total = bytes;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    total += __shfl_xor_sync(0xffffffffu, total, off);
                if (lane == 0)
                    mbar_expect_tx(full, total);
                __syncwarp();
                if (owner) {
                    if (!wrap) {
                        bulk_g2s(d, sp_row + as, bytes, full);
                    } else {
                        const int e2 = ((int)(addr + len - N) + 3) & ~3;
                        bulk_g2s(d, sp_row + as, 4u * (uint32_t)((int)N - as), full);
                        bulk_g2s(d + 4u * (uint32_t)((int)N - as), sp_row, 4u * (uint32_t)e2, full);
                    }
                }
                mbar_arrive(full);
                issued[s] = k + 1;
            }
            // copies still in flight must land before the CTA leaves
            for (int s = 0; s < STG; s++)
                if (issued[s] > 0 && !mbar_wait(smem_u32(&bar_full[s]), (uint32_t)((issued[s] - 1) & 1)))
                    atomicOr(&st->status, WL_ETIMEOUT);
        } else {
            // ---------------- consumer warps ----------------
            float *dstk[NSUB], *outk[NSUB];
            int mode[NSUB];   // 0: none of sub-vector k is returned, 1: all, 2: check each value
#pragma unroll
            for (int k = 0; k < NSUB; k++) {
                const int64_t q0 = k * N, q1 = q0 + N;
                mode[k] = (q1 <= w0 || q0 >= w1) ? 0 : ((q0 >= w0 && q1 <= w1) ? 1 : 2);
                dstk[k] = dst + k * Np;
                outk[k] = mode[k] == 1 ? out + (q0 - w0) : out;
            }
            uint32_t emax = 0;
            for (int it = 0;; it++) {
                const int s = it % STG;
                const int k = it / STG;
                if (s_abort)
                    break;
                if (!mbar_wait(smem_u32(&bar_full[s]), (uint32_t)(k & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int tile = s_stage_tile[s];
                if (tile >= ntiles)
                    break;
                const int t0 = tile * T;
                const int Tt = min(T, maxlen - t0);
                const float *sdata = stage0 + s * SW;
                const int *lead = (const int *)(sdata + SDW);
                uint64_t tl = 0;   // this tile's terms: at most 32 per thread, each below 2^48
                if constexpr (NSUB == 2) {
                    // lanes x 64-time chunks dealt round-robin over the
                    // consumer warps (21 to 55 lanes do not split evenly);
                    // the deal continues from tile to tile (item i of tile k
                    // goes to warp (k nitems + i) mod 15), so the extra items
                    // of a tile fall on different warps each time.  item =
                    // l nch + ch, stepped by the warp count without a division
                    const int nch = T >> 6, nitems = L * nch;
                    const int dq = tm_divc(TM_CONS_WARPS, nch), dr = TM_CONS_WARPS - dq * nch;
                    int item0 = warp - (int)(((uint32_t)tile * (uint32_t)nitems) % TM_CONS_WARPS);
                    item0 += item0 < 0 ? TM_CONS_WARPS : 0;
                    int l = tm_divc(item0, nch), ch = item0 - l * nch;
                    for (int item = item0; item < nitems;
                         item += TM_CONS_WARPS, l += dq + (ch + dr >= nch ? 1 : 0),
                         ch = ch + dr >= nch ? ch + dr - nch : ch + dr) {
                        const int jl = J[l];
                        const int tmax = min(Tt, J[l + 1] - jl - t0);
                        const int t = (ch << 6) + lane;
                        if (t >= tmax)
                            continue;
                        const float *gp[2];
#pragma unroll
                        for (int i = 0; i < 2; i++) {
                            const int lb = lanebase[i * LMAXN + l];
                            gp[i] = sdata + (lb >> 5) + lead[lb & 31];
                        }
                        const bool v2 = t + 32 < tmax;
                        float g[2], h[2], y[2], z[2];
#pragma unroll
                        for (int i = 0; i < 2; i++) {
                            g[i] = gp[i][alpha[i] * t];
                            h[i] = v2 ? gp[i][alpha[i] * (t + 32)] : 0.f;
                        }
                        wl_xform2(g, rC, rS, y);
                        wl_xform2(h, rC, rS, z);
                        const int64_t j = (int64_t)jl + t0 + t;
#pragma unroll
                        for (int kk = 0; kk < 2; kk++) {
                            dstk[kk][j] = y[kk];
                            if (v2) dstk[kk][j + 32] = z[kk];
                            tl += term32(y[kk], emax);
                            if (v2) tl += term32(z[kk], emax);
                            if (mode[kk] == 1) {
                                outk[kk][j] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                                if (v2) outk[kk][j + 32] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
                            } else if (mode[kk] == 2) {
                                int64_t q = kk * N + j;
                                if (q >= w0 && q < w1)
                                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                                q += 32;
                                if (v2 && q >= w0 && q < w1)
                                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
                            }
                        }
                    }
                } else
                for (int l = warp; l < L; l += TM_CONS_WARPS) {
                    const int jl = J[l];
                    const int tmax = min(Tt, J[l + 1] - jl - t0);   // lane times of lane l in this tile
                    const float *gp[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const int lb = lanebase[i * LMAXN + l];
                        gp[i] = sdata + (lb >> 5) + lead[lb & 31];
                    }
                    const int64_t jb = (int64_t)jl + t0;
                    for (int t = lane; t < tmax; t += 64) {
                        const bool v2 = t + 32 < tmax;
                        float g[4], h[4], y[4], z[4];
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            g[i] = gp[i][alpha[i] * t];
                            h[i] = v2 ? gp[i][alpha[i] * (t + 32)] : 0.f;
                            if (SG) {   // the pass's matrix is A D_k
                                g[i] = wl_sgn(g[i], signs, i);
                                h[i] = wl_sgn(h[i], signs, i);
                            }
                        }
                        wl_xform4(g, c, y);
                        wl_xform4(h, c, z);
                        const int64_t j = jb + t;
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            dstk[kk][j] = y[kk];
                            if (v2) dstk[kk][j + 32] = z[kk];
                            tl += term32(y[kk], emax);
                            if (v2) tl += term32(z[kk], emax);
                            if (mode[kk] == 1) {
                                outk[kk][j] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                                if (v2) outk[kk][j + 32] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
                            } else if (mode[kk] == 2) {
                                int64_t q = kk * N + j;
                                if (q >= w0 && q < w1)
                                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                                q += 32;
                                if (v2 && q >= w0 && q < w1)
                                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
                            }
                        }
                    }
                }
                // a CTA may take any number of tiles: carry into 128 bits
                lo += tl;
                hi += lo < tl ? 1ull : 0ull;
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(smem_u32(&bar_empty[s]));
            }
            bad = emax >= 135u ? 1u : 0u;
        }
    }

    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st))
        wl_finalise_cta(st, NSUB, N, a.nu, rnu, &dst[wl_last_phys(NSUB, N, Np)], SG ? 1 : 0);
}

bool g_tma_configured[3] = {false, false, false};

} // namespace

bool wl_tma_supported(int n, int64_t N, int fp64, int sm_count)
{
    // lane starts, span starts and slot offsets are held in 32-bit integers
    (void)sm_count;
    // n = 4: N coprime to 15, so every stride divides 45 (other N take the
    // per-thread tiled kernel, whose lanes go up to 315).  n = 2: any N; the
    // rare N whose RANN4 pair is excluded (a multiple of 15 or 77) runs the
    // in-kernel plain gather.
    const bool strides45 = n == 4 ? (N % 3 != 0 && N % 5 != 0) : true;
    return (n == 4 || n == 2) && !fp64 && strides45 && N >= TM_MIN_N && (N & 3) == 0 &&
           N <= ((int64_t)1 << 28);
}

cudaError_t wl_launch_tma(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream)
{
    const size_t smem = a.n == 2 ? tm_smem_bytes<2>() : tm_smem_bytes<4>();
    const int which = a.n == 2 ? 2 : (signs ? 1 : 0);
    auto kern = which == 2 ? tma_kernel<false, 2> : (which == 1 ? tma_kernel<true, 4> : tma_kernel<false, 4>);
    if (!g_tma_configured[which]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        g_tma_configured[which] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sm_count);
    cfg.blockDim = dim3(TM_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const double rnu = sqrt(2.0 * (double)a.nu - 1.0);   // IEEE square root: correctly rounded
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, rnu);
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}
