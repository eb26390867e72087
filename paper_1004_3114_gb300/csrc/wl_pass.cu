// One pass of Wallace's generator by direct strided gather (Eq. 1 of Brent's
// RANN4 paper): thread t handles j = t, t + G, t + 2G, ... and reads
// g_i = x_i[(alpha_i j + gamma_i) mod N] straight from global memory.  As in
// the paper's vector loop (Section 7), no modulo is taken inside the loop:
// each index advances by alpha_i G mod N with one conditional subtraction.
// Works for every n, N and both pool precisions; the lane-tiled kernel
// (wl_tiled.cu) is the fast path for large binary32 pools.
#include "wl_common.cuh"
#include "wl_launch.h"

namespace {

// IDENT: src already holds g_i in j order (the two-phase pass below):
// index j itself, one unit-stride read per sub-vector.
template <int NSUB, typename T, bool IDENT = false>
__global__ void __launch_bounds__(256) gather_kernel(WlPassArgs a)
{
    __shared__ uint64_t red[3 * 8];
    WlDevState *st = a.st;
    const T *__restrict__ src = (const T *)a.src;
    T *__restrict__ dst = (T *)a.dst;
    const int64_t N = a.N, Np = a.Np;
    constexpr bool f64 = sizeof(T) == 8;
    const T c = f64 ? (T)st->next.c64 : (T)st->next.c32;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t idx[NSUB], step[NSUB];
#pragma unroll
    for (int i = 0; i < NSUB; i++) {
        if constexpr (IDENT) {
            idx[i] = j;
            step[i] = G;
        } else {
            int64_t al = st->next.alpha[i], ga = st->next.gamma[i];
            idx[i] = (int64_t)(((uint64_t)al * (uint64_t)(j < N ? j : 0) + (uint64_t)ga) % (uint64_t)N);
            step[i] = (int64_t)(((uint64_t)al * (uint64_t)G) % (uint64_t)N);
        }
    }
    T *out = (T *)a.out;
    const T mu = (T)a.mu, sigma = (T)a.sigma;
    const uint32_t signs = st->next.signs;
    const T rC = f64 ? (T)st->next.rc64 : (T)st->next.rc32;   // n = 2: rotation with the scale
    const T rS = f64 ? (T)st->next.rs64 : (T)st->next.rs32;
    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    for (; j < N; j += G) {
        T g[NSUB], y[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            g[i] = wl_sgn(src[i * Np + idx[i]], signs, i);
            idx[i] += step[i];
            if (!IDENT && idx[i] >= N)
                idx[i] -= N;
        }
        if constexpr (sizeof(T) == 8) {
            if constexpr (NSUB == 2)
                wl_xform2d(g, rC, rS, y);
            else if constexpr (NSUB == 4)
                wl_xform4d(g, c, y);
            else
                wl_xform8d(g, c, y);
        } else {
            if constexpr (NSUB == 2)
                wl_xform2(g, rC, rS, y);
            else if constexpr (NSUB == 4)
                wl_xform4(g, c, y);
            else
                wl_xform8(g, c, y);
        }
#pragma unroll
        for (int k = 0; k < NSUB; k++) {
            dst[k * Np + j] = y[k];
            int64_t q = k * N + j;
            if constexpr (sizeof(T) == 8) {
                uint64_t tl, th;
                wl_term64(y[k], tl, th, bad);
                wl_add128(lo, hi, tl, th);
                if (q >= a.w0 && q < a.w1)
                    out[q - a.w0] = __dadd_rn(mu, __dmul_rn(sigma, y[k]));
            } else {
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                if (q >= a.w0 && q < a.w1)
                    out[q - a.w0] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
            }
        }
    }
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        double x = (double)__ldcg(&dst[wl_phys(a.nu - 1, N, Np)]);
        wl_finalise(st, a.n, N, a.nu, x, f64, WL_FIN_PASS);
    }
}

// Phase 1 of the two-phase pass: tmp_i[j] = x_i[(alpha_i j + gamma_i) mod N]
// for every sub-vector, with unit-stride reads and writes.  For one
// sub-vector the alpha lanes l (starting at J_l = ceil(l N / alpha)) read, at
// lane time t, the alpha consecutive addresses alpha t + gamma + [0, alpha)
// mod N, lane l the one at offset r_l = alpha J_l - l N (the r_l are a
// permutation of 0..alpha-1 since gcd(alpha, N) = 1; Eq. 2).  A tile of TT
// lane times is therefore one contiguous block of alpha TT values, loaded
// into shared memory, and alpha runs of TT values in j order, written from
// it.  Work items (sub-vector, tile) are dealt over the grid; inside a tile,
// (lane, 256-time chunk) items over the warps.
#define US_THREADS 256
// values per block: 64 KB of shared memory, three CTAs per SM
template <typename T>
__host__ __device__ constexpr int64_t us_bmax() { return sizeof(T) == 8 ? WL_TWOPHASE_MAX_STRIDE / 2 : WL_TWOPHASE_MAX_STRIDE; }

template <typename T>
__global__ void __launch_bounds__(US_THREADS) unstride_kernel(const T *__restrict__ src, T *__restrict__ tmp,
                                                               const WlDevState *st, int n, int64_t N,
                                                               int64_t Np)
{
    extern __shared__ __align__(16) unsigned char usm[];
    T *blk = (T *)usm;
    constexpr int64_t US_BMAX = us_bmax<T>();
    int64_t pre[9];
    pre[0] = 0;
    for (int i = 0; i < n; i++) {
        const int64_t al = st->next.alpha[i];
        const int64_t TT = al < US_BMAX ? US_BMAX / al : 1;
        const int64_t maxlen = (N + al - 1) / al;
        pre[i + 1] = pre[i] + (maxlen + TT - 1) / TT;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t w = blockIdx.x; w < pre[n]; w += gridDim.x) {
        int i = 0;
        while (w >= pre[i + 1])
            i++;
        const int64_t al = st->next.alpha[i], ga = st->next.gamma[i];
        const int64_t TT = al < US_BMAX ? US_BMAX / al : 1;
        const int64_t maxlen = (N + al - 1) / al;
        const int64_t t0 = (w - pre[i]) * TT;
        const int Tt = (int)min(TT, maxlen - t0);
        int64_t a0 = al * t0 + ga;   // < 3N
        if (a0 >= N)
            a0 -= N;
        if (a0 >= N)
            a0 -= N;
        const int blen = (int)min(al * Tt, N - al * t0);
        const T *row = src + (int64_t)i * Np;
        __syncthreads();   // the previous tile's readers are done
        // value e of the block goes to blk[lead + e].  16-byte async copies of
        // the block's aligned cover; when the block wraps past N, only the
        // whole chunks below N (the rest of the cover would land where the
        // wrapped values go), and the values from the last whole chunk up to
        // N and the wrapped ones from the row start, one copy per value.  A
        // block that does not wrap may read a few values past its end (the
        // row pitch leaves room past N) into unused words.
        constexpr int VPC = 16 / sizeof(T);
        const int64_t a0s = a0 & ~(int64_t)(VPC - 1);
        const int lead = (int)(a0 - a0s);
        const bool wraps = a0 + blen > N;
        const int nchunk = wraps ? (int)((N - a0s) / VPC) : (int)((a0 + blen - a0s + VPC - 1) / VPC);
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(blk);
        for (int ck = threadIdx.x; ck < nchunk; ck += US_THREADS)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sbase + 16u * (uint32_t)ck),
                         "l"(row + a0s + (int64_t)ck * VPC)
                         : "memory");
        if (wraps) {
            // positions nchunk VPC .. lead + blen - 1: row[a0s + p] below N, then row[p - (N - a0s)]
            const int p0 = nchunk * VPC, p1 = lead + blen, pN = (int)(N - a0s);
            for (int q = p0 + (int)threadIdx.x; q < p1; q += US_THREADS)
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(
                                 sbase + (uint32_t)sizeof(T) * (uint32_t)q),
                             "l"(q < pN ? row + a0s + q : row + (q - pN)), "n"(sizeof(T))
                             : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        T *out = tmp + (int64_t)i * Np;
        const int nch = (Tt + 255) >> 8;
        const int items = (int)al * nch;
        // 32-bit lane arithmetic: N < 2^31 and l rm < alpha^2 <= 2^28 (a
        // 64-bit division costs several times a 32-bit one here)
        const int al32 = (int)al, N32 = (int)N;
        const int q = N32 / al32, rm = N32 - q * al32;
        for (int it = warp; it < items; it += US_THREADS / 32) {
            const int l = it / nch, ch = it - l * nch;
            // J_l = l q + ceil(l rm / al); lane length J_{l+1} - J_l
            const int64_t Jl = (int64_t)l * q + (l * rm + al32 - 1) / al32;
            const int64_t Jn = (int64_t)(l + 1) * q + ((l + 1) * rm + al32 - 1) / al32;
            const int rl = (int)(al * Jl - (int64_t)l * N);
            const int tend = (int)min((int64_t)min(Tt, (ch + 1) << 8), Jn - Jl - t0);
            for (int t = (ch << 8) + lane; t < tend; t += 32)
                out[Jl + t0 + t] = blk[lead + rl + (int)al * t];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) drain_kernel(const T *__restrict__ pool, int64_t N,
                                                    int64_t Np, int64_t pos, int64_t count,
                                                    T *__restrict__ out, double mu, double sigma)
{
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += G) {
        T y = pool[wl_phys(pos + k, N, Np)];
        if constexpr (sizeof(T) == 8)
            out[k] = __dadd_rn(mu, __dmul_rn(sigma, y));
        else
            out[k] = __fadd_rn((float)mu, __fmul_rn((float)sigma, y));
    }
}

} // namespace

cudaError_t wl_launch_gather(const WlPassArgs &a, int fp64, int sm_count, cudaStream_t stream)
{
    int64_t want = (a.N + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (a.n == 2) {
        if (fp64)
            gather_kernel<2, double><<<grid, 256, 0, stream>>>(a);
        else
            gather_kernel<2, float><<<grid, 256, 0, stream>>>(a);
    } else if (a.n == 4) {
        if (fp64)
            gather_kernel<4, double><<<grid, 256, 0, stream>>>(a);
        else
            gather_kernel<4, float><<<grid, 256, 0, stream>>>(a);
    } else {
        if (fp64)
            gather_kernel<8, double><<<grid, 256, 0, stream>>>(a);
        else
            gather_kernel<8, float><<<grid, 256, 0, stream>>>(a);
    }
    return cudaGetLastError();
}

// Phase 2 of the two-phase pass for binary32 pools: the transform streamed
// over the j-ordered copy, four consecutive j per thread (16-byte loads and
// stores: the copy's and the pool's rows start on 256-byte boundaries), the
// returned values as 16-byte stores where a row's output offset is a multiple
// of 4, and the exact sum of squares of the four tuples added into 128 bits
// once.  The same arithmetic, in the same order, as gather_kernel<NSUB,
// float, true>.
template <int NSUB>
__global__ void __launch_bounds__(256) stream_kernel(WlPassArgs a)
{
    __shared__ uint64_t red[3 * 8];
    WlDevState *st = a.st;
    const float *__restrict__ src = (const float *)a.src;
    float *__restrict__ dst = (float *)a.dst;
    const int64_t N = a.N, Np = a.Np, w0 = a.w0, w1 = a.w1;
    const float c = st->next.c32, rC = st->next.rc32, rS = st->next.rs32;
    const uint32_t signs = st->next.signs;
    float *out = (float *)a.out;
    const float mu = (float)a.mu, sigma = (float)a.sigma;
    // row k's returned values: j in [r0[k], r1[k]) go to out[ofs[k] + j],
    // 16 bytes at a time when vec[k] (kept in shared memory: registers go to
    // the values)
    __shared__ int64_t r0[NSUB], r1[NSUB], ofs[NSUB];
    __shared__ bool vec[NSUB];
    if (threadIdx.x < NSUB) {
        const int k = threadIdx.x;
        r0[k] = max((int64_t)0, min(N, w0 - k * N));
        r1[k] = max(r0[k], min(N, w1 - k * N));
        ofs[k] = k * N - w0;
        vec[k] = ((ofs[k] & 3) == 0) && out != nullptr && (((uintptr_t)out & 15) == 0);
    }
    __syncthreads();
    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    const int64_t N4 = N & ~(int64_t)3;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    auto xform = [&](const float *g, float *y) {
        if constexpr (NSUB == 2)
            wl_xform2(g, rC, rS, y);
        else if constexpr (NSUB == 4)
            wl_xform4(g, c, y);
        else
            wl_xform8(g, c, y);
    };
    for (int64_t j = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < N4; j += 4 * G) {
        float4 g4[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++)
            g4[i] = *(const float4 *)(src + i * Np + j);
        float y[4][NSUB];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            float g[NSUB];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                const float v = u == 0 ? g4[i].x : u == 1 ? g4[i].y : u == 2 ? g4[i].z : g4[i].w;
                g[i] = wl_sgn(v, signs, i);
            }
            xform(g, y[u]);
        }
        uint64_t t = 0;   // 4 NSUB terms, each below 2^48
#pragma unroll
        for (int k = 0; k < NSUB; k++) {
            *(float4 *)(dst + k * Np + j) = make_float4(y[0][k], y[1][k], y[2][k], y[3][k]);
#pragma unroll
            for (int u = 0; u < 4; u++)
                t += wl_term32(y[u][k], bad);
            if (j + 4 <= r0[k] || j >= r1[k])
                continue;
            if (vec[k] && j >= r0[k] && j + 4 <= r1[k]) {
                *(float4 *)(out + ofs[k] + j) =
                    make_float4(__fadd_rn(mu, __fmul_rn(sigma, y[0][k])), __fadd_rn(mu, __fmul_rn(sigma, y[1][k])),
                                __fadd_rn(mu, __fmul_rn(sigma, y[2][k])), __fadd_rn(mu, __fmul_rn(sigma, y[3][k])));
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (j + u >= r0[k] && j + u < r1[k])
                        out[ofs[k] + j + u] = __fadd_rn(mu, __fmul_rn(sigma, y[u][k]));
            }
        }
        wl_add128(lo, hi, t, 0);
    }
    // the last N mod 4 values, one thread each
    const int64_t jt = N4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (jt < N) {
        float g[NSUB], y[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++)
            g[i] = wl_sgn(src[i * Np + jt], signs, i);
        xform(g, y);
#pragma unroll
        for (int k = 0; k < NSUB; k++) {
            dst[k * Np + jt] = y[k];
            wl_add128(lo, hi, wl_term32(y[k], bad), 0);
            if (jt >= r0[k] && jt < r1[k])
                out[ofs[k] + jt] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
        }
    }
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        double x = (double)__ldcg(&dst[wl_phys(a.nu - 1, N, Np)]);
        wl_finalise(st, a.n, N, a.nu, x, false, WL_FIN_PASS);
    }
}

// Two-phase pass: every sub-vector un-strided into `scratch` (same layout as
// a pool), then the transform streamed over j.
template <int NSUB, typename T>
static cudaError_t launch_twophase(const WlPassArgs &a, void *scratch, int sm_count, cudaStream_t stream)
{
    static bool configured = false;
    const size_t smem = sizeof(T) * (us_bmax<T>() + 32 / sizeof(T));   // + the lead and the cover's tail
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(unstride_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        configured = true;
    }
    const int per_sm = 3;
    unstride_kernel<T><<<sm_count * per_sm, US_THREADS, smem, stream>>>((const T *)a.src, (T *)scratch, a.st,
                                                                        NSUB, a.N, a.Np);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    WlPassArgs b = a;
    b.src = scratch;
    if constexpr (sizeof(T) == 4) {
        // four j per thread
        const int64_t want = (a.N / 4 + 255) / 256;
        const int64_t cap = (int64_t)sm_count * 8;
        const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
        stream_kernel<NSUB><<<grid, 256, 0, stream>>>(b);
    } else {
        int64_t want = (a.N + 255) / 256;
        int64_t cap = (int64_t)sm_count * 8;
        int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
        gather_kernel<NSUB, T, true><<<grid, 256, 0, stream>>>(b);
    }
    return cudaGetLastError();
}

cudaError_t wl_launch_twophase(const WlPassArgs &a, void *scratch, int fp64, int sm_count, cudaStream_t stream)
{
    if (a.n == 2)
        return fp64 ? launch_twophase<2, double>(a, scratch, sm_count, stream)
                    : launch_twophase<2, float>(a, scratch, sm_count, stream);
    if (a.n == 4)
        return fp64 ? launch_twophase<4, double>(a, scratch, sm_count, stream)
                    : launch_twophase<4, float>(a, scratch, sm_count, stream);
    return fp64 ? launch_twophase<8, double>(a, scratch, sm_count, stream)
                : launch_twophase<8, float>(a, scratch, sm_count, stream);
}

cudaError_t wl_launch_drain(const void *pool, int fp64, int64_t N, int64_t Np, int64_t pos,
                            int64_t count, void *out, double mu, double sigma, int sm_count,
                            cudaStream_t stream)
{
    if (count <= 0)
        return cudaSuccess;
    int64_t want = (count + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? want : cap);
    if (fp64)
        drain_kernel<double><<<grid, 256, 0, stream>>>((const double *)pool, N, Np, pos, count,
                                                       (double *)out, mu, sigma);
    else
        drain_kernel<float><<<grid, 256, 0, stream>>>((const float *)pool, N, Np, pos, count,
                                                      (float *)out, mu, sigma);
    return cudaGetLastError();
}
