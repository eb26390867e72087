// One pass of Wallace's generator (Eq. 1 of Brent's RANN4 paper, n = 4,
// binary32 pool) as a lane-tiled gather staged through shared memory.
//
// The paper's vector loop (Section 7) splits j into alpha+beta-1 wrap-free
// segments so the inner loop needs no "mod N".  The GPU analogue used here:
// with L = lcm(alpha_0..alpha_3), cut j = 0..N-1 into L lanes, lane l
// starting at J_l = ceil(l N / L).  For sub-vector i (m_i = L / alpha_i),
// write l = w m_i + p.  Inside lane l the wrap count of alpha_i j is the
// constant w, and alpha_i J_l - w N lies in [p N / m_i, p N / m_i + alpha_i).
// The alpha_i lanes sharing p have distinct residues, so at lane time t they
// read exactly the alpha_i consecutive addresses
//     C_ip + alpha_i t + [0, alpha_i),   C_ip = ceil(p N / m_i)   (+ gamma_i mod N).
// A tile of T lane times therefore reads, per sub-vector, m_i contiguous
// spans of alpha_i T values and uses every value: the gather becomes
// contiguous 16-byte copies into shared memory (odd strides alpha_i make the
// shared-memory reads bank-conflict free, the GPU counterpart of the paper's
// odd strides for interleaved banks) plus unit-stride stores of T values per
// lane.  Strides come from rows whose values divide 315, so L <= 315.
//
// Persistent kernel: each CTA builds the lane tables once, then loops over
// tiles t0 = T * tile.  If a pass's strides have L > 315 (fallback strides
// for N with small odd factors) the same launch runs a plain strided gather.
#include "wl_common.cuh"
#include "wl_launch.h"

#define TL_LMAX 315
#define TL_THREADS 256
#define TL_MAXSPANS 420     /* sum_i L / alpha_i <= 4 * 315 / 3 */
#define TL_MAXWRAP 64
#define TL_ETARGET 2560     /* lane-times per tile: L * T <= this */
#define TL_MIN_N 16384

namespace {

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// floor(f / d) as umulhi(f, ceil(2^32 / d)): exact when f * d < 2^32 and d >= 2
// (the error f (ceil(2^32/d) - 2^32/d) / 2^32 < f / 2^32 < 1/d); d = 1 is passed through.
__device__ __forceinline__ uint32_t magic_div(uint32_t d)
{
    return d > 1 ? (uint32_t)((0x100000000ull + d - 1) / d) : 0u;
}
__device__ __forceinline__ uint32_t fast_div(uint32_t f, uint32_t d, uint32_t m)
{
    return d > 1 ? __umulhi(f, m) : f;
}

__host__ __device__ constexpr int tl_data_words(int etarget)
{
    return 4 * etarget + 4 * TL_MAXSPANS;
}
__host__ __device__ constexpr int tl_int_words()
{
    return (TL_LMAX + 1) + 8 * TL_LMAX + 4 * TL_MAXSPANS;
}

__global__ void __launch_bounds__(TL_THREADS, 3) tiled_kernel(WlPassArgs a)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ uint64_t red[3 * (TL_THREADS / 32)];
    __shared__ int s_wrap[TL_MAXWRAP];
    __shared__ int s_nwrap;

    WlDevState *st = a.st;
    const float *__restrict__ src = (const float *)a.src;
    float *__restrict__ dst = (float *)a.dst;
    const int64_t N = a.N, Np = a.Np;
    const int tid = threadIdx.x;
    int alpha[4];
    int64_t gam[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        alpha[i] = st->next.alpha[i];
        gam[i] = st->next.gamma[i];
    }
    const float c = st->next.c32;
    float *out = (float *)a.out;
    const float mu = (float)a.mu, sigma = (float)a.sigma;
    const int64_t w0 = a.w0, w1 = a.w1;

    int L = alpha[0];
#pragma unroll
    for (int i = 1; i < 4; i++)
        L = L / (int)wl_gcd(L, alpha[i]) * alpha[i];

    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;

    if (L > TL_LMAX || N < (int64_t)TL_MIN_N) {
        // plain strided gather for this pass
        const int64_t G = (int64_t)gridDim.x * blockDim.x;
        int64_t j = (int64_t)blockIdx.x * blockDim.x + tid;
        int64_t idx[4], stp[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            idx[i] = (int64_t)(((uint64_t)alpha[i] * (uint64_t)(j < N ? j : 0) + (uint64_t)gam[i]) % (uint64_t)N);
            stp[i] = (int64_t)(((uint64_t)alpha[i] * (uint64_t)G) % (uint64_t)N);
        }
        for (; j < N; j += G) {
            float g[4], y[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                g[i] = src[i * Np + idx[i]];
                idx[i] += stp[i];
                if (idx[i] >= N)
                    idx[i] -= N;
            }
            wl_xform4(g, c, y);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                dst[k * Np + j] = y[k];
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                int64_t q = k * N + j;
                if (q >= w0 && q < w1)
                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
            }
        }
    } else {
        int m[4], sb[5], slot0[4], SL[4];
        const int T = (TL_ETARGET / L) & ~3;
        sb[0] = 0;
        slot0[0] = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            m[i] = L / alpha[i];
            SL[i] = alpha[i] * T + 4;  // copies cover at most alpha_i T + 4 values
            sb[i + 1] = sb[i] + m[i];
            if (i < 3)
                slot0[i + 1] = slot0[i] + m[i] * SL[i];
        }
        const int nspans = sb[4];
        int *J = (int *)(smem + tl_data_words(TL_ETARGET));
        int *lanebase = J + (TL_LMAX + 1);
        int *laneoff = lanebase + 4 * TL_LMAX;
        int *spanC = laneoff + 4 * TL_LMAX;
        int *spanAs = spanC + TL_MAXSPANS;
        int *spanLead = spanAs + TL_MAXSPANS;
        int *spanAddr = spanLead + TL_MAXSPANS;
        const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);

        // lane starts J_l = ceil(l N / L) and span bases C_ip = ceil(p N / m_i)
        for (int l = tid; l <= L; l += TL_THREADS)
            J[l] = (int)(((int64_t)l * N + L - 1) / L);
        for (int s = tid; s < nspans; s += TL_THREADS) {
            int i = (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
            int p = s - sb[i];
            spanC[s] = (int)(((int64_t)p * N + m[i] - 1) / m[i]);
        }
        __syncthreads();
        // lane l, sub-vector i: offset r in [0, alpha_i) inside its group's span
        for (int e = tid; e < 4 * L; e += TL_THREADS) {
            int i = e / L, l = e - i * L;
            int w = l / m[i], p = l - w * m[i];
            int64_t r = (int64_t)alpha[i] * J[l] - (int64_t)w * N - spanC[sb[i] + p];
            lanebase[i * TL_LMAX + l] = slot0[i] + p * SL[i] + (int)r;
        }
        const int maxlen = (int)((N + L - 1) / L);
        const int ntiles = (maxlen + T - 1) / T;
        __syncthreads();

        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int t0 = tile * T;
            const int Tt = min(T, maxlen - t0);
            if (tid == 0)
                s_nwrap = 0;
            __syncthreads();
            // where each span starts this tile; wrapping spans go to a list
            for (int s = tid; s < nspans; s += TL_THREADS) {
                int i = (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
                int64_t addr = (int64_t)spanC[s] + (int64_t)alpha[i] * t0 + gam[i];
                while (addr >= N)
                    addr -= N;
                int len = alpha[i] * Tt;
                spanAddr[s] = (int)addr;
                if (addr + len <= N) {
                    int as = (int)addr & ~3;
                    spanAs[s] = as;
                    spanLead[s] = (int)addr - as;
                } else {
                    spanAs[s] = -1;
                    spanLead[s] = 0;
                    int k = atomicAdd(&s_nwrap, 1);
                    if (k < TL_MAXWRAP)
                        s_wrap[k] = s;
                }
            }
            __syncthreads();
            // 16-byte copies of the aligned spans
#pragma unroll 1
            for (int i = 0; i < 4; i++) {
                const int K = (alpha[i] * Tt + 3) / 4 + 1;
                const uint32_t mk = magic_div((uint32_t)K);
                const int total = m[i] * K;
                const float *srci = src + (int64_t)i * Np;
                for (int f = tid; f < total; f += TL_THREADS) {
                    int p = (int)fast_div((uint32_t)f, (uint32_t)K, mk);
                    int ch = f - p * K;
                    int as = spanAs[sb[i] + p];
                    if (as >= 0)
                        cp_async16(smem_base + 4u * (uint32_t)(slot0[i] + p * SL[i] + 4 * ch),
                                   srci + as + 4 * ch);
                }
            }
            // spans that run past the end of a sub-vector wrap to its start
            const int nw = min(s_nwrap, TL_MAXWRAP);
            for (int k = 0; k < nw; k++) {
                int s = s_wrap[k];
                int i = (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
                int p = s - sb[i];
                int len = alpha[i] * Tt;
                int64_t addr = spanAddr[s];
                float *slot = smem + slot0[i] + p * SL[i];
                for (int u = tid; u < len; u += TL_THREADS) {
                    int64_t ad = addr + u;
                    if (ad >= N)
                        ad -= N;
                    slot[u] = src[(int64_t)i * Np + ad];
                }
            }
            // per-lane offsets for this tile
            for (int e = tid; e < 4 * L; e += TL_THREADS) {
                int i = e / L, l = e - i * L;
                int p = l % m[i];
                laneoff[i * TL_LMAX + l] = lanebase[i * TL_LMAX + l] + spanLead[sb[i] + p];
            }
            cp_async_wait_all();
            __syncthreads();
            // transform: pair f = (lane l, time t)
            const uint32_t mT = magic_div((uint32_t)Tt);
            const int npairs = L * Tt;
            for (int f = tid; f < npairs; f += TL_THREADS) {
                int l = (int)fast_div((uint32_t)f, (uint32_t)Tt, mT);
                int t = f - l * Tt;
                int jl = J[l];
                int tt = t0 + t;
                if (tt >= J[l + 1] - jl)
                    continue;
                float g[4], y[4];
#pragma unroll
                for (int i = 0; i < 4; i++)
                    g[i] = smem[laneoff[i * TL_LMAX + l] + alpha[i] * t];
                wl_xform4(g, c, y);
                const int64_t j = (int64_t)jl + tt;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    dst[k * Np + j] = y[k];
                    wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                    int64_t q = k * N + j;
                    if (q >= w0 && q < w1)
                        out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
                }
            }
            __syncthreads();
        }
    }

    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && tid == 0) {
        double x = (double)__ldcg(&dst[wl_phys(a.nu - 1, N, Np)]);
        wl_finalise(st, 4, N, a.nu, x, false, true);
    }
}

int g_tiled_ctas_per_sm = 0;

} // namespace

bool wl_tiled_supported(int n, int64_t N, int fp64)
{
    return n == 4 && !fp64 && N >= TL_MIN_N && N <= ((int64_t)1 << 28);
}

cudaError_t wl_launch_tiled(const WlPassArgs &a, int sm_count, cudaStream_t stream)
{
    const size_t smem = sizeof(float) * (size_t)(tl_data_words(TL_ETARGET) + tl_int_words());
    if (g_tiled_ctas_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tiled_kernel, TL_THREADS, smem);
        if (e != cudaSuccess)
            return e;
        g_tiled_ctas_per_sm = per > 0 ? per : 1;
    }
    int grid = sm_count * g_tiled_ctas_per_sm;
    tiled_kernel<<<grid, TL_THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}
