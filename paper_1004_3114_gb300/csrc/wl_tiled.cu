// One pass of Wallace's generator (Eq. 1 of Brent's RANN4 paper, n = 4,
// binary32 pool) as a grid-wide lane-tiled gather staged through shared
// memory with per-thread 16-byte async copies (wl_tiled_body.cuh).
//
// The paper's vector loop (Section 7) splits j into alpha+beta-1 wrap-free
// segments so the inner loop needs no "mod N".  The GPU analogue: with
// L = lcm(alpha_0..alpha_3), cut j = 0..N-1 into L lanes, lane l starting at
// J_l = ceil(l N / L).  For sub-vector i (m_i = L / alpha_i), write
// l = w m_i + p.  Inside lane l the wrap count of alpha_i j is the constant w,
// and alpha_i J_l - w N lies in [p N / m_i, p N / m_i + alpha_i).  The alpha_i
// lanes sharing p have distinct residues, so at lane time t they read exactly
// the alpha_i consecutive addresses C_ip + alpha_i t + [0, alpha_i),
// C_ip = ceil(p N / m_i) (+ gamma_i mod N): a tile of T lane times reads m_i
// contiguous spans of alpha_i T values per sub-vector and uses every value.
// Odd strides alpha_i make the shared-memory reads bank-conflict free, the GPU
// counterpart of the paper's odd strides for interleaved memory banks.
//
// Persistent kernel: CTA b handles tiles b, b + grid, ...  If a pass's
// strides have L > 315 (N a multiple of 15: the candidates divide 7^2 11 or a
// larger p^2 q) the same launch runs a plain strided gather.
#include "wl_launch.h"
#include "wl_tiled_body.cuh"

#define TL_THREADS 256
#define TL_MIN_N 16384

namespace {

__global__ void __launch_bounds__(TL_THREADS, 3) tiled_kernel(WlPassArgs a)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ uint64_t red[3 * (TL_THREADS / 32)];

    WlDevState *st = a.st;
    WlTileJob job;
    job.src = (const float *)a.src;
    job.dst = (float *)a.dst;
    job.N = a.N;
    job.Np = a.Np;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        job.alpha[i] = st->next.alpha[i];
        job.gam[i] = st->next.gamma[i];
    }
    job.c = st->next.c32;
    job.signs = st->next.signs;
    job.out = (float *)a.out;
    job.w0 = a.w0;
    job.w1 = a.w1;
    job.mu = (float)a.mu;
    job.sigma = (float)a.sigma;

    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    const int L = wl_lcm4(job.alpha);
    if (wl_tiled_ok(L, job.N))
        wl_tiled4_tiles(job, L, blockIdx.x, gridDim.x, TL_EMAX, smem, lo, hi, bad);
    else
        wl_gather4_range(job, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                         (int64_t)gridDim.x * blockDim.x, lo, hi, bad);

    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        double x = (double)__ldcg(&job.dst[wl_phys(a.nu - 1, job.N, job.Np)]);
        wl_finalise(st, 4, job.N, a.nu, x, false, WL_FIN_PASS);
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
    const size_t smem = tl_smem_bytes();
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
