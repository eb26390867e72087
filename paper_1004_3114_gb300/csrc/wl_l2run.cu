// Many passes of one generator in ONE launch, for pools that stay in L2
// between passes (Section 2: a pass is a few vector operations over the pool;
// for pools of a few MB the fixed cost of a launch and of the end-of-pass
// round trip is most of a pass).
//
// A cooperative grid of G CTAs (all resident) runs P passes.  In pass p each
// thread takes tuples j = t, t + T, ... (t its index in the grid, T the
// grid's thread count) and gathers g_i[j] = x_i[(alpha_i j + gamma_i) mod N]
// straight from L2 (loads that bypass L1: the previous pass's pool was
// written by other SMs), transforms, stores the new pool and the returned
// prefix with unit stride, and sums its exact squares.  The CTA adds its sum
// to accumulator set p mod 3 and arrives at a grid barrier.  After the
// barrier every CTA runs the end of pass itself -- the chi-squared rescale
// (Eq. 3), the strides drawn a pass ahead, the drift check (Section 8) -- on
// its own shared-memory copy of the generator's state, three threads at
// once, from the summed Q and the withheld value read together.  The
// arithmetic is the same in every CTA, so the copies stay identical and
// nothing is broadcast; CTA 0 writes its copy back at the end.
//
// Why a plain gather here: staging spans in shared memory (the pass kernels
// for pools in HBM) saves DRAM bytes, but a pool in L2 has none to save,
// while the staging pipeline's set-up and tile latency would be most of a
// pass.  Index arithmetic is 32-bit (pools of at most 2^23 values, strides
// small enough that alpha N < 2^32), since a 64-bit remainder costs hundreds
// of cycles on this part.
//
// Accumulator set (p + 1) mod 3 is cleared by CTA 0 during pass p: its last
// readers (after barrier p - 2) have all arrived at barrier p - 1 by then.
// The barrier counter only grows: pass p's barrier completes at (p + 1) G
// arrivals.  Every wait is bounded (about a second); a CTA that gives up
// raises the grid's abort flag, the others stop at their next barrier, and
// the generator's status gets WALLACE_ETIMEOUT.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "wl_common.cuh"
#include "wl_gridsync.cuh"
#include "wl_launch.h"

#define L2_THREADS 512

namespace {

struct L2Args {
    float *buf[2];
    int cur;
    WlDevState *st;
    WlGridSync *sy;
    int64_t N, Np, R;
    int64_t passes;
    float *out;           // pass p writes its first take values to out + p R (may be null)
    int64_t last_take;    // values the last pass returns (the others return R)
    float mu, sigma;
};

// SG: the generator draws a sign pattern each pass (matrix A D_k).
template <int NSUB, bool SG>
__global__ void __launch_bounds__(L2_THREADS, 2) l2run_kernel(L2Args a)
{
    __shared__ uint64_t red[3 * (L2_THREADS / 32)];
    __shared__ WlDevState sst;   // this CTA's copy of the generator's state
    wl_state_load(&sst, a.st);
    WlDevState *st = &sst;
    WlGridSync *sy = a.sy;
    const int tid = threadIdx.x, G = gridDim.x, b = blockIdx.x;
    const uint32_t N = (uint32_t)a.N;
    const int64_t Np = a.Np, nu = NSUB * a.N;
    const double rnu = wl_rnu(nu);
    const uint32_t gt = (uint32_t)b * blockDim.x + tid, GT = (uint32_t)G * blockDim.x;
    const float mu = a.mu, sigma = a.sigma;
    int cur = a.cur;
    // passes completed before this launch: pass p of the launch is pass k0 + p,
    // and its strides sit in ahead[(k0 + p) & 1] from the end of the pass before
    const int64_t k0 = st->passes;
    float pg[NSUB];      // the thread's first tuple of the pass, loaded during the last end of pass
    bool pre = false;
    for (int64_t p = 0; p < a.passes; p++) {
        // this pass's parameters become the most recent pass's (warp 0, word
        // by word; nothing reads `last` during the pass)
        if (tid < 32) {
            const uint32_t *from = (const uint32_t *)&st->next;
            uint32_t *to = (uint32_t *)&st->last;
            for (int w = tid; w < (int)(sizeof(WlParams) / 4); w += 32)
                to[w] = from[w];
        }
        // 32-bit index arithmetic: (alpha + 1) N < 2^32 (checked by the host)
        uint32_t idx[NSUB], stp[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            const uint32_t al = (uint32_t)st->next.alpha[i], ga = (uint32_t)st->next.gamma[i];
            idx[i] = (al * (gt < N ? gt : 0u) + ga) % N;
            stp[i] = (al * (GT % N)) % N;
        }
        const float c = st->next.c32;
        const uint32_t signs = SG ? st->next.signs : 0u;
        const float *src = a.buf[cur];
        float *dst = a.buf[1 - cur];
        float *o = a.out ? a.out + p * a.R : nullptr;
        const uint32_t w1 = o ? (uint32_t)(p + 1 < a.passes ? a.R : a.last_take) : 0u;
        uint64_t lo = 0, hi = 0;
        uint32_t bad = 0;
        for (uint32_t j = gt; j < N; j += GT) {
            float g[NSUB], y[NSUB];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                g[i] = pre ? pg[i] : __ldcg(src + i * Np + idx[i]);
                if (SG)
                    g[i] = wl_sgn(g[i], signs, i);
                idx[i] += stp[i];
                idx[i] -= idx[i] >= N ? N : 0u;
            }
            pre = false;
            if constexpr (NSUB == 4)
                wl_xform4(g, c, y);
            else
                wl_xform8(g, c, y);
#pragma unroll
            for (int k = 0; k < NSUB; k++) {
                dst[k * Np + j] = y[k];
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                const uint32_t q = (uint32_t)k * N + j;
                if (q < w1)
                    o[q] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
            }
        }
        WlGridAcc *acc = &sy->acc[p % 3];
        wl_grid_reduce_to(lo, hi, bad, acc, red);
        if (b == 0 && tid == 0) {
            WlGridAcc *nx = &sy->acc[(p + 1) % 3];
            nx->a0 = 0;
            nx->a1 = 0;
            nx->a2 = 0;
            nx->bad = 0;
        }
        wl_grid_arrive(sy);
        if (!wl_grid_wait(sy, (unsigned int)((p + 1) * G)))
            break;
        // the next pass's first tuple of this thread, loaded now so that its
        // latency passes during the end of pass: the next pass's strides were
        // drawn a pass ahead (ahead[(k + 1) & 1], which the stride role below
        // copies but does not write) and its pool is this pass's, complete at
        // the barrier; only the scale waits for the end of pass
        if (p + 1 < a.passes && gt < N && tid >= 96) {   // not the warps of the end-of-pass roles
            const WlStrides &nx = st->ahead[(k0 + p + 1) & 1];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                const uint32_t al = (uint32_t)nx.alpha[i], ga = (uint32_t)nx.gamma[i];
                pg[i] = __ldcg(dst + i * Np + (al * gt + ga) % N);
            }
            pre = true;
        }
        // end of pass from the summed Q: scale (thread 0), strides (32),
        // drift (64), each reading Q and the withheld value together
        if (tid == 0 || tid == 64) {
            const unsigned long long a0 = __ldcg(&acc->a0), a1 = __ldcg(&acc->a1), a2 = __ldcg(&acc->a2);
            const uint32_t qbad = __ldcg(&acc->bad);
            const double x = (double)__ldcg(&dst[wl_last_phys(NSUB, a.N, Np)]);
            const unsigned long long t = a0 + (a1 << 32);
            const uint64_t qhi = a2 + (a1 >> 32) + (t < a0 ? 1ull : 0ull);
            wl_end_pass_role(st, NSUB, a.N, nu, rnu, t, qhi, qbad, x, tid == 0 ? 0 : 2, SG ? 1 : 0, false);
        } else if (tid == 32) {
            wl_end_pass_role(st, NSUB, a.N, nu, rnu, 0, 0, 0, 0.0, 1, SG ? 1 : 0, false);
        }
        __syncthreads();
        cur = 1 - cur;
    }
    if (b == 0) {
        __syncthreads();
        if (tid == 0 && *(volatile int *)&sy->abort)
            st->status |= WL_ETIMEOUT;
        wl_state_store(a.st, st);
    }
}

int g_l2_max_grid = 0;   // co-resident CTAs of the kernel on this device (0: not looked up)

} // namespace

bool wl_l2run_supported(int n, int64_t N, int fp64, int64_t max_stride)
{
    // 32-bit indices: (alpha + 1) N < 2^32 and n N <= 2^23
    return (n == 4 || n == 8) && !fp64 && N >= 4 && (int64_t)n * N <= ((int64_t)1 << 23) &&
           (max_stride + 1) * N < ((int64_t)1 << 32);
}

size_t wl_l2run_sync_bytes() { return sizeof(WlGridSync); }

int wl_l2run_grid(int64_t nu, int sm_count)
{
    // measured: one CTA per SM is fastest up to 2^22 values (a pass is mostly
    // barrier and end-of-pass latency there); two per SM above
    return nu <= ((int64_t)1 << 22) ? sm_count : 2 * sm_count;
}

cudaError_t wl_launch_l2run(void *buf0, void *buf1, int cur, int n, int64_t N, int64_t Np, WlDevState *st,
                            void *sync, int64_t passes, int64_t R, int64_t last_take, void *out, double mu,
                            double sigma, int grid, int signs, cudaStream_t stream)
{
    auto kern = n == 8 ? (signs ? l2run_kernel<8, true> : l2run_kernel<8, false>)
                       : (signs ? l2run_kernel<4, true> : l2run_kernel<4, false>);
    if (!g_l2_max_grid) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // every instantiation has the same shape; the <8, true> one has the most registers
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, l2run_kernel<8, true>, L2_THREADS, 0);
        if (e != cudaSuccess)
            return e;
        g_l2_max_grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    if (grid > g_l2_max_grid)
        grid = g_l2_max_grid;
    cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(WlGridSync), stream);
    if (e != cudaSuccess)
        return e;
    L2Args a;
    a.buf[0] = (float *)buf0;
    a.buf[1] = (float *)buf1;
    a.cur = cur;
    a.st = st;
    a.sy = (WlGridSync *)sync;
    a.N = N;
    a.Np = Np;
    a.R = R;
    a.passes = passes;
    a.out = (float *)out;
    a.last_take = last_take;
    a.mu = (float)mu;
    a.sigma = (float)sigma;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(L2_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: they wait on one another
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}
