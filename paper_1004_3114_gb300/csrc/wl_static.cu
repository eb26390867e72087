// wallace_pass_static: one pass with no device allocation by the library
// or the caller beyond the caller's own pool and output.
//
// Some callers cannot allocate device memory: a host application that gives
// a plug-in a fixed set of buffers and a fixed memory budget and does not let
// it call cudaMalloc (so the library cannot create a handle with its own
// double buffer and state block), or code on a path where cudaMalloc's
// implicit device-wide synchronisation is not acceptable.  For them this
// file keeps the pass's scratch -- the second pool buffer and the reduction
// and finaliser block -- in one file-scope device array of fixed size.
//
// The array exists once per device that loads the library and stays
// allocated until the process exits.  Every call uses the same array, so
// calls must not overlap on the GPU (two calls in flight at once, on any
// streams, race on it).  The first call on each device looks up the array's
// device address (cudaGetSymbolAddress) with that device current; make that
// first call before any stream capture begins.
//
// The pass computes the next scale from the fixed Eq. 3 sample only: there is
// no Wilson-Hilferty option, and no drift check (the caller, who holds the
// pool between calls, holds the previous chi-squared target too).  Like a
// handle, it never returns the new pool's last value, which sets that scale.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wallace.h"
#include "wl_common.cuh"

#define WL_STATIC_STATE_BYTES 1024
#define WL_STATIC_BYTES (WL_STATIC_STATE_BYTES + 4ull * WALLACE_STATIC_MAX_VALUES)

static_assert(sizeof(WlDevState) <= WL_STATIC_STATE_BYTES, "state block does not fit");

// Scratch of wallace_pass_static: [0, 1024) reduction/finaliser block,
// [1024, 1024 + 4 * WALLACE_STATIC_MAX_VALUES) the new pool.
static __device__ __align__(256) unsigned char g_wl_static_scratch[WL_STATIC_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Same pass as the library's plain strided-gather kernel, with explicit
// parameters and the new pool and Q accumulators in the static scratch.
template <int NSUB>
__global__ void __launch_bounds__(256) static_gather_kernel(const float *__restrict__ src,
                                                            unsigned char *scratch, int64_t N,
                                                            WlParams prm, float *__restrict__ out,
                                                            int64_t out_count, float mu,
                                                            float sigma)
{
    __shared__ uint64_t red[3 * 8];
    WlDevState *st = (WlDevState *)scratch;
    float *dst = (float *)(scratch + WL_STATIC_STATE_BYTES);
    const int64_t nu = NSUB * N;
    const float c = prm.c32;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t idx[NSUB], step[NSUB];
#pragma unroll
    for (int i = 0; i < NSUB; i++) {
        idx[i] = (int64_t)(((uint64_t)prm.alpha[i] * (uint64_t)(j < N ? j : 0) +
                            (uint64_t)prm.gamma[i]) % (uint64_t)N);
        step[i] = (int64_t)(((uint64_t)prm.alpha[i] * (uint64_t)G) % (uint64_t)N);
    }
    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    for (; j < N; j += G) {
        float g[NSUB], y[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            g[i] = src[i * N + idx[i]];
            idx[i] += step[i];
            if (idx[i] >= N)
                idx[i] -= N;
        }
        if constexpr (NSUB == 4)
            wl_xform4(g, c, y);
        else
            wl_xform8(g, c, y);
#pragma unroll
        for (int k = 0; k < NSUB; k++) {
            const int64_t q = k * N + j;
            dst[q] = y[k];
            wl_add128(lo, hi, wl_term32(y[k], bad), 0);
            if (q < out_count)
                out[q] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
        }
    }
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        double x = (double)__ldcg(&dst[nu - 1]);
        wl_finalise(st, NSUB, N, nu, x, false, WL_FIN_SCALE);
    }
}

// Device address of the scratch array for the current device (looked up once).
cudaError_t scratch_for_current_device(unsigned char **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_wl_static_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[dev] = p;
    }
    *ptr = (unsigned char *)g_scratch_addr[dev];
    return cudaSuccess;
}

} // namespace

extern "C" int wallace_pass_static(int n, int64_t N, float *pool, const int32_t *alpha,
                                   const int64_t *gamma, float c32, float *out,
                                   int64_t out_count, float mu, float sigma,
                                   wallace_pass_result_t *result, void *cuda_stream)
{
    if ((n != 4 && n != 8) || N < 4 || !pool || !alpha || !gamma || !result)
        return WALLACE_EINVAL;
    const int64_t nu = (int64_t)n * N;
    if (nu > (int64_t)WALLACE_STATIC_MAX_VALUES)
        return WALLACE_EINVAL;   // beyond the fixed scratch array
    // the last value is withheld (Section 4): it sets the next pass's scale
    if (out_count < 0 || out_count > nu - 1 || (out_count > 0 && !out))
        return WALLACE_EINVAL;
    WlParams prm = {};
    for (int i = 0; i < n; i++) {
        if (alpha[i] < 1 || gamma[i] < 0 || gamma[i] >= N)
            return WALLACE_EINVAL;
        prm.alpha[i] = alpha[i];
        prm.gamma[i] = gamma[i];
    }
    prm.c32 = c32;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    // the block left by the previous call: accumulators, ticket, status and
    // drift history must start at zero
    if (e == cudaSuccess)
        e = cudaMemsetAsync(scratch, 0, WL_STATIC_STATE_BYTES, stream);
    if (e != cudaSuccess)
        return WALLACE_ECUDA;
    int sm_count = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (N + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? want : cap);
    if (n == 4)
        static_gather_kernel<4><<<grid, 256, 0, stream>>>(pool, scratch, N, prm, out, out_count,
                                                         mu, sigma);
    else
        static_gather_kernel<8><<<grid, 256, 0, stream>>>(pool, scratch, N, prm, out, out_count,
                                                         mu, sigma);
    e = cudaGetLastError();
    // the new pool replaces the caller's pool
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pool, scratch + WL_STATIC_STATE_BYTES, sizeof(float) * (size_t)nu,
                            cudaMemcpyDeviceToDevice, stream);
    WlDevState s;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s, scratch, sizeof(s), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return WALLACE_ECUDA;
    result->q_lo = s.q_lo;
    result->q_hi = s.q_hi;
    result->q = s.q;
    result->S = s.S;
    result->c = s.c;
    result->c32 = s.next.c32;
    result->bad = s.bad;
    result->status = s.status;
    return s.status;
}
