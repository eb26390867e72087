// The Box-Muller method as a stand-alone GPU generator: the comparison point
// of Brent's RANN4 paper (its abstract and Section 1 set Wallace's method
// against the Box-Muller and Polar methods).  Value k of the stream of
// (seed, stream id) is the k-th output of Box-Muller pairs formed from
// consecutive 32-bit uniforms of the generator's uniform source -- the same
// pairs that fill a Wallace generator's initial pool -- mapped to
// mu + sigma * y (binary32 multiply, then add).
//
// Two arithmetic modes:
//   exact -- the binary64 series of wl_bm.cuh, bit-identical to the initial
//            pool;
//   fast  -- binary32 with CUDA's logf / log1pf / sincospif: the logarithm
//            of u1 = (U1 + 1) 2^-32 is taken as logf(u1) for U1 < 2^31 and as
//            log1pf(-(2^32 - 1 - U1) 2^-32) above, so that u1 near 1 keeps its
//            relative accuracy; the angle is reduced to a quadrant from the
//            top two bits of U2 and the rest goes to sincospif.
// The Polar method is not built: its rejection step (acceptance pi/4) makes
// the lanes of a warp diverge, which Box-Muller does not.
//
// Each thread takes pairs p, p + G, p + 2G, ... (G threads in the grid), so a
// warp writes consecutive pairs; its uniform state hops 2G steps at a time by
// the composed affine map of the LCG.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wallace.h"
#include "wl_bm.cuh"
#include "wl_common.cuh"

namespace {

__device__ __forceinline__ void bm_fast(uint32_t u1, uint32_t u2, float &a, float &b)
{
    float l;
    if (u1 < 0x80000000u)
        l = logf(__fmul_rn((float)(u1 + 1u), 2.3283064365386963e-10f));
    else
        l = log1pf(-__fmul_rn((float)(0xFFFFFFFFu - u1), 2.3283064365386963e-10f));
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, l));
    const uint32_t quad = u2 >> 30;
    // angle within the quadrant as a fraction of a half turn: (u2 mod 2^30) 2^-31
    const float g = __fmul_rn((float)(u2 & 0x3FFFFFFFu), 4.656612873077393e-10f);
    float sp, cp;
    sincospif(g, &sp, &cp);
    float cs, sn;
    switch (quad) {
    case 0: cs = cp; sn = sp; break;
    case 1: cs = -sp; sn = cp; break;
    case 2: cs = -cp; sn = -sp; break;
    default: cs = sp; sn = -cp; break;
    }
    a = __fmul_rn(r, cs);
    b = __fmul_rn(r, sn);
}

template <bool EXACT>
__global__ void __launch_bounds__(256) bm_kernel(uint32_t seed, uint32_t stream_id, int64_t v0,
                                                 int64_t count, float *__restrict__ out, float mu,
                                                 float sigma)
{
    // pairs [p0, p1) cover values [v0, v0 + count)
    const int64_t p0 = v0 >> 1, p1 = (v0 + count + 1) >> 1;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1)
        return;
    const uint64_t one = wl_lcg_jump(0, 2 * (uint64_t)G);
    const uint64_t AG = wl_lcg_jump(1, 2 * (uint64_t)G) - one;
    uint64_t s = wl_lcg_jump(wl_seed_mix(seed, stream_id), 2 * (uint64_t)p);
    const int64_t v1 = v0 + count;
    for (; p < p1; p += G) {
        uint64_t t = s;
        const uint32_t u1 = wl_lcg_step(t);
        const uint32_t u2 = wl_lcg_step(t);
        float a, b;
        if (EXACT)
            wl_bm::box_muller(u1, u2, a, b);
        else
            bm_fast(u1, u2, a, b);
        a = __fadd_rn(mu, __fmul_rn(sigma, a));
        b = __fadd_rn(mu, __fmul_rn(sigma, b));
        const int64_t q = 2 * p - v0;   // output index of value 2p
        if (2 * p >= v0 && 2 * p + 1 < v1 && ((uintptr_t)(out + q) & 7) == 0) {
            *reinterpret_cast<float2 *>(out + q) = make_float2(a, b);
        } else {
            if (2 * p >= v0 && 2 * p < v1)
                out[q] = a;
            if (2 * p + 1 >= v0 && 2 * p + 1 < v1)
                out[q + 1] = b;
        }
        s = AG * s + one;
    }
}

} // namespace

extern "C" int wallace_boxmuller_fill(uint32_t seed, uint32_t stream_id, int64_t offset,
                                      float *out, int64_t count, float mu, float sigma, int exact,
                                      void *cuda_stream)
{
    if (offset < 0 || count < 0 || (count > 0 && !out) || offset > INT64_MAX / 2 - count)
        return WALLACE_EINVAL;
    if (count == 0)
        return WALLACE_OK;
    int dev = 0, sm_count = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return WALLACE_ECUDA;
    const int64_t pairs = ((offset + count + 1) >> 1) - (offset >> 1);
    const int64_t want = (pairs + 255) / 256;
    const int64_t cap = (int64_t)sm_count * 8;
    const int grid = (int)(want < cap ? want : cap);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (exact)
        bm_kernel<true><<<grid, 256, 0, st>>>(seed, stream_id, offset, count, out, mu, sigma);
    else
        bm_kernel<false><<<grid, 256, 0, st>>>(seed, stream_id, offset, count, out, mu, sigma);
    return cudaGetLastError() == cudaSuccess ? WALLACE_OK : WALLACE_ECUDA;
}
