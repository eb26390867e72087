// Host runtime behind include/wallace.h: generator handles, the fill cursor,
// kernel selection, per-launch timing and the host-buffer fill pipeline.
// Every arithmetic step of the method runs in the kernels; this file only
// allocates, launches and copies.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "wallace.h"
#include "wl_common.cuh"
#include "wl_launch.h"

struct wallace {
    int n = 0, mode = WALLACE_FP32;
    int64_t N = 0, Np = 0, nu = 0, R = 0;
    double frac = 1.0;
    int device = 0, sm_count = 1;
    cudaStream_t stream = nullptr;
    void *pool[2] = {nullptr, nullptr};
    void *scratch = nullptr;      // the two-phase pass's j-ordered copy (n = 8, binary64 pools)
    void *l2sync = nullptr;       // barrier and accumulators of the multi-pass L2 kernel
    int l2_grid = 0;              // its CTAs (0: two per SM)
    int cur = 0;
    int64_t pass_index = 0;   // passes launched (selects a pass's strides slot)
    uint32_t seed = 0, stream_id = 0;
    int64_t restart = 0;          // refill interval in passes (0: never)
    int msigns = 0;               // per-pass sign patterns (WALLACE_MATRIX_SIGNS)
    int64_t restarted_at = 0;     // pass index of the last refill
    WlDevState *st = nullptr;
    int64_t cursor = 0;
    int status = 0;
    int variant = WALLACE_VARIANT_AUTO;
    int timing = 0;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    double kernel_ms = 0.0;
    int64_t kernel_launches = 0;
    int64_t launches = 0;   // pass and drain kernels, always counted
    // host-fill pipeline
    float *stage[2] = {nullptr, nullptr};
    int64_t stage_cap = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_done[2] = {nullptr, nullptr};
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
};

namespace {

size_t elem_size(const wallace_t *h) { return h->mode == WALLACE_FP64POOL ? 8 : 4; }

int cuda_fail(wallace_t *h, cudaError_t e)
{
    if (e == cudaSuccess)
        return WALLACE_OK;
    if (h)
        h->status |= WALLACE_ECUDA;
    return WALLACE_ECUDA;
}

cudaEvent_t take_event(wallace_t *h)
{
    if (!h->ev_free.empty()) {
        cudaEvent_t e = h->ev_free.back();
        h->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct KernelTimer {
    wallace_t *h;
    cudaEvent_t a = nullptr, b = nullptr;
    explicit KernelTimer(wallace_t *hh) : h(hh)
    {
        h->launches++;
        if (h->timing) {
            a = take_event(h);
            b = take_event(h);
            cudaEventRecord(a, h->stream);
        }
    }
    ~KernelTimer()
    {
        if (h->timing && a && b) {
            cudaEventRecord(b, h->stream);
            h->ev_pending.emplace_back(a, b);
        }
    }
};

void collect_timing(wallace_t *h)
{
    for (auto &p : h->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            h->kernel_ms += ms;
            h->kernel_launches += 1;
        }
        h->ev_free.push_back(p.first);
        h->ev_free.push_back(p.second);
    }
    h->ev_pending.clear();
}

int pick_variant(const wallace_t *h)
{
    if (h->variant != WALLACE_VARIANT_AUTO)
        return h->variant;
    const int fp64 = h->mode == WALLACE_FP64POOL;
    // pools too large for shared memory but small enough to stay in L2:
    // every pass of a fill in one launch
    if (h->l2sync && h->nu <= WL_L2RUN_AUTO_MAX_VALUES && !wl_fused_supported(h->n, h->N, fp64, nullptr))
        return WALLACE_VARIANT_L2RUN;
    if (wl_tma8_supported(h->n, h->N, fp64) && !wl_fused_supported(h->n, h->N, fp64, nullptr))
        return WALLACE_VARIANT_TILED;
    // a handle with the two-phase buffer has strides the tiled kernels cannot
    // tile (n = 8 with N a multiple of 3, 5 or 7, or n = 4 with more than 315
    // lanes)
    if (h->scratch && !wl_fused_supported(h->n, h->N, fp64, nullptr))
        return WALLACE_VARIANT_TWOPHASE;
    if (wl_tiled_supported(h->n, h->N, fp64) || wl_tma_supported(h->n, h->N, fp64, h->sm_count))
        return WALLACE_VARIANT_TILED;
    if (wl_fused_supported(h->n, h->N, fp64, nullptr))
        return WALLACE_VARIANT_FUSED;
    return WALLACE_VARIANT_GATHER;
}

// Largest stride a pass of (n, N) can draw (the n = 4, 8 candidates are the
// odd divisors of p^2 q, p^2 q r; n = 2's fallback stays below 64): the
// two-phase pass needs every stride within its shared-memory block.
int64_t max_stride(int n, int64_t N)
{
    if (n == 2)
        return 64;
    const int64_t P[17] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61};
    int64_t pr[3] = {0, 0, 0};
    int got = 0;
    for (int k = 0; k < 17 && got < 3; k++)
        if (N % P[k] != 0)
            pr[got++] = P[k];
    return n == 8 ? pr[0] * pr[0] * pr[1] * pr[2] : pr[0] * pr[0] * pr[1];
}

// One pass on the device.  Values q in [w0, w1) of the new pool are also
// written, mapped, to out[q - w0].
// Section 5 (restarting): before the pass that follows every `restart`
// passes, refill the current pool by Box-Muller (restart r takes uniforms
// [r 2^40, r 2^40 + nu) of the generator's sequence) and take the scale and
// drift history afresh from it.
cudaError_t maybe_restart(wallace_t *h)
{
    if (h->restart <= 0 || h->pass_index == 0 || h->pass_index % h->restart != 0 ||
        h->restarted_at == h->pass_index)
        return cudaSuccess;
    h->restarted_at = h->pass_index;
    h->launches++;
    return wl_launch_restart(h->pool[h->cur], h->mode == WALLACE_FP64POOL, h->n, h->N, h->Np,
                             h->seed, h->stream_id, h->pass_index / h->restart, h->st,
                             h->sm_count, h->stream);
}

int l2_grid(const wallace_t *h)
{
    return h->l2_grid > 0 ? h->l2_grid : wl_l2run_grid(h->nu, h->sm_count);
}

int launch_pass(wallace_t *h, void *out, int64_t w0, int64_t w1, double mu, double sigma)
{
    const int fp64 = h->mode == WALLACE_FP64POOL;
    const int v = pick_variant(h);
    cudaError_t e = maybe_restart(h);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    if (v == WALLACE_VARIANT_L2RUN) {
        KernelTimer t(h);
        // one pass of the multi-pass kernel: output window is a prefix
        e = wl_launch_l2run(h->pool[0], h->pool[1], h->cur, h->n, h->N, h->Np, h->st, h->l2sync, 1, h->R,
                            w1 - w0, out, mu, sigma, l2_grid(h), h->msigns, h->stream);
        h->pass_index += 1;
        h->cur = 1 - h->cur;
        return cuda_fail(h, e);
    }
    if (v == WALLACE_VARIANT_FUSED) {
        KernelTimer t(h);
        // a single fused pass: output window must start at 0 (a prefix)
        e = wl_launch_fused(h->pool[h->cur], h->pool[1 - h->cur], fp64, h->n, h->N, h->Np, h->st,
                            1, h->R, w1 - w0, out, mu, sigma, h->stream);
        h->pass_index += 1;
        // fused writes the new pool back in place: current buffer unchanged
        return cuda_fail(h, e);
    }
    WlPassArgs a;
    a.src = h->pool[h->cur];
    a.dst = h->pool[1 - h->cur];
    a.n = h->n;
    a.N = h->N;
    a.Np = h->Np;
    a.nu = h->nu;
    a.st = h->st;
    a.out = out;
    a.w0 = w0;
    a.w1 = w1;
    a.mu = mu;
    a.sigma = sigma;
    a.pass = h->pass_index;
    {
        KernelTimer t(h);
        if ((v == WALLACE_VARIANT_TILED || v == WALLACE_VARIANT_TILED_TMA) &&
            wl_tma_supported(h->n, h->N, fp64, h->sm_count))
            e = wl_launch_tma(a, h->sm_count, h->msigns, h->stream);
        else if ((v == WALLACE_VARIANT_TILED_CLUSTER ||
                  (v == WALLACE_VARIANT_TILED && wl_tma8c_preferred(h->n, h->N, fp64))) &&
                 wl_tma8c_supported(h->n, h->N, fp64)) {
            e = wl_launch_tma8c(a, h->sm_count, h->msigns, h->stream);
            if (wl_tma8_return_kernel(a))
                h->launches++;   // the returned values' kernel
        }
        else if ((v == WALLACE_VARIANT_TILED || v == WALLACE_VARIANT_TILED_TMA) &&
                 wl_tma8_supported(h->n, h->N, fp64)) {
            e = wl_launch_tma8(a, h->sm_count, h->msigns, h->stream);
            if (wl_tma8_return_kernel(a))
                h->launches++;   // the returned values' kernel
        }
        else if ((v == WALLACE_VARIANT_TILED || v == WALLACE_VARIANT_TILED_ASYNC ||
                  v == WALLACE_VARIANT_TILED_TMA) &&
                 wl_tiled_supported(h->n, h->N, fp64))
            e = wl_launch_tiled(a, h->sm_count, h->stream);
        else if (v == WALLACE_VARIANT_TWOPHASE && h->scratch) {
            e = wl_launch_twophase(a, h->scratch, fp64, h->sm_count, h->stream);
            h->launches++;   // its second kernel
        } else
            e = wl_launch_gather(a, fp64, h->sm_count, h->stream);
    }
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    h->cur = 1 - h->cur;
    h->pass_index += 1;
    return WALLACE_OK;
}

int fill_impl(wallace_t *h, void *out, int64_t count, double mu, double sigma)
{
    const int fp64 = h->mode == WALLACE_FP64POOL;
    const size_t es = elem_size(h);
    char *o = (char *)out;
    int64_t done = 0;
    // values of the current pool not yet handed out
    if (h->cursor < h->R && count > 0) {
        int64_t take = h->R - h->cursor;
        if (take > count)
            take = count;
        h->launches++;
        cudaError_t e = wl_launch_drain(h->pool[h->cur], fp64, h->N, h->Np, h->cursor, take, o, mu,
                                        sigma, h->sm_count, h->stream);
        if (e != cudaSuccess)
            return cuda_fail(h, e);
        h->cursor += take;
        done += take;
    }
    if (done >= count)
        return WALLACE_OK;
    int64_t remaining = count - done;
    if (pick_variant(h) == WALLACE_VARIANT_L2RUN && h->restart == 0) {
        // all remaining passes in cooperative launches of up to 2^20 passes
        int64_t passes = (remaining + h->R - 1) / h->R;
        while (passes > 0) {
            const int64_t P = passes < ((int64_t)1 << 20) ? passes : ((int64_t)1 << 20);
            const int64_t take_last = P < passes ? h->R : remaining - (passes - 1) * h->R;
            cudaError_t e;
            {
                KernelTimer t(h);
                e = wl_launch_l2run(h->pool[0], h->pool[1], h->cur, h->n, h->N, h->Np, h->st, h->l2sync, P,
                                    h->R, take_last, o + done * es, mu, sigma, l2_grid(h), h->msigns,
                                    h->stream);
            }
            if (e != cudaSuccess)
                return cuda_fail(h, e);
            h->pass_index += P;
            if (P & 1)
                h->cur = 1 - h->cur;
            const int64_t got = (P - 1) * h->R + take_last;
            done += got;
            remaining -= got;
            passes -= P;
            h->cursor = take_last;
        }
        return WALLACE_OK;
    }
    if (pick_variant(h) == WALLACE_VARIANT_FUSED && h->restart == 0) {
        // all remaining passes in one launch (pass by pass when refills are due)
        int64_t passes = (remaining + h->R - 1) / h->R;
        int64_t last = remaining - (passes - 1) * h->R;
        cudaError_t e;
        {
            KernelTimer t(h);
            e = wl_launch_fused(h->pool[h->cur], h->pool[1 - h->cur], fp64, h->n, h->N, h->Np,
                                h->st, passes, h->R, last, o + done * es, mu, sigma, h->stream);
        }
        h->pass_index += passes;
        if (e != cudaSuccess)
            return cuda_fail(h, e);
        h->cursor = last;
        return WALLACE_OK;
    }
    while (remaining > 0) {
        int64_t take = remaining < h->R ? remaining : h->R;
        int rc = launch_pass(h, o + done * es, 0, take, mu, sigma);
        if (rc)
            return rc;
        h->cursor = take;
        done += take;
        remaining -= take;
    }
    return WALLACE_OK;
}

int check(const wallace_t *h) { return h ? WALLACE_OK : WALLACE_EINVAL; }

} // namespace

extern "C" {

const char *wallace_strerror(int code)
{
    if (code == 0)
        return "ok";
    if (code & WALLACE_EINVAL)
        return "invalid argument";
    if (code & WALLACE_ENOMEM)
        return "out of memory";
    if (code & WALLACE_ECORRUPT)
        return "sum-of-squares check failed: pool overwritten or corrupt";
    if (code & WALLACE_ECUDA)
        return "CUDA runtime error";
    if (code & WALLACE_ETIMEOUT)
        return "device-side wait timed out";
    if (code & WALLACE_ESTATE)
        return "call not valid in this mode";
    return "unknown status";
}

int wallace_create_ex(int n, int64_t N, uint32_t seed, uint32_t stream_id, double frac, int mode,
                      void *cuda_stream, wallace_t **out)
{
    if (!out)
        return WALLACE_EINVAL;
    *out = nullptr;
    if ((n != 2 && n != 4 && n != 8) || N < 4 || (int64_t)n * N > ((int64_t)1 << 30))
        return WALLACE_EINVAL;
    const int opts = ((mode & WALLACE_CHI_WH) ? 1 : 0) | ((mode & WALLACE_MATRIX_SIGNS) ? 2 : 0);
    mode &= ~(WALLACE_CHI_WH | WALLACE_MATRIX_SIGNS);
    if (n == 2 && (opts & 2))
        return WALLACE_EINVAL;   // RANN4 draws its own rotation each pass
    if (!(frac > 0.0 && frac <= 1.0) || (mode != WALLACE_FP32 && mode != WALLACE_FP64POOL))
        return WALLACE_EINVAL;
    const int64_t nu = (int64_t)n * N;
    // R = min(floor(frac nu), nu - 1): the last value feeds Eq. 3 (Section 4)
    double rr = frac * (double)nu;
    int64_t R = (int64_t)rr;
    if (R > nu - 1)
        R = nu - 1;
    if (R < 1)
        return WALLACE_EINVAL;
    wallace_t *h = new (std::nothrow) wallace;
    if (!h)
        return WALLACE_ENOMEM;
    h->n = n;
    h->N = N;
    h->Np = ((N + 8 + 63) / 64) * 64;   // row pitch: >= 8 spare elements, 256-byte rows
    h->nu = nu;
    h->R = R;
    h->frac = frac;
    h->mode = mode;
    h->msigns = (opts >> 1) & 1;
    h->seed = seed;
    h->stream_id = stream_id;
    h->stream = (cudaStream_t)cuda_stream;
    h->cursor = R;   // the initial pool is not returned
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return WALLACE_ECUDA;
    }
    const size_t bytes = elem_size(h) * (size_t)n * (size_t)h->Np;
    for (int b = 0; b < 2; b++) {
        if (cudaMalloc(&h->pool[b], bytes) != cudaSuccess) {
            wallace_destroy(h);
            return WALLACE_ENOMEM;
        }
    }
    if (cudaMalloc((void **)&h->st, sizeof(WlDevState)) != cudaSuccess) {
        wallace_destroy(h);
        return WALLACE_ENOMEM;
    }
    // binary32 pools whose strides the lane-tiled kernels cannot tile (n = 8:
    // 315 lanes; n = 4 with N a multiple of 15: 539 lanes or more) get the
    // two-phase pass's scratch copy, when every stride this N can draw fits
    // its block (else they keep the plain gather; binary64 pools keep it too:
    // their transform is bound by the binary64 units)
    const int64_t ms = max_stride(n, N);
    if (mode == WALLACE_FP32 && (n == 8 || (n == 4 && ms > 315)) && ms <= WL_TWOPHASE_MAX_STRIDE &&
        cudaMalloc(&h->scratch, bytes) != cudaSuccess) {
        wallace_destroy(h);
        return WALLACE_ENOMEM;
    }
    if (wl_l2run_supported(n, N, mode == WALLACE_FP64POOL, max_stride(n, N)) &&
        cudaMalloc(&h->l2sync, wl_l2run_sync_bytes()) != cudaSuccess) {
        wallace_destroy(h);
        return WALLACE_ENOMEM;
    }
    e = cudaMemsetAsync(h->pool[0], 0, bytes, h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->pool[1], 0, bytes, h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->st, 0, sizeof(WlDevState), h->stream);
    if (e == cudaSuccess)
        e = wl_launch_init(h->pool[0], mode == WALLACE_FP64POOL, n, N, h->Np, seed, stream_id,
                           h->st, h->sm_count, h->stream, opts);
    if (e != cudaSuccess) {
        wallace_destroy(h);
        return WALLACE_ECUDA;
    }
    *out = h;
    return WALLACE_OK;
}

int wallace_create(int n, int64_t N, uint32_t seed, double frac, wallace_t **out)
{
    return wallace_create_ex(n, N, seed, 0, frac, WALLACE_FP32, nullptr, out);
}

void wallace_destroy(wallace_t *h)
{
    if (!h)
        return;
    cudaStreamSynchronize(h->stream);
    if (h->copy_stream)
        cudaStreamSynchronize(h->copy_stream);
    cudaFree(h->scratch);
    cudaFree(h->l2sync);
    for (int b = 0; b < 2; b++) {
        cudaFree(h->pool[b]);
        cudaFree(h->stage[b]);
        if (h->stage_done[b])
            cudaEventDestroy(h->stage_done[b]);
        if (h->copy_done[b])
            cudaEventDestroy(h->copy_done[b]);
    }
    cudaFree(h->st);
    if (h->copy_stream)
        cudaStreamDestroy(h->copy_stream);
    for (auto &p : h->ev_pending) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    for (auto e : h->ev_free)
        cudaEventDestroy(e);
    delete h;
}

int wallace_pass(wallace_t *h)
{
    if (check(h))
        return WALLACE_EINVAL;
    int rc = launch_pass(h, nullptr, 0, 0, 0.0, 1.0);
    if (rc)
        return rc;
    h->cursor = 0;
    return h->status;
}

int wallace_fill(wallace_t *h, float *out, int64_t count, float mu, float sigma)
{
    if (check(h) || count < 0 || (count > 0 && !out))
        return WALLACE_EINVAL;
    if (h->mode != WALLACE_FP32)
        return WALLACE_ESTATE;
    int rc = fill_impl(h, out, count, (double)mu, (double)sigma);
    return rc ? rc : h->status;
}

int wallace_fill64(wallace_t *h, double *out, int64_t count, double mu, double sigma)
{
    if (check(h) || count < 0 || (count > 0 && !out))
        return WALLACE_EINVAL;
    if (h->mode != WALLACE_FP64POOL)
        return WALLACE_ESTATE;
    int rc = fill_impl(h, out, count, mu, sigma);
    return rc ? rc : h->status;
}

int wallace_fill_host(wallace_t *h, float *host_out, int64_t count, float mu, float sigma)
{
    if (check(h) || count < 0 || (count > 0 && !host_out))
        return WALLACE_EINVAL;
    if (h->mode != WALLACE_FP32)
        return WALLACE_ESTATE;
    if (count == 0)
        return h->status;
    // chunks of one pass's returned values, double-buffered in device memory
    const int64_t chunk = h->R;
    if (h->stage_cap < chunk) {
        for (int b = 0; b < 2; b++) {
            cudaFree(h->stage[b]);
            h->stage[b] = nullptr;
        }
        h->stage_cap = 0;
        for (int b = 0; b < 2; b++)
            if (cudaMalloc((void **)&h->stage[b], sizeof(float) * (size_t)chunk) != cudaSuccess)
                return WALLACE_ENOMEM;
        h->stage_cap = chunk;
    }
    cudaError_t e = cudaSuccess;
    if (!h->copy_stream) {
        e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; b++) {
            e = cudaEventCreateWithFlags(&h->stage_done[b], cudaEventDisableTiming);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&h->copy_done[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess)
            return cuda_fail(h, e);
    }
    int64_t done = 0;
    int k = 0;
    bool used[2] = {false, false};
    while (done < count) {
        const int b = k & 1;
        int64_t take = count - done < chunk ? count - done : chunk;
        if (used[b])
            cudaStreamWaitEvent(h->stream, h->copy_done[b], 0);
        int rc = fill_impl(h, h->stage[b], take, (double)mu, (double)sigma);
        if (rc)
            return rc;
        e = cudaEventRecord(h->stage_done[b], h->stream);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(h->copy_stream, h->stage_done[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_out + done, h->stage[b], sizeof(float) * (size_t)take,
                                cudaMemcpyDeviceToHost, h->copy_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(h->copy_done[b], h->copy_stream);
        if (e != cudaSuccess)
            return cuda_fail(h, e);
        used[b] = true;
        done += take;
        k++;
    }
    e = cudaStreamSynchronize(h->copy_stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    return h->status;
}

int wallace_set_stream(wallace_t *h, void *cuda_stream)
{
    if (check(h))
        return WALLACE_EINVAL;
    h->stream = (cudaStream_t)cuda_stream;
    return WALLACE_OK;
}

int wallace_set_variant(wallace_t *h, int variant)
{
    if (check(h))
        return WALLACE_EINVAL;
    const int fp64 = h->mode == WALLACE_FP64POOL;
    switch (variant) {
    case WALLACE_VARIANT_AUTO:
    case WALLACE_VARIANT_GATHER:
        break;
    case WALLACE_VARIANT_TILED:
    case WALLACE_VARIANT_TILED_TMA:
        if (!wl_tiled_supported(h->n, h->N, fp64) && !wl_tma_supported(h->n, h->N, fp64, h->sm_count) &&
            !wl_tma8_supported(h->n, h->N, fp64))
            return WALLACE_EINVAL;
        break;
    case WALLACE_VARIANT_TILED_ASYNC:
        if (!wl_tiled_supported(h->n, h->N, fp64))
            return WALLACE_EINVAL;
        break;
    case WALLACE_VARIANT_TWOPHASE:
        if (!h->scratch)
            return WALLACE_EINVAL;
        break;
    case WALLACE_VARIANT_FUSED:
        if (!wl_fused_supported(h->n, h->N, fp64, nullptr))
            return WALLACE_EINVAL;
        break;
    case WALLACE_VARIANT_L2RUN:
        if (!h->l2sync)
            return WALLACE_EINVAL;
        break;
    case WALLACE_VARIANT_TILED_CLUSTER:
        if (!wl_tma8c_supported(h->n, h->N, fp64))
            return WALLACE_EINVAL;
        break;
    default:
        return WALLACE_EINVAL;
    }
    h->variant = variant;
    return WALLACE_OK;
}

int wallace_set_l2_grid(wallace_t *h, int grid)
{
    if (check(h) || grid < 0)
        return WALLACE_EINVAL;
    h->l2_grid = grid;
    return WALLACE_OK;
}

int wallace_set_restart(wallace_t *h, int64_t interval)
{
    if (check(h) || interval < 0)
        return WALLACE_EINVAL;
    h->restart = interval;
    return WALLACE_OK;
}

int wallace_set_timing(wallace_t *h, int on)
{
    if (check(h))
        return WALLACE_EINVAL;
    h->timing = on ? 1 : 0;
    return WALLACE_OK;
}

int wallace_sync(wallace_t *h)
{
    if (check(h))
        return WALLACE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    int32_t dev_status = 0;
    e = cudaMemcpy(&dev_status, &h->st->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    h->status |= dev_status;
    return h->status;
}

int wallace_stats(wallace_t *h, wallace_stats_t *out)
{
    if (check(h) || !out)
        return WALLACE_EINVAL;
    int rc = wallace_sync(h);
    if (rc & WALLACE_ECUDA)
        return rc;
    collect_timing(h);
    WlDevState s;
    cudaError_t e = cudaMemcpy(&s, h->st, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    memset(out, 0, sizeof(*out));
    out->q_lo = s.q_lo;
    out->q_hi = s.q_hi;
    out->q = s.q;
    out->S = s.S;
    out->c = s.c;
    out->c32 = s.next.c32;
    out->drift = s.drift;
    out->passes = s.passes;
    out->status = h->status | s.status;
    out->bad = s.bad;
    out->lcg = s.lcg_rep;
    for (int i = 0; i < 8; i++) {
        out->alpha[i] = s.last.alpha[i];
        out->gamma[i] = s.last.gamma[i];
    }
    out->R = h->R;
    out->cursor = h->cursor;
    out->kernel_ms = h->kernel_ms;
    out->kernel_launches = h->kernel_launches;
    out->signs = s.last.signs;
    out->rot_c = s.last.rcos;
    out->rot_s = s.last.rsin;
    out->launches = h->launches;
    return out->status;
}

static int copy_pool_out(wallace_t *h, void *host, int want64)
{
    if (check(h) || !host)
        return WALLACE_EINVAL;
    int rc = wallace_sync(h);
    if (rc & WALLACE_ECUDA)
        return rc;
    const size_t es = elem_size(h);
    std::vector<char> tmp((size_t)h->n * (size_t)h->Np * es);
    cudaError_t e = cudaMemcpy(tmp.data(), h->pool[h->cur], tmp.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    for (int64_t q = 0; q < h->nu; q++) {
        int64_t i = q / h->N, j = q - i * h->N;
        size_t off = (size_t)(i * h->Np + j);
        if (es == 8) {
            double v = ((double *)tmp.data())[off];
            if (want64)
                ((double *)host)[q] = v;
            else
                ((float *)host)[q] = (float)v;
        } else {
            float v = ((float *)tmp.data())[off];
            if (want64)
                ((double *)host)[q] = (double)v;
            else
                ((float *)host)[q] = v;
        }
    }
    return h->status;
}

int wallace_get_pool(wallace_t *h, float *host_out) { return copy_pool_out(h, host_out, 0); }

int wallace_get_pool64(wallace_t *h, double *host_out) { return copy_pool_out(h, host_out, 1); }

int wallace_set_pool(wallace_t *h, const float *host_in)
{
    if (check(h) || !host_in)
        return WALLACE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e);
    const size_t es = elem_size(h);
    std::vector<char> tmp((size_t)h->n * (size_t)h->Np * es, 0);
    for (int64_t q = 0; q < h->nu; q++) {
        int64_t i = q / h->N, j = q - i * h->N;
        size_t off = (size_t)(i * h->Np + j);
        if (es == 8)
            ((double *)tmp.data())[off] = (double)host_in[q];
        else
            ((float *)tmp.data())[off] = host_in[q];
    }
    e = cudaMemcpy(h->pool[h->cur], tmp.data(), tmp.size(), cudaMemcpyHostToDevice);
    return cuda_fail(h, e);
}

int wallace_clear_error(wallace_t *h)
{
    if (check(h))
        return WALLACE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(&h->st->status, 0, sizeof(int32_t), h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    h->status = 0;
    return e == cudaSuccess ? WALLACE_OK : cuda_fail(h, e);
}

int64_t wallace_returned_per_pass(const wallace_t *h) { return h ? h->R : -1; }

} // extern "C"
