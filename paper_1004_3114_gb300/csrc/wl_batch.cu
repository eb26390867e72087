// Many independent Wallace generators (Brent's RANN4 paper: independent
// streams need no communication after initialisation, Section 9) advanced
// together in one persistent launch.
//
// The CTAs take whole generators from a work counter, largest pool first.  A
// CTA runs every pass of its generator itself, so the end-of-pass sum of
// squares and chi-squared rescale (Eq. 3) are CTA-local (wl_end_pass_cta)
// and no CTA ever waits for another.  Two runners:
//   * per-thread async copies (batch_kernel, 1 to 3 CTAs of 256 threads per
//     SM): a pool that fits in shared memory is loaded once and regenerated
//     there for all passes (only the returned values go to global memory); a
//     larger n = 4 pool whose strides have lcm <= 315 runs the lane-tiled
//     gather (wl_tiled_body.cuh) over all of its tiles; anything else runs
//     the plain strided gather;
//   * bulk copies (batch_tma_kernel, one 608-thread CTA per SM): n = 4 pools
//     with N >= 16384 go through the warp-specialised stage ring
//     (wl_tma_run.cuh), the others as above.
// The launch is a CUDA graph (work-counter reset + kernel) whose kernel
// arguments are updated per run.  An autotuner times candidate settings
// (runner and CTAs per SM, tile size, shared-memory pool limit) on a
// snapshot of the generators and caches the best in a JSON-lines file.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "wallace.h"
#include "wl_launch.h"
#include "wl_run_body.cuh"
#include "wl_tma_run.cuh"

#define BT_THREADS 256

namespace {

struct BatchStream {
    float *pool[2];
    WlDevState *st;
    int64_t N, Np, R;
    int64_t out_pref;   // sum of R over the streams before this one (stream order)
    int32_t cur;
    int32_t n;
};

struct BatchArgs {
    BatchStream *streams;
    const int *order;
    int *queue;
    int count;
    int etarget;
    int64_t passes;
    int64_t fused_max;   // pools with n*N <= this stay in shared memory
    float *out;
    float mu, sigma;
    // output layout of the whole run this launch belongs to (a run split at
    // restart points): generator s writes pass p of the launch to
    // out + out_passes * pref_s + (pass0 + p) * R_s
    int64_t out_passes, pass0;
};

template <bool SG>   // the batch's generators draw a sign pattern each pass
__global__ void __launch_bounds__(BT_THREADS, 3) batch_kernel(BatchArgs a)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ uint64_t red[3 * (BT_THREADS / 32)];
    __shared__ int s_k;
    __shared__ WlDevState sst;   // the running generator's state
    const int tid = threadIdx.x;
    const int64_t smem_values = (int64_t)(tl_smem_bytes() / sizeof(float));
    while (true) {
        __syncthreads();
        if (tid == 0)
            s_k = atomicAdd(a.queue, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= a.count)
            break;
        const BatchStream d = a.streams[a.order[k]];
        WlRunSpec r;
        r.buf[0] = d.pool[0];
        r.buf[1] = d.pool[1];
        r.cur = d.cur;
        r.st = d.st;
        r.N = d.N;
        r.Np = d.Np;
        r.R = d.R;
        r.n = d.n;
        r.passes = a.passes;
        r.out = a.out ? a.out + a.out_passes * d.out_pref + a.pass0 * d.R : nullptr;
        r.last_take = d.R;
        r.mu = a.mu;
        r.sigma = a.sigma;
        r.etarget = a.etarget;
        wl_state_load(&sst, d.st);
        r.st = &sst;
        const int cur = wl_run_spec<SG>(r, a.fused_max, smem_values, smem, red);
        wl_state_store(d.st, &sst);
        if (tid == 0)
            a.streams[a.order[k]].cur = cur;
    }
}

// The same work with the CTA-local bulk-copy runner for the pools it takes
// (wl_tma_run_eligible: n = 4, N >= TR_MIN_N): one CTA of TM_THREADS threads
// per SM; the other pools as in batch_kernel.
// SG: the batch's generators draw a sign pattern each pass (matrix A D_k)
template <bool SG>
__global__ void __launch_bounds__(TM_THREADS, 1) batch_tma_kernel(BatchArgs a)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ uint64_t red[3 * (TM_THREADS / 32 + 1)];
    __shared__ int s_k;
    __shared__ __align__(8) uint64_t bar_full[TR_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[TR_STAGES];
    __shared__ volatile int s_abort;
    __shared__ WlDevState sst;   // the running generator's state
    WlTmaRing ring;
    ring.full = bar_full;
    ring.empty = bar_empty;
    ring.abort_flag = &s_abort;
    wl_tma_ring_init(ring);
    const int tid = threadIdx.x;
    const int64_t smem_values = (int64_t)(wl_tma::tr_smem_bytes() / sizeof(float));
    while (true) {
        __syncthreads();
        if (tid == 0)
            s_k = atomicAdd(a.queue, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= a.count)
            break;
        const BatchStream d = a.streams[a.order[k]];
        WlRunSpec r;
        r.buf[0] = d.pool[0];
        r.buf[1] = d.pool[1];
        r.cur = d.cur;
        r.st = d.st;
        r.N = d.N;
        r.Np = d.Np;
        r.R = d.R;
        r.n = d.n;
        r.passes = a.passes;
        r.out = a.out ? a.out + a.out_passes * d.out_pref + a.pass0 * d.R : nullptr;
        r.last_take = d.R;
        r.mu = a.mu;
        r.sigma = a.sigma;
        r.etarget = a.etarget;
        int cur;
        wl_state_load(&sst, d.st);
        r.st = &sst;
        if (wl_tma_run_eligible(d.n, d.N) && !wl_run_is_fused(4, d.N, a.fused_max, smem_values))
            cur = wl_run_tma<SG>(r, smem, red, ring);
        else
            cur = wl_run_spec<SG>(r, a.fused_max, smem_values, smem, red);
        wl_state_store(d.st, &sst);
        if (tid == 0)
            a.streams[a.order[k]].cur = cur;
    }
}

struct Tuning {
    int ctas_per_sm = 2;
    int etarget = TL_EMAX;
    int64_t fused_max = 4096;
    int runner = 0;   // 0: per-thread async-copy runner; 1: bulk-copy runner (batch_tma_kernel)
};

} // namespace

struct wallace_batch {
    int count = 0, n = 4;
    double frac = 1.0;
    std::vector<int64_t> N, Np, R, pref;
    std::vector<int> order;
    std::vector<size_t> pool_off;   // float offset of each stream's first buffer in the arena
    size_t arena_floats = 0;
    float *arena = nullptr;
    WlDevState *states = nullptr;
    BatchStream *d_streams = nullptr;
    int *d_order = nullptr;
    int *d_queue = nullptr;
    cudaStream_t stream = nullptr;
    int sm_count = 1, device = 0, max_ctas_per_sm = 1;
    Tuning tune;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    int graph_ctas = 0;
    int graph_runner = -1;
    int status = 0;
    double last_run_ms = 0.0;
    std::vector<uint32_t> seed;
    int opts = 0;                 // wl_launch_init options: Wilson-Hilferty sample, sign patterns
    int64_t restart = 0;          // refill every generator before the pass after each multiple of this
    int64_t passes_done = 0;      // passes every generator has run (all advance together)
    int64_t restarted_at = 0;
};

namespace {

int bfail(wallace_batch_t *b, cudaError_t e)
{
    if (e == cudaSuccess)
        return WALLACE_OK;
    if (b)
        b->status |= WALLACE_ECUDA;
    return WALLACE_ECUDA;
}

// Restart r of every generator: its current pool refilled by Box-Muller
// from uniforms [r 2^40, r 2^40 + nu) of its sequence, the scale and drift
// history taken afresh (the single-generator refill, one launch each; the
// buffer each pool is in is read back from the device first).
cudaError_t refill_all(wallace_batch_t *b, int64_t r)
{
    std::vector<BatchStream> hs(b->count);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(hs.data(), b->d_streams, sizeof(BatchStream) * (size_t)b->count, cudaMemcpyDeviceToHost);
    for (int s = 0; s < b->count && e == cudaSuccess; s++)
        e = wl_launch_restart(hs[s].pool[hs[s].cur], 0, b->n, b->N[s], b->Np[s], b->seed[s], 0, r, hs[s].st,
                              b->sm_count, b->stream);
    return e;
}

BatchArgs make_args(wallace_batch_t *b, int64_t passes, float *out, float mu, float sigma)
{
    BatchArgs a;
    a.streams = b->d_streams;
    a.order = b->d_order;
    a.queue = b->d_queue;
    a.count = b->count;
    a.etarget = b->tune.etarget;
    a.passes = passes;
    a.fused_max = b->tune.fused_max;
    a.out = out;
    a.mu = mu;
    a.sigma = sigma;
    a.out_passes = passes;
    a.pass0 = 0;
    return a;
}

cudaError_t ensure_configured()
{
    static bool done = false;
    if (done)
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tl_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tl_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_tma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wl_tma::tr_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_tma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wl_tma::tr_smem_bytes());
    if (e == cudaSuccess)
        done = true;
    return e;
}

// Graph: reset the work counter, then the persistent kernel.  Rebuilt when the
// CTA count changes; otherwise only the kernel's arguments are updated.
cudaError_t launch_graph(wallace_batch_t *b, const BatchArgs &args)
{
    cudaError_t e = ensure_configured();
    if (e != cudaSuccess)
        return e;
    const bool tma = b->tune.runner == 1;
    const int ctas = tma ? b->sm_count : b->sm_count * std::min(b->tune.ctas_per_sm, b->max_ctas_per_sm);
    BatchArgs a = args;
    void *params[] = {&a};
    cudaKernelNodeParams kp = {};
    kp.func = tma ? ((b->opts & 2) ? (void *)batch_tma_kernel<true> : (void *)batch_tma_kernel<false>)
                  : ((b->opts & 2) ? (void *)batch_kernel<true> : (void *)batch_kernel<false>);
    kp.gridDim = dim3(ctas);
    kp.blockDim = dim3(tma ? TM_THREADS : BT_THREADS);
    kp.sharedMemBytes = (unsigned)(tma ? wl_tma::tr_smem_bytes() : tl_smem_bytes());
    kp.kernelParams = params;
    if (!b->exec || b->graph_ctas != ctas || b->graph_runner != b->tune.runner) {
        if (b->exec)
            cudaGraphExecDestroy(b->exec);
        if (b->graph)
            cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        e = cudaGraphCreate(&b->graph, 0);
        if (e != cudaSuccess)
            return e;
        cudaMemsetParams mp = {};
        mp.dst = b->d_queue;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 1;
        mp.height = 1;
        cudaGraphNode_t mnode;
        e = cudaGraphAddMemsetNode(&mnode, b->graph, nullptr, 0, &mp);
        if (e == cudaSuccess)
            e = cudaGraphAddKernelNode(&b->knode, b->graph, &mnode, 1, &kp);
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess)
            return e;
        b->graph_ctas = ctas;
        b->graph_runner = b->tune.runner;
    } else {
        e = cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp);
        if (e != cudaSuccess)
            return e;
    }
    return cudaGraphLaunch(b->exec, b->stream);
}

std::string tune_key(const wallace_batch_t *b)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, b->device);
    // pool-size histogram on powers of two, plus count, n and frac
    std::vector<int> hist(40, 0);
    for (int s = 0; s < b->count; s++) {
        int lg = 0;
        while (((int64_t)1 << (lg + 1)) <= b->N[s] && lg < 39)
            lg++;
        hist[lg]++;
    }
    std::string k = std::string(prop.name) + "|sm" + std::to_string(b->sm_count) + "|n" +
                    std::to_string(b->n) + "|count" + std::to_string(b->count) + "|frac" +
                    std::to_string(b->frac) + "|h";
    for (int v : hist)
        k += std::to_string(v) + ",";
    for (char &ch : k)
        if (ch == '"' || ch == '\n')
            ch = '_';
    return k;
}

bool read_cached(const char *path, const std::string &key, Tuning *t)
{
    if (!path)
        return false;
    FILE *f = fopen(path, "r");
    if (!f)
        return false;
    char line[8192];
    bool found = false;
    const std::string needle = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof line, f)) {
        if (!strstr(line, needle.c_str()))
            continue;
        int ctas = 0, et = 0, runner = 0;
        long long fm = 0;
        const char *pc = strstr(line, "\"ctas_per_sm\": ");
        const char *pe = strstr(line, "\"etarget\": ");
        const char *pf = strstr(line, "\"fused_max\": ");
        const char *pr = strstr(line, "\"runner\": ");
        if (pc && pe && pf && pr && sscanf(pc, "\"ctas_per_sm\": %d", &ctas) == 1 &&
            sscanf(pe, "\"etarget\": %d", &et) == 1 && sscanf(pf, "\"fused_max\": %lld", &fm) == 1 &&
            sscanf(pr, "\"runner\": %d", &runner) == 1) {
            t->ctas_per_sm = ctas;
            t->etarget = et;
            t->fused_max = fm;
            t->runner = runner;
            found = true;   // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

} // namespace

extern "C" {

int wallace_batch_create(int count, int n, const int64_t *N, const uint32_t *seed, double frac,
                         void *cuda_stream, wallace_batch_t **out)
{
    return wallace_batch_create_ex(count, n, N, seed, frac, WALLACE_FP32, cuda_stream, out);
}

int wallace_batch_create_ex(int count, int n, const int64_t *N, const uint32_t *seed, double frac, int mode,
                            void *cuda_stream, wallace_batch_t **out)
{
    if (!out || count < 1 || !N || !seed || (n != 4 && n != 8) || !(frac > 0.0 && frac <= 1.0) ||
        (mode & ~(WALLACE_CHI_WH | WALLACE_MATRIX_SIGNS)) != WALLACE_FP32)
        return WALLACE_EINVAL;
    *out = nullptr;
    wallace_batch_t *b = new (std::nothrow) wallace_batch;
    if (!b)
        return WALLACE_ENOMEM;
    b->count = count;
    b->n = n;
    b->frac = frac;
    b->seed.assign(seed, seed + count);
    b->opts = ((mode & WALLACE_CHI_WH) ? 1 : 0) | ((mode & WALLACE_MATRIX_SIGNS) ? 2 : 0);
    b->stream = (cudaStream_t)cuda_stream;
    b->N.resize(count);
    b->Np.resize(count);
    b->R.resize(count);
    b->pref.resize(count);
    b->pool_off.resize(count);
    int64_t pr = 0;
    for (int s = 0; s < count; s++) {
        const int64_t Ns = N[s];
        if (Ns < 4 || (int64_t)n * Ns > ((int64_t)1 << 30)) {
            delete b;
            return WALLACE_EINVAL;
        }
        const int64_t nu = (int64_t)n * Ns;
        int64_t R = (int64_t)(frac * (double)nu);
        if (R > nu - 1)
            R = nu - 1;
        if (R < 1) {
            delete b;
            return WALLACE_EINVAL;
        }
        b->N[s] = Ns;
        b->Np[s] = ((Ns + 8 + 63) / 64) * 64;
        b->R[s] = R;
        b->pref[s] = pr;
        pr += R;
        b->pool_off[s] = b->arena_floats;
        b->arena_floats += 2 * (size_t)n * (size_t)b->Np[s];
    }
    // largest pools first (longest-processing-time order)
    b->order.resize(count);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->N[x] > b->N[y]; });
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess)
        e = ensure_configured();
    if (e == cudaSuccess) {
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<true>, BT_THREADS, tl_smem_bytes());
        b->max_ctas_per_sm = per > 0 ? per : 1;
    }
    if (e != cudaSuccess) {
        delete b;
        return WALLACE_ECUDA;
    }
    if (cudaMalloc(&b->arena, sizeof(float) * b->arena_floats) != cudaSuccess ||
        cudaMalloc(&b->states, sizeof(WlDevState) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&b->d_streams, sizeof(BatchStream) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&b->d_order, sizeof(int) * (size_t)count) != cudaSuccess ||
        cudaMalloc(&b->d_queue, sizeof(int)) != cudaSuccess) {
        wallace_batch_destroy(b);
        return WALLACE_ENOMEM;
    }
    std::vector<BatchStream> hs(count);
    for (int s = 0; s < count; s++) {
        float *p0 = b->arena + b->pool_off[s];
        hs[s].pool[0] = p0;
        hs[s].pool[1] = p0 + (size_t)n * (size_t)b->Np[s];
        hs[s].st = b->states + s;
        hs[s].N = b->N[s];
        hs[s].Np = b->Np[s];
        hs[s].R = b->R[s];
        hs[s].out_pref = b->pref[s];
        hs[s].cur = 0;
        hs[s].n = n;
    }
    e = cudaMemsetAsync(b->arena, 0, sizeof(float) * b->arena_floats, b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->states, 0, sizeof(WlDevState) * (size_t)count, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_streams, hs.data(), sizeof(BatchStream) * (size_t)count,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_order, b->order.data(), sizeof(int) * (size_t)count,
                            cudaMemcpyHostToDevice, b->stream);
    for (int s = 0; s < count && e == cudaSuccess; s++)
        e = wl_launch_init(hs[s].pool[0], 0, n, b->N[s], b->Np[s], seed[s], 0, b->states + s,
                           b->sm_count, b->stream, b->opts);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        wallace_batch_destroy(b);
        return WALLACE_ECUDA;
    }
    *out = b;
    return WALLACE_OK;
}

void wallace_batch_destroy(wallace_batch_t *b)
{
    if (!b)
        return;
    cudaStreamSynchronize(b->stream);
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    cudaFree(b->arena);
    cudaFree(b->states);
    cudaFree(b->d_streams);
    cudaFree(b->d_order);
    cudaFree(b->d_queue);
    delete b;
}

int64_t wallace_batch_returned_per_pass(const wallace_batch_t *b, int s)
{
    if (!b || s < 0 || s >= b->count)
        return -1;
    return b->R[s];
}

int64_t wallace_batch_out_offset(const wallace_batch_t *b, int s, int64_t passes)
{
    if (!b || s < 0 || s > b->count || passes < 0)
        return -1;
    if (s == b->count)
        return passes * (b->pref[b->count - 1] + b->R[b->count - 1]);
    return passes * b->pref[s];
}

int wallace_batch_run(wallace_batch_t *b, int64_t passes, float *out, float mu, float sigma)
{
    if (!b || passes < 0)
        return WALLACE_EINVAL;
    if (passes == 0)
        return b->status;
    if (b->restart <= 0) {
        cudaError_t e = launch_graph(b, make_args(b, passes, out, mu, sigma));
        if (e != cudaSuccess)
            return bfail(b, e);
        b->passes_done += passes;
        return b->status;
    }
    // Section 5 (restarting): the run is split at the restart points; before
    // the pass that follows each multiple of the interval every pool is
    // refilled, and the launches write into the whole run's output layout
    const int64_t K = b->restart;
    for (int64_t p = 0; p < passes;) {
        if (b->passes_done > 0 && b->passes_done % K == 0 && b->restarted_at != b->passes_done) {
            cudaError_t e = refill_all(b, b->passes_done / K);
            if (e != cudaSuccess)
                return bfail(b, e);
            b->restarted_at = b->passes_done;
        }
        const int64_t seg = std::min(passes - p, K - b->passes_done % K);
        BatchArgs a = make_args(b, seg, out, mu, sigma);
        a.out_passes = passes;
        a.pass0 = p;
        cudaError_t e = launch_graph(b, a);
        if (e != cudaSuccess)
            return bfail(b, e);
        p += seg;
        b->passes_done += seg;
    }
    return b->status;
}

int wallace_batch_set_restart(wallace_batch_t *b, int64_t interval)
{
    if (!b || interval < 0)
        return WALLACE_EINVAL;
    b->restart = interval;
    return WALLACE_OK;
}

int wallace_batch_sync(wallace_batch_t *b)
{
    if (!b)
        return WALLACE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bfail(b, e);
    std::vector<WlDevState> s(b->count);
    e = cudaMemcpy(s.data(), b->states, sizeof(WlDevState) * (size_t)b->count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return bfail(b, e);
    int st = 0;
    for (auto &x : s)
        st |= x.status;
    return b->status | st;
}

int wallace_batch_stats(wallace_batch_t *b, int s, wallace_stats_t *out)
{
    if (!b || s < 0 || s >= b->count || !out)
        return WALLACE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bfail(b, e);
    WlDevState x;
    e = cudaMemcpy(&x, b->states + s, sizeof(x), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return bfail(b, e);
    memset(out, 0, sizeof(*out));
    out->q_lo = x.q_lo;
    out->q_hi = x.q_hi;
    out->q = x.q;
    out->S = x.S;
    out->c = x.c;
    out->c32 = x.next.c32;
    out->drift = x.drift;
    out->passes = x.passes;
    out->status = b->status | x.status;
    out->bad = x.bad;
    out->lcg = x.lcg_rep;
    for (int i = 0; i < 8; i++) {
        out->alpha[i] = x.last.alpha[i];
        out->gamma[i] = x.last.gamma[i];
    }
    out->R = b->R[s];
    out->cursor = b->R[s];
    out->signs = x.last.signs;
    out->kernel_ms = b->last_run_ms;
    return out->status;
}

int wallace_batch_get_pool(wallace_batch_t *b, int s, float *host_out)
{
    if (!b || s < 0 || s >= b->count || !host_out)
        return WALLACE_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bfail(b, e);
    BatchStream d;
    e = cudaMemcpy(&d, b->d_streams + s, sizeof(d), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return bfail(b, e);
    for (int i = 0; i < b->n && e == cudaSuccess; i++)
        e = cudaMemcpy(host_out + (size_t)i * b->N[s], d.pool[d.cur] + (size_t)i * b->Np[s],
                       sizeof(float) * (size_t)b->N[s], cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? b->status : bfail(b, e);
}

int wallace_batch_set_tuning(wallace_batch_t *b, int ctas_per_sm, int etarget, int64_t fused_max)
{
    if (!b || ctas_per_sm < 0 || etarget < 4 || etarget > TL_EMAX || fused_max < 0)
        return WALLACE_EINVAL;
    b->tune.runner = ctas_per_sm == 0 ? 1 : 0;
    b->tune.ctas_per_sm = ctas_per_sm == 0 ? 1 : ctas_per_sm;
    b->tune.etarget = etarget;
    b->tune.fused_max = fused_max;
    return WALLACE_OK;
}

int wallace_batch_get_tuning(const wallace_batch_t *b, int *ctas_per_sm, int *etarget, int64_t *fused_max)
{
    if (!b)
        return WALLACE_EINVAL;
    if (ctas_per_sm)
        *ctas_per_sm = b->tune.runner == 1 ? 0 : std::min(b->tune.ctas_per_sm, b->max_ctas_per_sm);
    if (etarget)
        *etarget = b->tune.etarget;
    if (fused_max)
        *fused_max = b->tune.fused_max;
    return WALLACE_OK;
}

int wallace_batch_autotune(wallace_batch_t *b, const char *cache_path, int trial_passes)
{
    if (!b || trial_passes < 1)
        return WALLACE_EINVAL;
    const std::string key = tune_key(b);
    Tuning cached;
    if (read_cached(cache_path, key, &cached)) {
        b->tune = cached;
        return WALLACE_OK;
    }
    // snapshot of pools, states and buffer indices: trials must not advance the generators
    float *bk_arena = nullptr;
    WlDevState *bk_states = nullptr;
    BatchStream *bk_streams = nullptr;
    cudaError_t e = cudaMalloc(&bk_arena, sizeof(float) * b->arena_floats);
    if (e == cudaSuccess)
        e = cudaMalloc(&bk_states, sizeof(WlDevState) * (size_t)b->count);
    if (e == cudaSuccess)
        e = cudaMalloc(&bk_streams, sizeof(BatchStream) * (size_t)b->count);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bk_arena, b->arena, sizeof(float) * b->arena_floats,
                            cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bk_states, b->states, sizeof(WlDevState) * (size_t)b->count,
                            cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bk_streams, b->d_streams, sizeof(BatchStream) * (size_t)b->count,
                            cudaMemcpyDeviceToDevice, b->stream);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess)
        e = cudaEventCreate(&t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t1);
    Tuning best = b->tune;
    float best_ms = 1e30f;
    // async-copy runner: CTAs per SM x tile size x shared-memory pool limit;
    // bulk-copy runner (one CTA per SM): shared-memory pool limit x the async
    // tile size its smaller global pools use
    // (the bulk-copy runner's shared memory holds pools of up to ~24.5K
    // values across passes; the async runner's, about 8K)
    const int ctas_list[] = {1, 2, 3, 0};
    const int et_list[] = {1280, 1920, TL_EMAX};
    const int64_t fm_list[] = {2048, 4096, 8192, 16384, 24576};
    for (int ci = 0; ci < 4 && e == cudaSuccess; ci++) {
        const bool tma = ctas_list[ci] == 0;
        if (!tma && ctas_list[ci] > b->max_ctas_per_sm)
            continue;
        for (int ei = 0; ei < 3 && e == cudaSuccess; ei++)
            for (int fi = 0; fi < 5 && e == cudaSuccess; fi++) {
                if (!tma && fm_list[fi] > 8192)
                    continue;
                b->tune.runner = tma ? 1 : 0;
                b->tune.ctas_per_sm = tma ? 1 : ctas_list[ci];
                b->tune.etarget = et_list[ei];
                b->tune.fused_max = fm_list[fi];
                e = cudaEventRecord(t0, b->stream);
                if (e == cudaSuccess)
                    e = launch_graph(b, make_args(b, trial_passes, nullptr, 0.f, 1.f));
                if (e == cudaSuccess)
                    e = cudaEventRecord(t1, b->stream);
                if (e == cudaSuccess)
                    e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess)
                    e = cudaEventElapsedTime(&ms, t0, t1);
                if (e == cudaSuccess && ms < best_ms) {
                    best_ms = ms;
                    best = b->tune;
                }
                // back to the snapshot
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b->arena, bk_arena, sizeof(float) * b->arena_floats,
                                        cudaMemcpyDeviceToDevice, b->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b->states, bk_states, sizeof(WlDevState) * (size_t)b->count,
                                        cudaMemcpyDeviceToDevice, b->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b->d_streams, bk_streams, sizeof(BatchStream) * (size_t)b->count,
                                        cudaMemcpyDeviceToDevice, b->stream);
            }
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (t0)
        cudaEventDestroy(t0);
    if (t1)
        cudaEventDestroy(t1);
    cudaFree(bk_arena);
    cudaFree(bk_states);
    cudaFree(bk_streams);
    b->tune = best;
    if (e != cudaSuccess)
        return bfail(b, e);
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f,
                    "{\"key\": \"%s\", \"ctas_per_sm\": %d, \"etarget\": %d, \"fused_max\": %lld, "
                    "\"runner\": %d, \"trial_passes\": %d, \"ms\": %.4f}\n",
                    key.c_str(), best.ctas_per_sm, best.etarget, (long long)best.fused_max,
                    best.runner, trial_passes, best_ms);
            fclose(f);
        }
    }
    return WALLACE_OK;
}

} // extern "C"
