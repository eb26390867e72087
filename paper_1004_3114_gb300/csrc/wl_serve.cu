// Serving many clients, each with its own Wallace generator (Brent's RANN4
// paper; independent streams, Section 9), by continuous batching.
//
// Each client's pool stays resident in device memory (one buffer).  A fill
// request (client, count, mu, sigma) waits in a queue until it is admitted:
// the client has no request in flight (a client's stream is sequential) and
// its output buffer -- and, for pools too large for shared memory, a second
// pool buffer -- fit in the device-memory budget.  A scheduler tick turns
// every active request into one work item (first the values left in the
// client's current pool, then passes whose returned prefixes go straight into
// the request's output).  Pools of up to a set size (2^22 values by default:
// wallace_server_set_tick) run in one persistent kernel, a CTA per request
// doing many passes in a row (in shared memory when the pool fits -- up to
// 24576 values in the bulk-copy kernel's block -- else from global memory),
// up to a per-tick budget of pool values.  Larger pools run pass-major: each of up to
// `passes_per_tick` launches does one pass of every large request, split
// into units of about 2^17 pool values spread over all CTAs; the last unit
// of a request (by ticket) runs its chi-squared rescale (Eq. 3), so no CTA
// waits for another.  Requests arriving while ticks run are admitted at the
// next tick as slots and memory free up, so their work shares launches with
// requests already in flight.
//
// Each tick slot has its own stream, and a tick takes only the active
// requests that are not in a tick still in flight, so a long item (a pass
// over a large pool) does not hold up the other requests: they go on in the
// next ticks on other streams.  A request is in at most one tick in flight,
// and its client stays busy until that tick's event, so the host's view of
// every client (cursor, which buffer holds the pool) -- updated when a tick is
// enqueued -- is exact.  A tick's event tells when its finishing requests are
// done; memory that a tick still reads is freed only after that event.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "wallace.h"
#include "wl_launch.h"
#include "wl_run_body.cuh"
#include "wl_tma_run.cuh"

#define SV_THREADS 256
#define SV_MAX_PPT 14                /* passes per tick of a large pool (queue counters per slot - 1) */
#define SV_QUEUES_PER_SLOT (SV_MAX_PPT + 2)
// tick slots: ticks in flight at once, a stream each (16 served 1-2% more than
// 8 with p50 7.5 against 8.5 ms on the serving mix; 4 and 32 timed as 8)
#ifndef SV_NSLOTS
#define SV_NSLOTS 16
#endif

namespace {

struct ServeItem {
    WlRunSpec spec;
    const float *drain_src;   // current pool (before the passes)
    int64_t drain_pos, drain_take;
    float *drain_out;
};

template <bool SG>   // the clients draw a sign pattern each pass (matrix A D_k)
__global__ void __launch_bounds__(SV_THREADS, 3) serve_kernel(const ServeItem *items, int count,
                                                             int *queue, int64_t fused_max)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ uint64_t red[3 * (SV_THREADS / 32)];
    __shared__ int s_k;
    __shared__ WlDevState sst;   // the running request's generator state
    const int tid = threadIdx.x;
    const int64_t smem_values = (int64_t)(tl_smem_bytes() / sizeof(float));
    while (true) {
        __syncthreads();
        if (tid == 0)
            s_k = atomicAdd(queue, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= count)
            break;
        const ServeItem it = items[k];
        // values of the current pool not yet handed out
        for (int64_t q = tid; q < it.drain_take; q += blockDim.x) {
            const float y = it.drain_src[wl_phys(it.drain_pos + q, it.spec.N, it.spec.Np)];
            it.drain_out[q] = __fadd_rn(it.spec.mu, __fmul_rn(it.spec.sigma, y));
        }
        if (it.spec.passes > 0) {
            WlRunSpec r = it.spec;
            wl_state_load(&sst, it.spec.st);
            r.st = &sst;
            wl_run_spec<SG>(r, fused_max, smem_values, smem, red);
            wl_state_store(it.spec.st, &sst);
        }
    }
}

// Whether a one-CTA request's pool takes the bulk-copy runner (wl_tma_run.cuh).
__host__ __device__ inline bool sv_bulk_eligible(int n, int64_t N, int64_t passes, int64_t fused_max,
                                                 int64_t smem_values)
{
    return passes > 0 && wl_tma_run_eligible(n, N) && !wl_run_is_fused(n, N, fused_max, smem_values);
}

// The same items with the CTA-local bulk-copy runner: one 608-thread CTA per
// SM, running beside serve_kernel's CTAs on another stream.
template <bool SG>   // the clients draw a sign pattern each pass (matrix A D_k)
__global__ void __launch_bounds__(TM_THREADS, 1) serve_tma_kernel(const ServeItem *items, int count,
                                                                  int *queue, int64_t fused_max)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ uint64_t red[3 * (TM_THREADS / 32 + 1)];
    __shared__ int s_k;
    __shared__ __align__(8) uint64_t bar_full[TR_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[TR_STAGES];
    __shared__ volatile int s_abort;
    __shared__ WlDevState sst;   // the running request's generator state
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
            s_k = atomicAdd(queue, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= count)
            break;
        const ServeItem it = items[k];
        for (int64_t q = tid; q < it.drain_take; q += blockDim.x) {
            const float y = it.drain_src[wl_phys(it.drain_pos + q, it.spec.N, it.spec.Np)];
            it.drain_out[q] = __fadd_rn(it.spec.mu, __fmul_rn(it.spec.sigma, y));
        }
        if (it.spec.passes > 0) {
            WlRunSpec r = it.spec;
            wl_state_load(&sst, it.spec.st);
            r.st = &sst;
            if (sv_bulk_eligible(it.spec.n, it.spec.N, it.spec.passes, fused_max, smem_values))
                wl_run_tma<SG>(r, smem, red, ring);
            else
                wl_run_spec<SG>(r, fused_max, smem_values, smem, red);
            wl_state_store(it.spec.st, &sst);
        }
    }
}

// One pass of one large request.
struct PassItem {
    const float *src;
    float *dst;
    WlDevState *st;
    int64_t N, Np, nu;
    int32_t n, nunits;
    float *out;        // the pass's returned prefix (may be null)
    int64_t w1;        // values of the prefix to write
    float mu, sigma;
    const float *drain_src;   // values of the current pool still to hand out (first pass only)
    int64_t drain_pos, drain_take;
    float *drain_out;
};

struct PassUnit {
    int32_t item;
    int32_t part;      // this unit's share of the pass: part of nunits
};

__device__ __forceinline__ bool last_unit(WlDevState *st, int nunits)
{
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(&st->ticket, 1u) == (unsigned)(nunits - 1);
    __syncthreads();
    if (s_last)
        __threadfence();
    return s_last;
}

__global__ void __launch_bounds__(SV_THREADS, 3) pass_units_kernel(const PassItem *items,
                                                                  const PassUnit *units, int nunits,
                                                                  int *queue)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ uint64_t red[3 * (SV_THREADS / 32)];
    __shared__ int s_k;
    const int tid = threadIdx.x;
    while (true) {
        __syncthreads();
        if (tid == 0)
            s_k = atomicAdd(queue, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= nunits)
            break;
        const PassUnit u = units[k];
        const PassItem it = items[u.item];
        const int64_t N = it.N;
        if (u.part == 0)
            for (int64_t q = tid; q < it.drain_take; q += blockDim.x) {
                const float y = it.drain_src[wl_phys(it.drain_pos + q, N, it.Np)];
                it.drain_out[q] = __fadd_rn(it.mu, __fmul_rn(it.sigma, y));
            }
        uint64_t lo = 0, hi = 0;
        uint32_t bad = 0;
        int32_t alpha[8];
        int64_t gam[8];
        for (int i = 0; i < it.n; i++) {
            alpha[i] = it.st->next.alpha[i];
            gam[i] = it.st->next.gamma[i];
        }
        const float c = it.st->next.c32;
        const int64_t jb = N * u.part / it.nunits, je = N * (u.part + 1) / it.nunits;
        if (it.n == 4) {
            WlTileJob job;
            job.src = it.src;
            job.dst = it.dst;
            job.N = N;
            job.Np = it.Np;
            for (int i = 0; i < 4; i++) {
                job.alpha[i] = alpha[i];
                job.gam[i] = gam[i];
            }
            job.c = c;
            job.signs = it.st->next.signs;
            job.out = it.out;
            job.w0 = 0;
            job.w1 = it.out ? it.w1 : 0;
            job.mu = it.mu;
            job.sigma = it.sigma;
            const int L = wl_lcm4(job.alpha);
            if (wl_tiled_ok(L, N))
                wl_tiled4_tiles(job, L, 0, 1, TL_EMAX, smem, lo, hi, bad, u.part, it.nunits);
            else
                wl_gather4_range(job, jb + tid, blockDim.x, lo, hi, bad, je);
        } else {
            wl_gather_range_n<8>(it.src, it.dst, N, it.Np, alpha, gam, c, it.out, it.out ? it.w1 : 0,
                                 it.mu, it.sigma, lo, hi, bad, jb, je, it.st->next.signs);
        }
        wl_cta_reduce_to_state(lo, hi, bad, it.st, red);
        if (last_unit(it.st, it.nunits) && tid == 0)
            wl_finalise(it.st, it.n, N, it.nu, (double)__ldcg(&it.dst[wl_phys(it.nu - 1, N, it.Np)]),
                        false, WL_FIN_PASS);
    }
}

// Best-fit allocator over one device arena, with coalescing of free blocks.
class Arena {
public:
    static constexpr size_t kAlign = 256;
    void init(char *base, size_t bytes)
    {
        base_ = base;
        size_ = bytes;
        by_off_.clear();
        by_size_.clear();
        insert(0, bytes);
        used_ = peak_ = 0;
    }
    char *alloc(size_t bytes)
    {
        bytes = (bytes + kAlign - 1) / kAlign * kAlign;
        if (bytes == 0)
            bytes = kAlign;
        auto it = by_size_.lower_bound(bytes);
        if (it == by_size_.end())
            return nullptr;
        const size_t sz = it->first, off = it->second;
        erase(off, sz);
        if (sz > bytes)
            insert(off + bytes, sz - bytes);
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        live_[off] = bytes;
        return base_ + off;
    }
    void free(void *p)
    {
        if (!p)
            return;
        size_t off = (size_t)((char *)p - base_);
        auto lv = live_.find(off);
        if (lv == live_.end())
            return;
        size_t sz = lv->second;
        live_.erase(lv);
        used_ -= sz;
        auto next = by_off_.lower_bound(off);
        if (next != by_off_.end() && next->first == off + sz) {
            size_t nsz = next->second;
            erase(next->first, nsz);
            sz += nsz;
        }
        auto prev = by_off_.lower_bound(off);
        if (prev != by_off_.begin()) {
            --prev;
            if (prev->first + prev->second == off) {
                size_t poff = prev->first, psz = prev->second;
                erase(poff, psz);
                off = poff;
                sz += psz;
            }
        }
        insert(off, sz);
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    void insert(size_t off, size_t sz)
    {
        by_off_[off] = sz;
        by_size_.emplace(sz, off);
    }
    void erase(size_t off, size_t sz)
    {
        by_off_.erase(off);
        auto r = by_size_.equal_range(sz);
        for (auto i = r.first; i != r.second; ++i)
            if (i->second == off) {
                by_size_.erase(i);
                break;
            }
    }
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> by_off_;
    std::multimap<size_t, size_t> by_size_;
    std::map<size_t, size_t> live_;
};

struct Client {
    int64_t N, Np, R;
    float *buf;           // resident pool buffer
    WlDevState *st;
    uint32_t seed = 0;
    int64_t passes = 0;         // passes run (host count, exact by the tick order)
    int64_t restarted_at = 0;   // pass count of the last refill (Section 5)
    int64_t cursor;       // next value of the current pool to hand out
    bool active = false;
    std::deque<int64_t> waiting;   // this client's requests not yet admitted, in order
};

struct Request {
    int client;
    int64_t count, done = 0;
    float mu, sigma;
    float *out = nullptr;
    float *scratch = nullptr;   // second pool buffer (global-memory path)
    int loc = 0;                // 0: pool in the client's buffer, 1: in scratch
    bool finished = false, reaped = false, released = false;
    bool busy = false;          // in a tick still in flight
    double t_submit = 0, t_done = 0;
};

struct CopyBack {
    float *dst;
    const float *src;
    size_t bytes;
};

struct Tick {
    cudaEvent_t ev;
    int slot;
    std::vector<int64_t> members;     // requests with work in this tick
    std::vector<int64_t> finishing;
    std::vector<void *> deferred_free;
    std::vector<CopyBack> copies;   // pools that end in a scratch buffer, copied home
};

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

} // namespace

struct wallace_server {
    int n = 4, nclients = 0;
    double frac = 1.0;
    cudaStream_t stream = nullptr;          // creation and the final synchronisation
    std::vector<cudaStream_t> sstream;      // one per tick slot
    std::vector<cudaStream_t> aux;          // per slot: the bulk-copy runner's stream (forked per tick)
    std::vector<cudaEvent_t> ev_fork, ev_join;
    bool bulk = false;                      // one-CTA requests of large enough pools use the bulk-copy runner
    int sm_count = 1, max_ctas_per_sm = 1;
    char *pool_mem = nullptr;
    size_t budget = 0;
    WlDevState *states = nullptr;
    Arena arena;
    std::vector<Client> clients;
    std::vector<Request> reqs;
    std::deque<int> admit_order;   // clients with waiting requests, in arrival order of their head
    std::vector<int64_t> active;
    std::deque<Tick> inflight;
    std::vector<int64_t> completed_unpolled;
    int64_t held_outputs = 0;   // completed requests whose output is not yet released
    // tick slots: device work arrays and work counters
    int nslots = SV_NSLOTS;
    std::vector<char *> d_work;
    std::vector<size_t> work_cap;
    int *d_queues = nullptr;   // kQueuesPerSlot counters per slot
    std::vector<bool> slot_busy;
    // tuning
    int passes_per_tick = 2;          // large pools: passes per request per tick
    int64_t small_values_per_tick = 1 << 20;   // one-CTA pools: pool values per request per tick
    int64_t onchip_max_values = 1 << 22;       // pools up to this run one CTA per request (measured:
                                               // every pool of the serving mix; pass-major above)
    int64_t unit_values = 1 << 17;    // large pools: pool values per CTA work unit
    int64_t fused_max = 4096;
    int ctas_per_sm = 3;
    int opts = 0;           // wl_launch_init options: Wilson-Hilferty sample, sign patterns
    int64_t restart = 0;    // refill a client's pool before the pass after each multiple of this
    // statistics
    int64_t submitted = 0, admitted = 0, completed = 0, ticks = 0, values = 0;
    std::vector<double> latencies;
    double host_tick_s = 0, host_wait_s = 0, admit_wait_s = 0;
    int64_t items = 0;
    double t_first = -1, t_last = 0;
    int status = 0;
};

namespace {

int sfail(wallace_server_t *s, cudaError_t e)
{
    if (e == cudaSuccess)
        return WALLACE_OK;
    if (s)
        s->status |= WALLACE_ECUDA;
    return WALLACE_ECUDA;
}

// Shared-memory capacity (floats) of the kernel that runs a one-CTA item:
// with the bulk-copy runner on, pools that fit its larger block but not the
// 256-thread kernel's stay in shared memory there too.
int64_t small_smem_values() { return (int64_t)(tl_smem_bytes() / sizeof(float)); }
int64_t big_smem_values() { return (int64_t)(wl_tma::tr_smem_bytes() / sizeof(float)); }

bool uses_fused(const wallace_server_t *s, const Client &c)
{
    return wl_run_is_fused(s->n, c.N, s->fused_max, s->bulk ? big_smem_values() : small_smem_values());
}

size_t pool_bytes(const wallace_server_t *s, const Client &c)
{
    return sizeof(float) * (size_t)s->n * (size_t)c.Np;
}

// Admit waiting requests whose memory fits.  A client is in admit_order
// exactly when it has waiting requests; its requests are admitted one at a
// time and in order.
void admit(wallace_server_t *s)
{
    const size_t n = s->admit_order.size();
    for (size_t k = 0; k < n; k++) {
        const int ci = s->admit_order.front();
        s->admit_order.pop_front();
        Client &c = s->clients[ci];
        if (c.waiting.empty())
            continue;
        if (c.active) {
            s->admit_order.push_back(ci);
            continue;
        }
        Request &r = s->reqs[c.waiting.front()];
        float *out = r.count > 0 ? (float *)s->arena.alloc(sizeof(float) * (size_t)r.count) : nullptr;
        float *scr = nullptr;
        bool ok = r.count == 0 || out != nullptr;
        if (ok && r.count > 0 && !uses_fused(s, c)) {
            scr = (float *)s->arena.alloc(pool_bytes(s, c));
            ok = scr != nullptr;
        }
        if (!ok) {
            s->arena.free(out);
            s->admit_order.push_back(ci);   // retry once memory is freed
            continue;
        }
        r.out = out;
        r.scratch = scr;
        r.loc = 0;
        s->admit_wait_s += now_s() - r.t_submit;
        c.active = true;
        s->active.push_back(c.waiting.front());
        c.waiting.pop_front();
        s->admitted++;
        if (!c.waiting.empty())
            s->admit_order.push_back(ci);
    }
}

int acquire_slot(wallace_server_t *s)
{
    for (int k = 0; k < s->nslots; k++)
        if (!s->slot_busy[k])
            return k;
    return -1;
}

// Finish the ticks whose events have completed (in any order: each slot has
// its own stream); with `block`, wait for the oldest first when none has.
void reap(wallace_server_t *s, bool block)
{
    bool done_any = false;
    for (size_t k = 0; k < s->inflight.size();) {
        Tick &t = s->inflight[k];
        cudaError_t q = cudaEventQuery(t.ev);
        if (q == cudaErrorNotReady && block && !done_any && k == 0) {
            const double w0 = now_s();
            q = cudaEventSynchronize(t.ev);
            s->host_wait_s += now_s() - w0;
        }
        if (q == cudaErrorNotReady) {
            k++;
            continue;
        }
        if (q != cudaSuccess) {
            s->status |= WALLACE_ECUDA;
            return;
        }
        done_any = true;
        const double tn = now_s();
        for (int64_t id : t.members)
            s->reqs[id].busy = false;
        for (int64_t id : t.finishing) {
            Request &r = s->reqs[id];
            r.reaped = true;
            s->clients[r.client].active = false;   // its pool is settled: the next request may start
            if (r.out)
                s->held_outputs++;
            r.t_done = tn;
            s->latencies.push_back(1e3 * (tn - r.t_submit));
            s->completed++;
            s->values += r.count;
            s->t_last = tn;
            s->completed_unpolled.push_back(id);
        }
        for (void *p : t.deferred_free)
            s->arena.free(p);
        s->slot_busy[t.slot] = false;
        cudaEventDestroy(t.ev);
        s->inflight.erase(s->inflight.begin() + (std::ptrdiff_t)k);
    }
}

// Build and enqueue one tick over every active request: one on-chip kernel
// for the shared-memory pools, then one pass-major launch per pass for the
// large pools.
int enqueue_tick_impl(wallace_server_t *s);

int enqueue_tick(wallace_server_t *s)
{
    const double t0 = now_s();
    const int rc = enqueue_tick_impl(s);
    s->host_tick_s += now_s() - t0;
    return rc;
}

int enqueue_tick_impl(wallace_server_t *s)
{
    // the active requests not in a tick still in flight
    bool any = false;
    for (int64_t id : s->active)
        if (!s->reqs[id].busy) {
            any = true;
            break;
        }
    if (!any)
        return WALLACE_OK;
    int slot = acquire_slot(s);
    if (slot < 0) {
        reap(s, true);
        slot = acquire_slot(s);
        if (slot < 0)
            return WALLACE_OK;
    }
    std::vector<ServeItem> small;
    std::vector<std::vector<PassItem>> pitems(s->passes_per_tick);
    std::vector<std::vector<PassUnit>> punits(s->passes_per_tick);
    Tick t;
    t.slot = slot;
    std::vector<int64_t> still;
    struct Refill {
        float *pool;
        int64_t N, Np;
        uint32_t seed;
        int64_t r;
        WlDevState *st;
    };
    std::vector<Refill> refills;   // pools refilled on this tick's stream before its kernels
    for (int64_t id : s->active) {
        Request &r = s->reqs[id];
        if (r.busy) {
            still.push_back(id);   // its previous tick has not finished
            continue;
        }
        r.busy = true;
        t.members.push_back(id);
        Client &c = s->clients[r.client];
        float *bufs[2] = {c.buf, r.scratch ? r.scratch : c.buf};
        const int64_t nu = (int64_t)s->n * c.N;
        const bool fused = uses_fused(s, c);
        const bool one_cta = nu <= s->onchip_max_values;   // whole request on one CTA per tick
        const int64_t remaining = r.count - r.done;
        int64_t drain = std::max<int64_t>(0, std::min(remaining, c.R - c.cursor));
        const float *drain_src = bufs[r.loc];
        const int64_t drain_pos = c.cursor;
        float *drain_out = r.out + r.done;
        c.cursor += drain;
        r.done += drain;
        const int64_t left = r.count - r.done;
        int64_t P = (left + c.R - 1) / c.R;
        const int64_t cap = one_cta ? std::max<int64_t>(1, s->small_values_per_tick / nu) : s->passes_per_tick;
        if (P > cap)
            P = cap;
        if (s->restart > 0 && P > 0) {
            // Section 5: refill before the pass that follows a multiple of the
            // interval; values of the current pool still owed go out first
            // (a drain-only item this tick), and no item crosses a restart point
            const int64_t K = s->restart;
            if (c.passes > 0 && c.passes % K == 0 && c.restarted_at != c.passes) {
                if (drain > 0) {
                    P = 0;
                } else {
                    refills.push_back(Refill{bufs[r.loc], c.N, c.Np, c.seed, c.passes / K, c.st});
                    c.restarted_at = c.passes;
                }
            }
            P = std::min(P, K - c.passes % K);
        }
        c.passes += P;
        const int64_t last = P > 0 ? std::min(c.R, left - (P - 1) * c.R) : 0;
        if (one_cta || P == 0) {
            ServeItem it;
            memset(&it, 0, sizeof(it));
            it.drain_src = drain_src;
            it.drain_pos = drain_pos;
            it.drain_take = drain;
            it.drain_out = drain_out;
            WlRunSpec &sp = it.spec;
            sp.buf[0] = bufs[0];
            sp.buf[1] = bufs[1];
            sp.cur = r.loc;
            sp.st = c.st;
            sp.N = c.N;
            sp.Np = c.Np;
            sp.R = c.R;
            sp.n = s->n;
            sp.passes = P;
            sp.out = r.out + r.done;
            sp.last_take = last;
            sp.mu = r.mu;
            sp.sigma = r.sigma;
            sp.etarget = TL_EMAX;
            small.push_back(it);
            if (P > 0) {
                r.done += (P - 1) * c.R + last;
                c.cursor = last;
                if (!fused)
                    r.loc ^= (int)(P & 1);   // global-memory passes alternate the two buffers
            }
        } else {
            const int units = (int)std::max<int64_t>(1, (nu + s->unit_values - 1) / s->unit_values);
            for (int64_t p = 0; p < P; p++) {
                PassItem pi;
                memset(&pi, 0, sizeof(pi));
                pi.src = bufs[r.loc ^ (int)(p & 1)];
                pi.dst = bufs[r.loc ^ (int)((p + 1) & 1)];
                pi.st = c.st;
                pi.N = c.N;
                pi.Np = c.Np;
                pi.nu = nu;
                pi.n = s->n;
                pi.nunits = units;
                const int64_t take = p + 1 < P ? c.R : last;
                pi.out = r.out + r.done;
                pi.w1 = take;
                pi.mu = r.mu;
                pi.sigma = r.sigma;
                if (p == 0) {
                    pi.drain_src = drain_src;
                    pi.drain_pos = drain_pos;
                    pi.drain_take = drain;
                    pi.drain_out = drain_out;
                }
                r.done += take;
                const int idx = (int)pitems[p].size();
                pitems[p].push_back(pi);
                for (int u = 0; u < units; u++)
                    punits[p].push_back(PassUnit{idx, u});
            }
            c.cursor = last;
            r.loc ^= (int)(P & 1);
        }
        if (r.done >= r.count) {
            r.finished = true;
            t.finishing.push_back(id);
            // Client pools never move: a pool that ends in the scratch buffer
            // is copied back to its home after this tick.  (Adopting the
            // scratch buffer as the new home would scatter pools through the
            // arena until no free block fits a request, with nothing in flight
            // to free one.)
            if (r.scratch) {
                if (r.loc == 1)
                    t.copies.push_back(CopyBack{c.buf, r.scratch, pool_bytes(s, c)});
                t.deferred_free.push_back(r.scratch);
                r.scratch = nullptr;
                r.loc = 0;
            }
            // the client stays busy until this tick completes (see reap)
        } else {
            still.push_back(id);
        }
    }
    s->active.swap(still);
    // largest work first; with the bulk-copy runner on, its items go last
    std::sort(small.begin(), small.end(), [](const ServeItem &a, const ServeItem &b) {
        return a.spec.N * (a.spec.passes + 1) > b.spec.N * (b.spec.passes + 1);
    });
    int nrest = (int)small.size();
    if (s->bulk) {
        const int64_t tma_values = (int64_t)(wl_tma::tr_smem_bytes() / sizeof(float));
        auto mid = std::stable_partition(small.begin(), small.end(), [&](const ServeItem &it) {
            const int64_t nu = (int64_t)it.spec.n * it.spec.N;
            const bool big_fused = it.spec.passes > 0 && wl_run_is_fused(it.spec.n, it.spec.N, s->fused_max, tma_values) &&
                                   2 * nu > small_smem_values();
            return !(sv_bulk_eligible(it.spec.n, it.spec.N, it.spec.passes, s->fused_max, tma_values) || big_fused);
        });
        nrest = (int)(mid - small.begin());
    }
    // one device buffer per slot: [small items][pass items...][pass units...]
    size_t bytes = sizeof(ServeItem) * small.size();
    std::vector<size_t> off_items(s->passes_per_tick), off_units(s->passes_per_tick);
    for (int p = 0; p < s->passes_per_tick; p++) {
        bytes = (bytes + 15) & ~(size_t)15;
        off_items[p] = bytes;
        bytes += sizeof(PassItem) * pitems[p].size();
    }
    for (int p = 0; p < s->passes_per_tick; p++) {
        bytes = (bytes + 15) & ~(size_t)15;
        off_units[p] = bytes;
        bytes += sizeof(PassUnit) * punits[p].size();
    }
    cudaError_t e = cudaSuccess;
    if (bytes > s->work_cap[slot]) {
        cudaFree(s->d_work[slot]);
        s->d_work[slot] = nullptr;
        size_t cap = std::max(bytes, 2 * s->work_cap[slot]);
        e = cudaMalloc(&s->d_work[slot], cap);
        s->work_cap[slot] = e == cudaSuccess ? cap : 0;
    }
    std::vector<char> host(bytes);
    if (!small.empty())
        memcpy(host.data(), small.data(), sizeof(ServeItem) * small.size());
    for (int p = 0; p < s->passes_per_tick; p++) {
        if (!pitems[p].empty())
            memcpy(host.data() + off_items[p], pitems[p].data(), sizeof(PassItem) * pitems[p].size());
        if (!punits[p].empty())
            memcpy(host.data() + off_units[p], punits[p].data(), sizeof(PassUnit) * punits[p].size());
    }
    char *dw = s->d_work[slot];
    int *dq = s->d_queues + slot * SV_QUEUES_PER_SLOT;
    cudaStream_t st = s->sstream[slot], aux = s->aux[slot];
    cudaEvent_t ev_fork = s->ev_fork[slot], ev_join = s->ev_join[slot];
    if (e == cudaSuccess && bytes)
        e = cudaMemcpyAsync(dw, host.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dq, 0, sizeof(int) * SV_QUEUES_PER_SLOT, st);
    for (size_t k = 0; k < refills.size() && e == cudaSuccess; k++)
        e = wl_launch_restart(refills[k].pool, 0, s->n, refills[k].N, refills[k].Np, refills[k].seed, 0,
                              refills[k].r, refills[k].st, s->sm_count, st);
    const int ctas = s->sm_count * std::min(s->ctas_per_sm, s->max_ctas_per_sm);
    // bulk-copy items (placed after the others) run on the aux stream, beside the rest
    const int nbulk = (int)small.size() - nrest;
    if (e == cudaSuccess && nbulk > 0) {
        e = cudaEventRecord(ev_fork, st);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(aux, ev_fork, 0);
        if (e == cudaSuccess) {
            auto kern = (s->opts & 2) ? serve_tma_kernel<true> : serve_tma_kernel<false>;
            kern<<<std::min(s->sm_count, nbulk), TM_THREADS, wl_tma::tr_smem_bytes(), aux>>>(
                (const ServeItem *)dw + nrest, nbulk, dq + SV_MAX_PPT + 1, s->fused_max);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_join, aux);
    }
    if (e == cudaSuccess && nrest > 0) {
        const int grid = std::min(ctas, nrest);
        auto skern = (s->opts & 2) ? serve_kernel<true> : serve_kernel<false>;
        skern<<<grid, SV_THREADS, tl_smem_bytes(), st>>>((const ServeItem *)dw, nrest, dq, s->fused_max);
        e = cudaGetLastError();
    }
    for (int p = 0; p < s->passes_per_tick && e == cudaSuccess; p++) {
        if (punits[p].empty())
            continue;
        const int grid = std::min(ctas, (int)punits[p].size());
        pass_units_kernel<<<grid, SV_THREADS, tl_smem_bytes(), st>>>(
            (const PassItem *)(dw + off_items[p]), (const PassUnit *)(dw + off_units[p]),
            (int)punits[p].size(), dq + 1 + p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && nbulk > 0)
        e = cudaStreamWaitEvent(st, ev_join, 0);
    for (size_t k = 0; k < t.copies.size() && e == cudaSuccess; k++)
        e = cudaMemcpyAsync(t.copies[k].dst, t.copies[k].src, t.copies[k].bytes, cudaMemcpyDeviceToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventRecord(t.ev, st);
    if (e != cudaSuccess)
        return sfail(s, e);
    s->slot_busy[slot] = true;
    s->items += (int64_t)t.members.size();
    s->inflight.push_back(std::move(t));
    s->ticks++;
    return WALLACE_OK;
}

void percentile(std::vector<double> v, double *p50, double *p99, double *mean)
{
    if (v.empty()) {
        *p50 = *p99 = *mean = 0;
        return;
    }
    std::sort(v.begin(), v.end());
    auto at = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
    *p50 = at(0.50);
    *p99 = at(0.99);
    double s = 0;
    for (double x : v)
        s += x;
    *mean = s / (double)v.size();
}

} // namespace

extern "C" {

int wallace_server_create(int n_clients, int n, const int64_t *N, const uint32_t *seed, double frac,
                          int64_t hbm_budget_bytes, void *cuda_stream, wallace_server_t **out)
{
    return wallace_server_create_ex(n_clients, n, N, seed, frac, WALLACE_FP32, hbm_budget_bytes, cuda_stream,
                                    out);
}

int wallace_server_create_ex(int n_clients, int n, const int64_t *N, const uint32_t *seed, double frac,
                             int mode, int64_t hbm_budget_bytes, void *cuda_stream, wallace_server_t **out)
{
    if ((mode & ~(WALLACE_CHI_WH | WALLACE_MATRIX_SIGNS)) != WALLACE_FP32)
        return WALLACE_EINVAL;
    if (!out || n_clients < 1 || !N || !seed || (n != 4 && n != 8) || !(frac > 0.0 && frac <= 1.0) ||
        hbm_budget_bytes <= 0)
        return WALLACE_EINVAL;
    *out = nullptr;
    wallace_server_t *s = new (std::nothrow) wallace_server;
    if (!s)
        return WALLACE_ENOMEM;
    s->n = n;
    s->nclients = n_clients;
    s->frac = frac;
    s->opts = ((mode & WALLACE_CHI_WH) ? 1 : 0) | ((mode & WALLACE_MATRIX_SIGNS) ? 2 : 0);
    s->stream = (cudaStream_t)cuda_stream;
    s->budget = (size_t)hbm_budget_bytes;
    s->clients.resize(n_clients);
    size_t resident = 0;
    for (int c = 0; c < n_clients; c++) {
        Client &cl = s->clients[c];
        const int64_t nu = (int64_t)n * N[c];
        if (N[c] < 4 || nu > ((int64_t)1 << 30)) {
            delete s;
            return WALLACE_EINVAL;
        }
        int64_t R = (int64_t)(frac * (double)nu);
        if (R > nu - 1)
            R = nu - 1;
        if (R < 1) {
            delete s;
            return WALLACE_EINVAL;
        }
        cl.N = N[c];
        cl.seed = seed[c];
        cl.Np = ((N[c] + 8 + 63) / 64) * 64;
        cl.R = R;
        cl.cursor = R;   // the initial pool is not returned
        resident += (pool_bytes(s, cl) + Arena::kAlign - 1) / Arena::kAlign * Arena::kAlign;
    }
    const size_t state_bytes = sizeof(WlDevState) * (size_t)n_clients;
    if (resident + state_bytes >= s->budget) {
        delete s;
        return WALLACE_ENOMEM;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tl_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tl_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pass_units_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tl_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_tma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wl_tma::tr_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_tma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wl_tma::tr_smem_bytes());
    s->sstream.assign(s->nslots, nullptr);
    s->aux.assign(s->nslots, nullptr);
    s->ev_fork.assign(s->nslots, nullptr);
    s->ev_join.assign(s->nslots, nullptr);
    for (int k = 0; k < s->nslots && e == cudaSuccess; k++) {
        e = cudaStreamCreateWithFlags(&s->sstream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&s->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s->ev_fork[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, serve_kernel<true>, SV_THREADS, tl_smem_bytes());
        s->max_ctas_per_sm = per > 0 ? per : 1;
    }
    if (e == cudaSuccess && cudaMalloc(&s->pool_mem, s->budget - state_bytes) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess && cudaMalloc(&s->states, state_bytes) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess &&
        cudaMalloc(&s->d_queues, sizeof(int) * (size_t)(s->nslots * SV_QUEUES_PER_SLOT)) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        wallace_server_destroy(s);
        return e == cudaErrorMemoryAllocation ? WALLACE_ENOMEM : WALLACE_ECUDA;
    }
    s->arena.init(s->pool_mem, s->budget - state_bytes);
    s->d_work.assign(s->nslots, nullptr);
    s->work_cap.assign(s->nslots, 0);
    s->slot_busy.assign(s->nslots, false);
    e = cudaMemsetAsync(s->states, 0, state_bytes, s->stream);
    for (int c = 0; c < n_clients && e == cudaSuccess; c++) {
        Client &cl = s->clients[c];
        cl.buf = (float *)s->arena.alloc(pool_bytes(s, cl));
        cl.st = s->states + c;
        if (!cl.buf) {
            e = cudaErrorMemoryAllocation;
            break;
        }
        e = cudaMemsetAsync(cl.buf, 0, pool_bytes(s, cl), s->stream);
        if (e == cudaSuccess)
            e = wl_launch_init(cl.buf, 0, n, cl.N, cl.Np, seed[c], 0, cl.st, s->sm_count, s->stream, s->opts);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        wallace_server_destroy(s);
        return e == cudaErrorMemoryAllocation ? WALLACE_ENOMEM : WALLACE_ECUDA;
    }
    *out = s;
    return WALLACE_OK;
}

void wallace_server_destroy(wallace_server_t *s)
{
    if (!s)
        return;
    cudaStreamSynchronize(s->stream);
    for (size_t k = 0; k < s->sstream.size(); k++) {
        if (s->sstream[k]) {
            cudaStreamSynchronize(s->sstream[k]);
            cudaStreamDestroy(s->sstream[k]);
        }
        if (s->aux[k]) {
            cudaStreamSynchronize(s->aux[k]);
            cudaStreamDestroy(s->aux[k]);
        }
        if (s->ev_fork[k])
            cudaEventDestroy(s->ev_fork[k]);
        if (s->ev_join[k])
            cudaEventDestroy(s->ev_join[k]);
    }
    for (auto &t : s->inflight)
        cudaEventDestroy(t.ev);
    for (auto *p : s->d_work)
        cudaFree(p);
    cudaFree(s->d_queues);
    cudaFree(s->states);
    cudaFree(s->pool_mem);
    delete s;
}

int wallace_server_set_tuning(wallace_server_t *s, int passes_per_tick, int64_t fused_max, int ctas_per_sm)
{
    if (!s || passes_per_tick < 1 || passes_per_tick > SV_MAX_PPT || fused_max < 0 || ctas_per_sm < 0 ||
        !s->active.empty() || !s->inflight.empty())
        return WALLACE_EINVAL;
    s->passes_per_tick = passes_per_tick;
    s->fused_max = fused_max;
    s->bulk = ctas_per_sm == 0;
    s->ctas_per_sm = ctas_per_sm == 0 ? 3 : ctas_per_sm;
    return WALLACE_OK;
}

int wallace_server_set_restart(wallace_server_t *s, int64_t interval)
{
    if (!s || interval < 0 || !s->active.empty() || !s->inflight.empty())
        return WALLACE_EINVAL;
    s->restart = interval;
    return WALLACE_OK;
}

int wallace_server_set_tick(wallace_server_t *s, int64_t one_cta_max_values, int64_t values_per_tick)
{
    if (!s || one_cta_max_values < 0 || values_per_tick < 1 || !s->active.empty() || !s->inflight.empty())
        return WALLACE_EINVAL;
    s->onchip_max_values = one_cta_max_values;
    s->small_values_per_tick = values_per_tick;
    return WALLACE_OK;
}

int wallace_server_submit(wallace_server_t *s, int client, int64_t count, float mu, float sigma,
                          int64_t *request_id)
{
    if (!s || client < 0 || client >= s->nclients || count < 0)
        return WALLACE_EINVAL;
    Request r;
    r.client = client;
    r.count = count;
    r.mu = mu;
    r.sigma = sigma;
    r.t_submit = now_s();
    if (s->t_first < 0)
        s->t_first = r.t_submit;
    const int64_t id = (int64_t)s->reqs.size();
    s->reqs.push_back(r);
    Client &c = s->clients[client];
    if (c.waiting.empty())
        s->admit_order.push_back(client);
    c.waiting.push_back(id);
    s->submitted++;
    if (request_id)
        *request_id = id;
    return WALLACE_OK;
}

int wallace_server_progress(wallace_server_t *s)
{
    if (!s)
        return WALLACE_EINVAL;
    reap(s, false);
    admit(s);
    int rc = enqueue_tick(s);
    reap(s, false);
    // Requests wait, none runs, nothing in flight and every output released:
    // no later call can free memory, so the head request can never fit.
    if (!rc && s->active.empty() && s->inflight.empty() && !s->admit_order.empty() &&
        s->held_outputs == 0)
        s->status |= WALLACE_ENOMEM;
    return rc ? rc : s->status;
}

int wallace_server_drain(wallace_server_t *s)
{
    if (!s)
        return WALLACE_EINVAL;
    while (true) {
        reap(s, false);
        admit(s);
        if (s->active.empty() && s->admit_order.empty())
            break;
        if (s->active.empty()) {
            // nothing fits until in-flight work frees memory
            if (s->inflight.empty()) {
                s->status |= WALLACE_ENOMEM;   // a request larger than the whole arena
                break;
            }
            reap(s, true);
            continue;
        }
        const int64_t before = s->ticks;
        int rc = enqueue_tick(s);
        if (rc)
            return rc;
        if (s->ticks == before)
            reap(s, true);   // every active request is in a tick in flight
    }
    while (!s->inflight.empty() && !(s->status & WALLACE_ECUDA))
        reap(s, true);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? s->status : sfail(s, e);
}

int wallace_server_poll(wallace_server_t *s, int64_t *ids, int max_ids, int *n_out)
{
    if (!s || !n_out || (max_ids > 0 && !ids))
        return WALLACE_EINVAL;
    reap(s, false);
    int k = 0;
    while (k < max_ids && !s->completed_unpolled.empty()) {
        ids[k++] = s->completed_unpolled.front();
        s->completed_unpolled.erase(s->completed_unpolled.begin());
    }
    *n_out = k;
    return s->status;
}

int wallace_server_result(wallace_server_t *s, int64_t id, float **dev_out, int64_t *count,
                          double *latency_ms)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size())
        return WALLACE_EINVAL;
    const Request &r = s->reqs[id];
    if (!r.reaped)
        return WALLACE_ESTATE;
    if (dev_out)
        *dev_out = r.released ? nullptr : r.out;
    if (count)
        *count = r.count;
    if (latency_ms)
        *latency_ms = 1e3 * (r.t_done - r.t_submit);
    return WALLACE_OK;
}

int wallace_server_release(wallace_server_t *s, int64_t id)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size())
        return WALLACE_EINVAL;
    Request &r = s->reqs[id];
    if (!r.reaped)
        return WALLACE_ESTATE;
    if (!r.released) {
        if (r.out)
            s->held_outputs--;
        s->arena.free(r.out);
        r.out = nullptr;
        r.released = true;
    }
    return WALLACE_OK;
}

int wallace_server_run_trace(wallace_server_t *s, int64_t n, const double *arrival_s,
                             const int32_t *client, const int64_t *count, const float *mu,
                             const float *sigma, double *latency_ms)
{
    if (!s || n < 0 || (n > 0 && (!arrival_s || !client || !count || !mu || !sigma)))
        return WALLACE_EINVAL;
    const int64_t id0 = (int64_t)s->reqs.size();
    const double t0 = now_s();
    int64_t next = 0;
    std::vector<int64_t> ids;
    while (true) {
        const double t = now_s() - t0;
        while (next < n && arrival_s[next] <= t) {
            int64_t id;
            int rc = wallace_server_submit(s, client[next], count[next], mu[next], sigma[next], &id);
            if (rc)
                return rc;
            s->reqs[id].t_submit = t0 + arrival_s[next];   // latency from the scheduled arrival
            next++;
        }
        reap(s, false);
        // outputs are not kept: free them as soon as their request is done
        for (int64_t id : s->completed_unpolled)
            if (id >= id0)
                wallace_server_release(s, id);
        s->completed_unpolled.clear();
        admit(s);
        if (!s->active.empty()) {
            int rc = enqueue_tick(s);
            if (rc)
                return rc;
        } else if (!s->admit_order.empty()) {
            if (s->inflight.empty()) {
                // nothing in flight will free memory: a request larger than the arena
                s->status |= WALLACE_ENOMEM;
                break;
            }
            reap(s, true);   // wait for memory held by in-flight work
        } else if (next >= n) {
            if (s->inflight.empty())
                break;
            reap(s, true);
        }
        if ((int)s->inflight.size() >= s->nslots)
            reap(s, true);
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess)
        return sfail(s, e);
    if (latency_ms)
        for (int64_t k = 0; k < n; k++) {
            const Request &r = s->reqs[id0 + k];
            latency_ms[k] = 1e3 * (r.t_done - r.t_submit);
        }
    return s->status;
}

int wallace_server_stats(wallace_server_t *s, wallace_server_stats_t *out)
{
    if (!s || !out)
        return WALLACE_EINVAL;
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->active = (int64_t)s->active.size();
    int64_t queued = 0;
    for (auto &c : s->clients)
        queued += (int64_t)c.waiting.size();
    out->queued = queued;
    out->ticks = s->ticks;
    out->values_delivered = s->values;
    out->hbm_budget = (int64_t)s->budget;
    out->hbm_in_use = (int64_t)(s->arena.used() + sizeof(WlDevState) * (size_t)s->nclients);
    out->hbm_peak = (int64_t)(s->arena.peak() + sizeof(WlDevState) * (size_t)s->nclients);
    percentile(s->latencies, &out->p50_ms, &out->p99_ms, &out->mean_ms);
    out->elapsed_s = s->t_first >= 0 ? s->t_last - s->t_first : 0.0;
    out->status = s->status;
    out->host_tick_s = s->host_tick_s;
    out->host_wait_s = s->host_wait_s;
    out->items = s->items;
    out->mean_admit_wait_ms = s->admitted ? 1e3 * s->admit_wait_s / (double)s->admitted : 0.0;
    return WALLACE_OK;
}

} // extern "C"
