// Serving many clients, each with its own Wallace generator (Brent's RANN4
// paper; independent streams, Section 9), by continuous batching.
//
// Each client's pool stays resident in device memory (one buffer).  A fill
// request (client, count, mu, sigma) waits in a queue until it is admitted:
// the client has no request in flight (a client's stream is sequential) and
// its output buffer -- and, for pools too large for shared memory, a second
// pool buffer -- fit in the device-memory budget.  A scheduler tick turns
// every active request into one work item (first the values left in the
// client's current pool, then up to `passes_per_tick` passes whose returned
// prefixes go straight into the request's output) and launches ONE
// persistent kernel over all items; CTAs take items largest first and run
// them with the per-generator runners of wl_run_body.cuh.  Requests arriving
// while ticks run are admitted at the next tick as slots and memory free up,
// so their work shares launches with requests already in flight.
//
// Ticks are enqueued back to back on the server's stream: the host's view of
// every client (cursor, which buffer holds the pool) is updated when a tick
// is enqueued, which the stream order makes exact.  A tick's event tells when
// its finishing requests are done; memory that a tick still reads is freed
// only after that event.
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

#define SV_THREADS 256

namespace {

struct ServeItem {
    WlRunSpec spec;
    const float *drain_src;   // current pool (before the passes)
    int64_t drain_pos, drain_take;
    float *drain_out;
};

__global__ void __launch_bounds__(SV_THREADS, 3) serve_kernel(const ServeItem *items, int count,
                                                             int *queue, int64_t fused_max)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ uint64_t red[3 * (SV_THREADS / 32)];
    __shared__ int32_t s_prm[20];
    __shared__ int s_k;
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
        if (it.spec.passes > 0)
            wl_run_spec(it.spec, fused_max, smem_values, smem, red, s_prm);
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
    double t_submit = 0, t_done = 0;
};

struct Tick {
    cudaEvent_t ev;
    int slot;
    std::vector<int64_t> finishing;
    std::vector<void *> deferred_free;
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
    cudaStream_t stream = nullptr;
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
    // tick slots: device item arrays and counters
    int nslots = 4;
    std::vector<ServeItem *> d_items;
    std::vector<int> items_cap;
    int *d_queues = nullptr;
    std::vector<bool> slot_busy;
    // tuning
    int passes_per_tick = 4;
    int64_t fused_max = 4096;
    int ctas_per_sm = 3;
    // statistics
    int64_t submitted = 0, admitted = 0, completed = 0, ticks = 0, values = 0;
    std::vector<double> latencies;
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

bool uses_fused(const wallace_server_t *s, const Client &c)
{
    return wl_run_is_fused(s->n, c.N, s->fused_max, (int64_t)(tl_smem_bytes() / sizeof(float)));
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

void reap(wallace_server_t *s, bool block)
{
    while (!s->inflight.empty()) {
        Tick &t = s->inflight.front();
        cudaError_t q = block ? cudaEventSynchronize(t.ev) : cudaEventQuery(t.ev);
        if (q == cudaErrorNotReady)
            return;
        if (q != cudaSuccess) {
            s->status |= WALLACE_ECUDA;
            return;
        }
        const double tn = now_s();
        for (int64_t id : t.finishing) {
            Request &r = s->reqs[id];
            r.reaped = true;
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
        s->inflight.pop_front();
    }
}

// Build and enqueue one tick over every active request.
int enqueue_tick(wallace_server_t *s)
{
    if (s->active.empty())
        return WALLACE_OK;
    int slot = acquire_slot(s);
    if (slot < 0) {
        reap(s, true);
        slot = acquire_slot(s);
        if (slot < 0)
            return WALLACE_OK;
    }
    std::vector<ServeItem> items;
    items.reserve(s->active.size());
    Tick t;
    t.slot = slot;
    std::vector<int64_t> still;
    for (int64_t id : s->active) {
        Request &r = s->reqs[id];
        Client &c = s->clients[r.client];
        ServeItem it;
        memset(&it, 0, sizeof(it));
        float *bufs[2] = {c.buf, r.scratch ? r.scratch : c.buf};
        const int64_t remaining = r.count - r.done;
        int64_t drain = std::min(remaining, c.R - c.cursor);
        if (drain < 0)
            drain = 0;
        it.drain_src = bufs[r.loc];
        it.drain_pos = c.cursor;
        it.drain_take = drain;
        it.drain_out = r.out + r.done;
        c.cursor += drain;
        r.done += drain;
        int64_t left = r.count - r.done;
        int64_t P = (left + c.R - 1) / c.R;
        if (P > s->passes_per_tick)
            P = s->passes_per_tick;
        int64_t last = P > 0 ? std::min(c.R, left - (P - 1) * c.R) : 0;
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
        if (P > 0) {
            r.done += (P - 1) * c.R + last;
            c.cursor = last;
            if (!uses_fused(s, c))
                r.loc ^= (int)(P & 1);
        }
        items.push_back(it);
        if (r.done >= r.count) {
            r.finished = true;
            t.finishing.push_back(id);
            // the pool ends in the scratch buffer: it becomes the resident one
            if (r.scratch) {
                if (r.loc == 1) {
                    t.deferred_free.push_back(c.buf);
                    c.buf = r.scratch;
                } else {
                    t.deferred_free.push_back(r.scratch);
                }
                r.scratch = nullptr;
                r.loc = 0;
            }
            c.active = false;
        } else {
            still.push_back(id);
        }
    }
    s->active.swap(still);
    // largest pools first
    std::sort(items.begin(), items.end(), [](const ServeItem &a, const ServeItem &b) {
        return a.spec.N * (a.spec.passes + 1) > b.spec.N * (b.spec.passes + 1);
    });
    cudaError_t e = cudaSuccess;
    if ((int)items.size() > s->items_cap[slot]) {
        cudaFree(s->d_items[slot]);
        s->d_items[slot] = nullptr;
        int cap = std::max((int)items.size(), 2 * s->items_cap[slot]);
        e = cudaMalloc(&s->d_items[slot], sizeof(ServeItem) * (size_t)cap);
        s->items_cap[slot] = e == cudaSuccess ? cap : 0;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_items[slot], items.data(), sizeof(ServeItem) * items.size(),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->d_queues + slot, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) {
        const int ctas = s->sm_count * std::min(s->ctas_per_sm, s->max_ctas_per_sm);
        const int grid = std::min(ctas, (int)items.size());
        serve_kernel<<<grid, SV_THREADS, tl_smem_bytes(), s->stream>>>(s->d_items[slot], (int)items.size(),
                                                                    s->d_queues + slot, s->fused_max);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventRecord(t.ev, s->stream);
    if (e != cudaSuccess)
        return sfail(s, e);
    s->slot_busy[slot] = true;
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
        e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tl_smem_bytes());
    if (e == cudaSuccess) {
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, serve_kernel, SV_THREADS, tl_smem_bytes());
        s->max_ctas_per_sm = per > 0 ? per : 1;
    }
    if (e == cudaSuccess && cudaMalloc(&s->pool_mem, s->budget - state_bytes) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess && cudaMalloc(&s->states, state_bytes) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess && cudaMalloc(&s->d_queues, sizeof(int) * (size_t)s->nslots) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        wallace_server_destroy(s);
        return e == cudaErrorMemoryAllocation ? WALLACE_ENOMEM : WALLACE_ECUDA;
    }
    s->arena.init(s->pool_mem, s->budget - state_bytes);
    s->d_items.assign(s->nslots, nullptr);
    s->items_cap.assign(s->nslots, 0);
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
            e = wl_launch_init(cl.buf, 0, n, cl.N, cl.Np, seed[c], 0, cl.st, s->sm_count, s->stream);
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
    for (auto &t : s->inflight)
        cudaEventDestroy(t.ev);
    for (auto *p : s->d_items)
        cudaFree(p);
    cudaFree(s->d_queues);
    cudaFree(s->states);
    cudaFree(s->pool_mem);
    delete s;
}

int wallace_server_set_tuning(wallace_server_t *s, int passes_per_tick, int64_t fused_max, int ctas_per_sm)
{
    if (!s || passes_per_tick < 1 || fused_max < 0 || ctas_per_sm < 1 || !s->active.empty() ||
        !s->inflight.empty())
        return WALLACE_EINVAL;
    s->passes_per_tick = passes_per_tick;
    s->fused_max = fused_max;
    s->ctas_per_sm = ctas_per_sm;
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
        int rc = enqueue_tick(s);
        if (rc)
            return rc;
    }
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
    return WALLACE_OK;
}

} // extern "C"
