// Serving: a persistent request loop with continuous batching of mixed solves
// (declared in include/stencilfft.h).
//
// A worker thread owns the GPU side. Requests (any dimension, size, T,
// boundary, radius, weights) are queued by stencil_server_submit and admitted
// in arrival order whenever a slot (a non-blocking CUDA stream) is free and
// the device memory the request's plan needs fits the budget. Plans --
// twiddles, symbol tables, workspaces -- stay on the device in a pool keyed by
// shape and are handed to one in-flight request at a time; a request only sets
// its weights on the plan it gets. Requests admitted while others run overlap
// on the device through their slots' streams.
//
// Small periodic requests that one CTA can solve in shared memory are batched
// across shapes: every queued such request of the head's precision (up to
// kListCap) goes into one run of a batch executor (stencil_batch_*), one
// persistent launch over a device work list in which each CTA solves whole
// requests. Larger small periodic requests of one shape are stacked: up to
// kMaxItems queued requests share one buffer and one launch per pass, each
// with its own Lambda^T / N table (built from its weights and T).
//
// Latency is measured from submit to the worker observing the request's
// completion event.
//
// Locking: the mutex guards the queue, the results and the statistics. The
// plan pool and the slots belong to the worker thread alone, so plan creation
// and eviction run with the mutex released: a submit never waits for them. An
// evicted plan is idle -- the completion event of its last launch has been
// observed -- and is freed without a device-wide synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/stencilfft.h"
#include "internal.h"
#include "plan_impl.h"

using namespace sfft;

namespace {

constexpr int64_t kBatchMaxCells = 1 << 16;   // periodic requests at most this big are batched
constexpr int kListCap = 256;                  // requests per run of the batch executor

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Key {
    int ndim, radius, boundary, precision, batch;
    int64_t dims[3];
    bool operator==(const Key& o) const {
        return ndim == o.ndim && radius == o.radius && boundary == o.boundary &&
               precision == o.precision && batch == o.batch && dims[0] == o.dims[0] &&
               dims[1] == o.dims[1] && dims[2] == o.dims[2];
    }
};

struct Pending {
    uint64_t ticket;
    stencil_request r;
    std::vector<double> w;
    double t_submit;
};

struct PlanEntry {
    Key key;
    stencil_plan_s* plan = nullptr;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
    // batch plans: stacked grids, stacked half spectra and per-item tables
    void* stackS = nullptr;
    void* stackH = nullptr;
    void* vt[kMaxItems] = {};
    size_t cells = 0, h_item = 0, v_item = 0;
    stencil_batch_t exec = nullptr;   // batch key 2: the mixed-shape executor
    cudaEvent_t last = nullptr;   // recorded after the plan's latest launch
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Pending> reqs;
    PlanEntry* pe = nullptr;
    int status = STENCIL_OK;
    int batched = 0;   // requests of the last launch, when it was a batch
};

int validate_request(const stencil_request* r) {
    if (!r || !r->weights || !r->grid || r->T < 0 || r->ndim < 1 || r->ndim > 3 ||
        r->radius < 0 || r->radius > kMaxRadius)
        return STENCIL_EINVAL;
    if (r->boundary != STENCIL_PERIODIC && r->boundary != STENCIL_ZERO_DIRICHLET)
        return STENCIL_EINVAL;
    if (r->precision != STENCIL_FP32 && r->precision != STENCIL_FP64) return STENCIL_EINVAL;
    if (reinterpret_cast<uintptr_t>(r->grid) % 16) return STENCIL_EINVAL;
    for (int a = 0; a < r->ndim; ++a) {
        if (r->dims[a] < 2 * r->radius + 1 || r->dims[a] < 4) return STENCIL_EINVAL;
        if (ilog2_exact(r->dims[a]) < 0 || r->dims[a] > max_axis(r->ndim, r->precision, a))
            return STENCIL_EUNSUPPORTED;
    }
    return STENCIL_OK;
}

int64_t cells_of(const stencil_request& r) {
    int64_t n = 1;
    for (int a = 0; a < r.ndim; ++a) n *= r.dims[a];
    return n;
}

bool batchable(const stencil_request& r) {
    // the batched path needs the register kernels (last axis >= 32) and
    // per-item tables; a 1-D row must fit one CTA (longer rows take the
    // n1 x n2 passes, which evaluate their multiplier per element)
    const int64_t one_cta = 2 * 16 * (r.precision == STENCIL_FP32 ? kMaxThreadsF32 : kMaxThreadsF64);
    return r.boundary == STENCIL_PERIODIC && cells_of(r) <= kBatchMaxCells &&
           r.dims[r.ndim - 1] >= 32 && (r.ndim != 1 || r.dims[0] <= one_cta);
}

// Solved whole by one CTA of the batch executor, whatever its shape.
bool list_batchable(const stencil_request& r) {
    return r.boundary == STENCIL_PERIODIC && stencil_batch_smem_bytes(r.ndim, r.dims, r.precision) > 0;
}

Key list_key(int precision) {
    Key k;
    std::memset(&k, 0, sizeof(k));
    k.precision = precision;
    k.boundary = STENCIL_PERIODIC;
    k.batch = 2;
    k.radius = -1;
    return k;
}

Key key_of(const stencil_request& r, bool batch) {
    Key k;
    std::memset(&k, 0, sizeof(k));
    k.ndim = r.ndim;
    k.radius = batch ? -1 : r.radius;
    k.boundary = r.boundary;
    k.precision = r.precision;
    k.batch = batch ? 1 : 0;
    for (int a = 0; a < 3; ++a) k.dims[a] = a < r.ndim ? r.dims[a] : 1;
    return k;
}

size_t estimate_bytes(const Key& k) {
    if (k.batch == 2)   // executor tables for 8192-point axes, work list, parameters
        return 8192 * (16 + 8 + 16) + (size_t)kListCap * (sizeof(SymbolParams) + 64);
    const size_t elem = k.precision == STENCIL_FP32 ? 4 : 8;
    int64_t cells = 1;
    for (int a = 0; a < k.ndim; ++a) cells *= k.dims[a];
    const size_t grid = (size_t)cells * elem;
    const size_t H = periodic_workspace_bytes(k.ndim, k.dims, k.precision);
    size_t tables = 0;
    for (int a = 0; a < k.ndim; ++a) tables += 48 * (size_t)k.dims[a];
    if (k.batch) return tables + kMaxItems * (grid + 2 * H + 2 * grid);
    if (k.boundary == STENCIL_PERIODIC) return tables + H;
    // zero Dirichlet: base-case scratch, interior, strip buffers per level, tables
    return tables + H + 10 * grid;
}

}  // namespace

struct stencil_server_s {
    size_t budget = 0;
    int max_slots = 1;
    int qcap = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<Pending> pending;
    struct Result {
        bool done = false;
        int status = STENCIL_OK;
        double latency = 0.0;
    };
    std::unordered_map<uint64_t, Result> results;
    std::vector<PlanEntry*> plans;
    std::vector<Slot> slots;
    size_t in_use = 0;
    uint64_t tick = 0;
    stencil_server_stats_t stats;

    void loop();
    bool admit_one(std::unique_lock<std::mutex>& lock);
    PlanEntry* acquire(const Key& k, int* status);
    int launch(Slot& sl);
    void release_plan(PlanEntry* pe);
    void complete(Slot& sl, double t);
};

// Frees an idle plan: its last launch has completed (the event is waited on,
// which returns at once for an idle plan), so no device-wide synchronisation.
void stencil_server_s::release_plan(PlanEntry* pe) {
    if (pe->last) {
        cudaEventSynchronize(pe->last);
        cudaEventDestroy(pe->last);
    }
    if (pe->plan) plan_free_idle(pe->plan);
    if (pe->exec) stencil_batch_destroy(pe->exec);
    cudaFree(pe->stackS);
    cudaFree(pe->stackH);
    for (void* v : pe->vt) cudaFree(v);
    in_use -= std::min(in_use, pe->bytes);
    delete pe;
}

// An idle plan for key k, creating one (and evicting idle plans of other keys)
// when needed. Returns nullptr with *status = 0 when the budget is full for now.
PlanEntry* stencil_server_s::acquire(const Key& k, int* status) {
    *status = STENCIL_OK;
    for (PlanEntry* pe : plans)
        if (!pe->busy && pe->key == k) return pe;
    const size_t need = estimate_bytes(k);
    while (in_use + need > budget) {
        PlanEntry* victim = nullptr;
        for (PlanEntry* pe : plans)
            if (!pe->busy && (!victim || pe->last_use < victim->last_use)) victim = pe;
        if (!victim) break;
        plans.erase(std::find(plans.begin(), plans.end(), victim));
        release_plan(victim);
    }
    if (in_use + need > budget) {
        bool any_busy = false;
        for (PlanEntry* pe : plans) any_busy |= pe->busy;
        if (!any_busy) *status = STENCIL_ENOMEM;   // can never fit this budget
        return nullptr;
    }
    PlanEntry* pe = new PlanEntry();
    pe->key = k;
    if (k.batch == 2) {
        int rc = stencil_batch_create(&pe->exec, kListCap, k.precision);
        if (rc == STENCIL_OK && cudaEventCreateWithFlags(&pe->last, cudaEventDisableTiming) != cudaSuccess)
            rc = STENCIL_ECUDA;
        if (rc != STENCIL_OK) {
            *status = rc;
            release_plan(pe);
            return nullptr;
        }
        pe->bytes = need;
        in_use += need;
        plans.push_back(pe);
        return pe;
    }
    double w0[kMaxWeights];
    std::fill(w0, w0 + kMaxWeights, 0.0);
    const int r = k.batch ? 0 : k.radius;
    int nw = 1;
    for (int a = 0; a < k.ndim; ++a) nw *= 2 * r + 1;
    w0[nw / 2] = 1.0;
    int rc = stencil_plan(&pe->plan, k.ndim, k.dims, r, w0, k.boundary, k.precision);
    if (rc == STENCIL_OK && pe->plan->vflags) {
        // every request sets its own weights, so the repeated-T table of a 2-D
        // plan would rarely be reused: the pool does not hold it
        stencil_plan_s* p = pe->plan;
        const int64_t nx = blocked_item_elems(ilog2_exact(p->dims[0]), ilog2_exact(p->dims[1]) - 1) >> 13;
        p->dev_bytes -= multiplier_table_bytes(p->ndim, p->dims, p->precision) + nx * sizeof(int);
        cudaFree(p->vt);
        cudaFree(p->vflags);
        p->vt = nullptr;
        p->vflags = nullptr;
    }
    if (rc == STENCIL_OK && k.batch) {
        const size_t elem = k.precision == STENCIL_FP32 ? 4 : 8;
        int64_t cells = 1;
        for (int a = 0; a < k.ndim; ++a) cells *= k.dims[a];
        pe->cells = (size_t)cells;
        pe->h_item = periodic_workspace_bytes(k.ndim, k.dims, k.precision);
        const int64_t n = k.dims[k.ndim - 1] / 2;
        pe->v_item = k.ndim == 1 ? (size_t)(n + 1) * 2 * elem : pe->h_item;
        cudaError_t err = cudaMalloc(&pe->stackS, kMaxItems * pe->cells * elem);
        if (err == cudaSuccess && pe->h_item) err = cudaMalloc(&pe->stackH, kMaxItems * pe->h_item);
        for (int i = 0; i < kMaxItems && err == cudaSuccess; ++i) err = cudaMalloc(&pe->vt[i], pe->v_item);
        if (err != cudaSuccess) rc = err == cudaErrorMemoryAllocation ? STENCIL_ENOMEM : STENCIL_ECUDA;
    }
    if (rc == STENCIL_OK && cudaEventCreateWithFlags(&pe->last, cudaEventDisableTiming) != cudaSuccess)
        rc = STENCIL_ECUDA;
    if (rc != STENCIL_OK) {
        *status = rc;
        release_plan(pe);
        return nullptr;
    }
    pe->plan->use_graphs = false;   // every request brings its own weights
    pe->bytes = need;
    in_use += need;
    plans.push_back(pe);
    return pe;
}

// Enqueue the slot's request(s) on its stream; returns a status for them.
int stencil_server_s::launch(Slot& sl) {
    PlanEntry* pe = sl.pe;
    if (pe->key.batch == 2) {
        // mixed shapes: one run of the batch executor, in place on every grid
        std::vector<stencil_request> reqs(sl.reqs.size());
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            reqs[i] = sl.reqs[i].r;
            reqs[i].weights = sl.reqs[i].w.data();
        }
        const int rc = stencil_batch_run(pe->exec, (int)reqs.size(), reqs.data(), sl.stream);
        if (rc == STENCIL_OK) sl.batched = (int)reqs.size();
        return rc;
    }
    stencil_plan_s* p = pe->plan;
    if (!pe->key.batch) {
        const Pending& q = sl.reqs[0];
        plan_set_weights(p, q.r.radius, q.w.data());
        return stencil_run(p, q.r.grid, q.r.T, sl.stream);
    }
    // batched small periodic requests
    const size_t elem = p->elem;
    const int items = (int)sl.reqs.size();
    cudaError_t err = cudaSuccess;
    const void* vitems[kMaxItems] = {};
    for (int i = 0; i < items && err == cudaSuccess; ++i) {
        const Pending& q = sl.reqs[i];
        err = cudaMemcpyAsync(static_cast<char*>(pe->stackS) + i * pe->cells * elem, q.r.grid,
                              pe->cells * elem, cudaMemcpyDeviceToDevice, sl.stream);
        if (err != cudaSuccess) break;
        // the request's multipliers V = Lambda^T / N (its weights, its T)
        stencil_plan_s tmp;
        tmp.ndim = p->ndim;
        tmp.precision = p->precision;
        for (int a = 0; a < 3; ++a) tmp.dims[a] = p->dims[a];
        tmp.radius = q.r.radius;
        tmp.nweights = 1;
        for (int a = 0; a < p->ndim; ++a) tmp.nweights *= 2 * q.r.radius + 1;
        std::copy(q.w.begin(), q.w.end(), tmp.weights);
        plan_set_weights(&tmp, q.r.radius, q.w.data());
        const SymbolParams sp = make_symbol_params(&tmp, p->dims, q.r.T, p->E64, p->E32, nullptr);
        err = p->precision == STENCIL_FP32 ? launch_vtable<float>(pe->vt[i], sp, p->Mp, sl.stream)
                                           : launch_vtable<double>(pe->vt[i], sp, p->Mp, sl.stream);
        vitems[i] = pe->vt[i];
    }
    if (err == cudaSuccess) {
        err = p->precision == STENCIL_FP32
                  ? batched_solve<float>(p, static_cast<float*>(pe->stackS), p->dims, items, 1,
                                         pe->stackH, p->Mp, nullptr, nullptr, 1, p->tw, p->twn_log2,
                                         p->E64, p->E32, p->status, sl.stream, nullptr, vitems)
                  : batched_solve<double>(p, static_cast<double*>(pe->stackS), p->dims, items, 1,
                                          pe->stackH, p->Mp, nullptr, nullptr, 1, p->tw,
                                          p->twn_log2, p->E64, p->E32, p->status, sl.stream,
                                          nullptr, vitems);
    }
    for (int i = 0; i < items && err == cudaSuccess; ++i)
        err = cudaMemcpyAsync(sl.reqs[i].r.grid,
                              static_cast<char*>(pe->stackS) + i * pe->cells * elem,
                              pe->cells * elem, cudaMemcpyDeviceToDevice, sl.stream);
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? STENCIL_ENOMEM : STENCIL_ECUDA;
    sl.batched = items;   // counted in the statistics under the lock
    return STENCIL_OK;
}

void stencil_server_s::complete(Slot& sl, double t) {
    cudaError_t err = cudaEventQuery(sl.done);
    int st = sl.status;
    if (st == STENCIL_OK && err != cudaSuccess) st = STENCIL_ECUDA;
    if (sl.pe) {
        sl.pe->busy = false;
        sl.pe->last_use = ++tick;
        // the zero-Dirichlet buffers exist after the first run: charge what is held
        const size_t held = sl.pe->plan ? sl.pe->plan->dev_bytes + aperiodic_bytes(sl.pe->plan) : 0;
        if (held > sl.pe->bytes) {
            in_use += held - sl.pe->bytes;
            sl.pe->bytes = held;
        }
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Pending& q : sl.reqs) {
            Result& r = results[q.ticket];
            r.done = true;
            r.status = st;
            r.latency = t - q.t_submit;
            if (st == STENCIL_OK) ++stats.completed;
            else ++stats.failed;
        }
        stats.bytes_in_use = in_use;
        stats.peak_bytes = std::max(stats.peak_bytes, in_use);
    }
    sl.reqs.clear();
    sl.pe = nullptr;
    sl.busy = false;
    cv.notify_all();
}

// Admit the head of the queue (and same-shape small periodic followers) into a
// free slot. Called with the lock held; returns false when nothing was admitted.
bool stencil_server_s::admit_one(std::unique_lock<std::mutex>& lock) {
    if (pending.empty()) return false;
    Slot* sl = nullptr;
    for (Slot& s : slots)
        if (!s.busy) {
            sl = &s;
            break;
        }
    if (!sl) return false;
    const stencil_request head = pending.front().r;
    const bool list = list_batchable(head);
    const bool batch = !list && batchable(head);
    const Key k = list ? list_key(head.precision) : key_of(head, batch);
    int status = STENCIL_OK;
    // plan pool work (eviction, creation) without the lock; the head stays at
    // the front meanwhile (only this thread removes requests)
    lock.unlock();
    PlanEntry* pe = acquire(k, &status);
    lock.lock();
    if (!pe) {
        if (status == STENCIL_OK) return false;   // wait for memory to free up
        Pending q = pending.front();
        pending.pop_front();
        Result& r = results[q.ticket];
        r.done = true;
        r.status = status;
        r.latency = now_s() - q.t_submit;
        ++stats.failed;
        cv.notify_all();
        return true;
    }
    sl->reqs.clear();
    sl->reqs.push_back(pending.front());
    pending.pop_front();
    if (list) {
        // continuous batching across shapes: every queued request one CTA can
        // solve (same precision) joins this run of the executor
        for (auto it = pending.begin(); it != pending.end() && (int)sl->reqs.size() < kListCap;) {
            if (it->r.precision == head.precision && list_batchable(it->r)) {
                sl->reqs.push_back(*it);
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
    } else if (batch) {
        // continuous batching: pull queued requests of the same shape into this launch
        for (auto it = pending.begin(); it != pending.end() && (int)sl->reqs.size() < kMaxItems;) {
            if (batchable(it->r) && key_of(it->r, true) == k) {
                sl->reqs.push_back(*it);
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
    }
    pe->busy = true;
    sl->pe = pe;
    sl->busy = true;
    lock.unlock();
    sl->batched = 0;
    sl->status = launch(*sl);
    if (sl->status == STENCIL_OK) {
        if (cudaEventRecord(sl->done, sl->stream) != cudaSuccess ||
            cudaEventRecord(pe->last, sl->stream) != cudaSuccess)
            sl->status = STENCIL_ECUDA;
    }
    int busy = 0;
    for (Slot& s : slots) busy += s.busy;
    lock.lock();
    if (sl->batched) {
        ++stats.batched_launches;
        stats.batched_requests += sl->batched;
    }
    stats.max_in_flight = std::max(stats.max_in_flight, busy);
    stats.bytes_in_use = in_use;
    stats.peak_bytes = std::max(stats.peak_bytes, in_use);
    if (sl->status != STENCIL_OK) {
        lock.unlock();
        complete(*sl, now_s());
        lock.lock();
    }
    return true;
}

void stencil_server_s::loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        // completions
        bool any_busy = false;
        for (Slot& sl : slots) {
            if (!sl.busy) continue;
            if (cudaEventQuery(sl.done) != cudaErrorNotReady) {
                lock.unlock();
                complete(sl, now_s());
                lock.lock();
            } else {
                any_busy = true;
            }
        }
        // admissions
        while (admit_one(lock)) {
        }
        any_busy = false;
        for (Slot& sl : slots) any_busy |= sl.busy;
        if (stop && pending.empty() && !any_busy) break;
        if (!any_busy && pending.empty()) {
            cv.wait(lock, [&] { return stop || !pending.empty(); });
        } else {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        }
    }
}

extern "C" {

int stencil_server_create(stencil_server_t* out, size_t hbm_budget_bytes, int max_slots,
                          int queue_capacity) {
    if (!out || max_slots < 1 || max_slots > 64 || queue_capacity < 1 || hbm_budget_bytes == 0)
        return STENCIL_EINVAL;
    *out = nullptr;
    stencil_server_s* s = new (std::nothrow) stencil_server_s();
    if (!s) return STENCIL_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->qcap = queue_capacity;
    std::memset(&s->stats, 0, sizeof(s->stats));
    s->stats.budget_bytes = hbm_budget_bytes;
    cudaGetDevice(&s->device);
    s->slots.resize(max_slots);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            for (Slot& t : s->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
            }
            delete s;
            return STENCIL_ECUDA;
        }
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return STENCIL_OK;
}

int stencil_server_submit(stencil_server_t s, const stencil_request* r, uint64_t* ticket) {
    if (!s || !ticket) return STENCIL_EINVAL;
    const int rc = validate_request(r);
    if (rc != STENCIL_OK) return rc;
    Pending q;
    q.r = *r;
    int nw = 1;
    for (int a = 0; a < r->ndim; ++a) nw *= 2 * r->radius + 1;
    q.w.assign(r->weights, r->weights + nw);
    for (double v : q.w)
        if (!std::isfinite(v)) return STENCIL_EINVAL;
    q.r.weights = nullptr;   // the copy in q.w is used
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return STENCIL_EINVAL;
        if ((int)s->pending.size() >= s->qcap) return STENCIL_EQUEUEFULL;
        q.ticket = s->next_ticket++;
        q.t_submit = now_s();
        s->results[q.ticket] = stencil_server_s::Result();
        s->pending.push_back(q);
        ++s->stats.submitted;
        *ticket = q.ticket;
    }
    s->cv.notify_all();
    return STENCIL_OK;
}

int stencil_server_poll(stencil_server_t s, uint64_t ticket, int* done, double* latency_s) {
    if (!s || !done) return STENCIL_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return STENCIL_EINVAL;
    *done = it->second.done ? 1 : 0;
    if (latency_s) *latency_s = it->second.latency;
    return it->second.done ? it->second.status : STENCIL_OK;
}

int stencil_server_wait(stencil_server_t s, uint64_t ticket, double timeout_s, double* latency_s) {
    if (!s) return STENCIL_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return STENCIL_EINVAL;
    const bool ok = s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                   [&] { return s->results[ticket].done; });
    if (!ok) return STENCIL_ETIMEOUT;
    if (latency_s) *latency_s = s->results[ticket].latency;
    return s->results[ticket].status;
}

int stencil_server_stats(stencil_server_t s, stencil_server_stats_t* out) {
    if (!s || !out) return STENCIL_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    return STENCIL_OK;
}

int stencil_server_destroy(stencil_server_t s) {
    if (!s) return STENCIL_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
    }
    for (PlanEntry* pe : s->plans) s->release_plan(pe);
    delete s;
    return STENCIL_OK;
}

}  // extern "C"
