// Served form of the library (include/osscir.h, "served form"): a worker
// thread admits queued reconstruction requests into slots under a device
// memory budget and runs each admitted request's MOCCA iterations on its own
// stream, so requests that arrive while others are on the GPU join the work
// in flight (continuous batching).  Contexts are cached by configuration and
// reused; a request's arithmetic is exactly that of the plain form.
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <deque>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "osscir_ctx.h"

namespace {

using clk = std::chrono::steady_clock;

double ms_between(clk::time_point a, clk::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// A request's own copy of its problem.
struct Config {
    osscir_geometry geom{};
    int nE = 0;
    std::vector<float> s, N, mu;
    osscir_params params{};

    bool same(const Config& o) const {
        return std::memcmp(&geom, &o.geom, sizeof geom) == 0 && nE == o.nE && s == o.s && N == o.N && mu == o.mu &&
               params.lambda == o.params.lambda && params.model == o.params.model && params.spc == o.params.spc &&
               params.use_box == o.params.use_box && std::memcmp(params.lo, o.params.lo, sizeof params.lo) == 0 &&
               std::memcmp(params.hi, o.params.hi, sizeof params.hi) == 0;
    }
    uint64_t hash() const {   // FNV-1a over the configuration bytes
        uint64_t h = 1469598103934665603ULL;
        auto mix = [&](const void* p, size_t n) {
            const unsigned char* b = static_cast<const unsigned char*>(p);
            for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
        };
        mix(&geom, sizeof geom);
        mix(s.data(), s.size() * sizeof(float));
        mix(N.data(), N.size() * sizeof(float));
        mix(mu.data(), mu.size() * sizeof(float));
        mix(&params.lambda, sizeof params.lambda);
        mix(&params.model, sizeof params.model);
        mix(&params.spc, sizeof params.spc);
        return h;
    }
};

struct Ticket {
    uint64_t id = 0;
    Config cfg;
    uint64_t key = 0;
    std::vector<float> counts;
    int n_iters = 0;
    size_t need = 0;
    clk::time_point t_submit, t_start, t_done;
    bool done = false;
    osscir_status status = OSSCIR_OK;
    std::vector<float> maps;
    double dtpl = 0.0;
    float gpu_ms = 0.f;
};

constexpr int kChunk = 4;      // MOCCA iterations per enqueued chunk
constexpr int kInFlight = 2;   // chunks queued per stream at a time

struct Slot {
    osscir_ctx* ctx = nullptr;
    Config cfg;
    uint64_t key = 0;
    cudaStream_t stream = nullptr;
    float* h_counts = nullptr;   // pinned
    float* h_maps = nullptr;     // pinned
    double* h_dtpl = nullptr;    // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evc[kInFlight] = {nullptr, nullptr};
    Ticket* running = nullptr;
    int enq = 0;        // iterations enqueued
    int head = 0;       // oldest chunk event in flight
    int in_flight = 0;  // chunks in flight
    bool tail = false;  // results copy-back enqueued
    bool failed = false;
    uint64_t last_used = 0;
    size_t bytes = 0;
};

// Device bytes a context of this configuration needs (exception table estimated).
size_t estimate_bytes(const Config& c) {
    const size_t L = (size_t)c.geom.n_views * c.geom.n_bins, P = (size_t)c.geom.n * c.geom.n;
    const size_t per_ray = 64 + 32 + 4 + 4 + 16 + 16 + 8 * 4 / 128 + 2;   // records, FP64 rays, chord, offsets, c, y, partials
    return L * per_ray + P * 32 + (size_t)c.nE * c.geom.n_bins * 16 + c.geom.n_bins * 16 + 12 * c.nE +
           c.geom.n_views * 8 + (L / 8) * 8 + (1 << 16);
}

void release_slot(Slot* s) {
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->ctx) osscir::ctx_destroy(s->ctx);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    for (cudaEvent_t e : s->evc)
        if (e) cudaEventDestroy(e);
    if (s->h_counts) cudaFreeHost(s->h_counts);
    if (s->h_maps) cudaFreeHost(s->h_maps);
    if (s->h_dtpl) cudaFreeHost(s->h_dtpl);
    delete s;
}

}  // namespace

struct osscir_server {
    int device = 0;
    size_t budget = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Ticket*> queue;
    std::unordered_map<uint64_t, Ticket*> tickets;
    std::list<Slot*> slots;
    size_t bytes_in_use = 0;
    int running = 0;
    bool stop = false;
    uint64_t next_id = 1, clock = 0;
    std::thread worker;

    void run();
    Slot* acquire(Ticket* t);   // with mu held
    bool begin(Slot* s);        // worker thread, no lock
    bool advance(Slot* s);      // worker thread, no lock; true if anything happened
    void finish(Slot* s);       // with mu held
};

// An idle cached context of the same configuration, or a new one once memory
// allows (idle contexts are released least recently used first).  nullptr: wait.
Slot* osscir_server::acquire(Ticket* t) {
    for (Slot* s : slots)
        if (!s->running && s->key == t->key && s->cfg.same(t->cfg)) return s;
    while (bytes_in_use + t->need > budget) {
        Slot* victim = nullptr;
        for (Slot* s : slots)
            if (!s->running && (!victim || s->last_used < victim->last_used)) victim = s;
        if (!victim) return nullptr;
        slots.remove(victim);
        bytes_in_use -= victim->bytes;
        release_slot(victim);
    }
    Slot* s = new (std::nothrow) Slot();
    if (!s) return nullptr;
    s->cfg = t->cfg;
    s->key = t->key;
    osscir_spectra sp{t->cfg.nE, t->cfg.s.data(), t->cfg.N.data()};
    osscir_status st = osscir::ctx_create(&t->cfg.geom, &sp, t->cfg.mu.data(), &t->cfg.params, &s->ctx);
    const size_t L = (size_t)t->cfg.geom.n_views * t->cfg.geom.n_bins, P = (size_t)t->cfg.geom.n * t->cfg.geom.n;
    if (st == OSSCIR_OK && (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
                            cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess ||
                            cudaEventCreateWithFlags(&s->evc[0], cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventCreateWithFlags(&s->evc[1], cudaEventDisableTiming) != cudaSuccess ||
                            cudaHostAlloc(&s->h_counts, L * 16, cudaHostAllocDefault) != cudaSuccess ||
                            cudaHostAlloc(&s->h_maps, P * 16, cudaHostAllocDefault) != cudaSuccess ||
                            cudaHostAlloc(&s->h_dtpl, sizeof(double), cudaHostAllocDefault) != cudaSuccess))
        st = OSSCIR_E_NOMEM;
    if (st == OSSCIR_OK) st = osscir::ctx_ensure_graph(s->ctx);
    if (st != OSSCIR_OK) {
        release_slot(s);
        t->status = st;
        return reinterpret_cast<Slot*>(-1);
    }
    s->bytes = s->ctx->bytes;
    bytes_in_use += s->bytes;
    slots.push_back(s);
    return s;
}

// Copy the counts in and reset the state (the iterations follow in chunks).
bool osscir_server::begin(Slot* s) {
    Ticket* t = s->running;
    osscir_ctx* h = s->ctx;
    std::memcpy(s->h_counts, t->counts.data(), t->counts.size() * sizeof(float));
    cudaStream_t st = s->stream;
    s->enq = s->head = s->in_flight = 0;
    s->tail = s->failed = false;
    h->iter = 0;
    return cudaEventRecord(s->ev0, st) == cudaSuccess &&
           cudaMemcpyAsync(h->c, s->h_counts, sizeof(float4) * h->L, cudaMemcpyHostToDevice, st) == cudaSuccess &&
           cudaMemsetAsync(h->y, 0, sizeof(float4) * h->L, st) == cudaSuccess &&
           cudaMemsetAsync(h->x, 0, sizeof(float4) * h->P, st) == cudaSuccess &&
           cudaMemsetAsync(h->xbar, 0, sizeof(float4) * h->P, st) == cudaSuccess &&
           cudaMemsetAsync(h->dtpl_out, 0, sizeof(double) * 2, st) == cudaSuccess;
}

// Keep at most kInFlight chunks of kChunk iterations queued on the slot's
// stream, then the copy-back of the results; returns true if it did anything.
bool osscir_server::advance(Slot* s) {
    Ticket* t = s->running;
    osscir_ctx* h = s->ctx;
    bool acted = false;
    while (s->in_flight > 0) {
        const cudaError_t q = cudaEventQuery(s->evc[s->head]);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) s->failed = true;
        s->head = (s->head + 1) % kInFlight;
        --s->in_flight;
        acted = true;
    }
    while (!s->tail && !s->failed && s->in_flight < kInFlight && s->enq < t->n_iters) {
        const int k = std::min(kChunk, t->n_iters - s->enq);
        bool ok = true;
        for (int i = 0; ok && i < k; ++i) ok = cudaGraphLaunch(h->gexec, s->stream) == cudaSuccess;
        ok = ok && cudaEventRecord(s->evc[(s->head + s->in_flight) % kInFlight], s->stream) == cudaSuccess;
        if (!ok) s->failed = true;
        ++s->in_flight;
        s->enq += k;
        acted = true;
    }
    if (!s->tail && (s->enq >= t->n_iters || s->failed)) {
        const bool ok =
            cudaMemcpyAsync(s->h_maps, h->x, sizeof(float4) * h->P, cudaMemcpyDeviceToHost, s->stream) == cudaSuccess &&
            cudaMemcpyAsync(s->h_dtpl, h->dtpl_out + 1, sizeof(double), cudaMemcpyDeviceToHost, s->stream) ==
                cudaSuccess &&
            cudaEventRecord(s->ev1, s->stream) == cudaSuccess;
        if (!ok) s->failed = true;
        h->iter = s->enq;
        s->tail = true;
        acted = true;
    }
    return acted;
}

void osscir_server::finish(Slot* s) {
    Ticket* t = s->running;
    const osscir_ctx* h = s->ctx;
    if (s->failed) {
        cudaStreamSynchronize(s->stream);
        t->status = OSSCIR_E_CUDA;
        t->t_done = clk::now();
        t->done = true;
        s->running = nullptr;
        --running;
        return;
    }
    t->maps.assign(s->h_maps, s->h_maps + (size_t)h->P * 4);
    t->dtpl = *s->h_dtpl;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev0, s->ev1);
    t->gpu_ms = ms;
    t->status = (t->n_iters > 0 && !std::isfinite(t->dtpl)) ? OSSCIR_E_DIVERGED : OSSCIR_OK;
    for (float v : t->maps)
        if (!std::isfinite(v)) {
            t->status = OSSCIR_E_DIVERGED;
            break;
        }
    t->t_done = clk::now();
    t->done = true;
    s->running = nullptr;
    --running;
}

void osscir_server::run() {
    cudaSetDevice(device);
    std::vector<Slot*> started;
    while (true) {
        started.clear();
        {
            std::unique_lock<std::mutex> lock(mu);
            if (stop && running == 0) break;
            // admissions, first come first served, while a slot and the memory budget allow
            while (!stop && !queue.empty() && running < max_slots) {
                Ticket* t = queue.front();
                Slot* s = acquire(t);
                if (!s) break;   // wait for memory
                queue.pop_front();
                if (s == reinterpret_cast<Slot*>(-1)) {
                    t->t_start = t->t_done = clk::now();
                    t->done = true;
                    cv_done.notify_all();
                    continue;
                }
                s->running = t;
                s->last_used = ++clock;
                t->t_start = clk::now();
                ++running;
                started.push_back(s);
            }
        }
        // CUDA work without the lock: the worker thread alone touches the slots' streams
        bool acted = !started.empty();
        for (Slot* s : started)
            if (!begin(s)) s->failed = true;
        std::vector<Slot*> done;
        for (Slot* s : slots) {
            if (!s->running) continue;
            if (advance(s)) acted = true;
            if (s->tail) {
                const cudaError_t q = cudaEventQuery(s->ev1);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) s->failed = true;
                done.push_back(s);
            }
        }
        std::unique_lock<std::mutex> lock(mu);
        for (Slot* s : done) finish(s);
        if (!done.empty()) {
            cv_done.notify_all();
            acted = true;
        }
        if (!acted) {
            if (running > 0) cv_work.wait_for(lock, std::chrono::microseconds(20));
            else if (!stop && queue.empty()) cv_work.wait(lock);
        }
    }
}

extern "C" {

osscir_status osscir_server_create(size_t hbm_budget_bytes, int max_slots, osscir_server_t* out) {
    if (!out) return OSSCIR_E_INVALID;
    *out = nullptr;
    if (max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0) return OSSCIR_E_INVALID;
    osscir_server* s = new (std::nothrow) osscir_server();
    if (!s) return OSSCIR_E_NOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return OSSCIR_E_CUDA;
    }
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    try {
        s->worker = std::thread([s] { s->run(); });
    } catch (...) {
        delete s;
        return OSSCIR_E_NOMEM;
    }
    *out = s;
    return OSSCIR_OK;
}

osscir_status osscir_server_destroy(osscir_server_t s) {
    if (!s) return OSSCIR_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (Ticket* t : s->queue) {
            t->status = OSSCIR_E_NOTFOUND;
            t->done = true;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot* sl : s->slots) release_slot(sl);
    for (auto& kv : s->tickets) delete kv.second;
    delete s;
    return OSSCIR_OK;
}

osscir_status osscir_submit(osscir_server_t s, const osscir_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || !req->counts || req->n_iters < 0) return OSSCIR_E_INVALID;
    const osscir_status v = osscir::ctx_validate(&req->geom, &req->spectra, req->mu, &req->params);
    if (v != OSSCIR_OK) return v;
    Ticket* t = new (std::nothrow) Ticket();
    if (!t) return OSSCIR_E_NOMEM;
    const osscir_geometry& g = req->geom;
    const size_t L = (size_t)g.n_views * g.n_bins, nE = req->spectra.n_energies;
    try {
        t->cfg.geom = g;
        t->cfg.nE = (int)nE;
        t->cfg.s.assign(req->spectra.s, req->spectra.s + (size_t)g.n_bins * nE * 4);
        t->cfg.N.assign(req->spectra.N, req->spectra.N + (size_t)g.n_bins * 4);
        t->cfg.mu.assign(req->mu, req->mu + 3 * nE);
        t->cfg.params = req->params;
        t->counts.assign(req->counts, req->counts + L * 4);
    } catch (...) {
        delete t;
        return OSSCIR_E_NOMEM;
    }
    for (float c : t->counts)
        if (!std::isfinite(c) || c < 0.f) {
            delete t;
            return OSSCIR_E_INVALID;
        }
    t->n_iters = req->n_iters;
    t->key = t->cfg.hash();
    t->need = estimate_bytes(t->cfg);
    if (t->need > s->budget) {
        delete t;
        return OSSCIR_E_BUSY;
    }
    t->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete t;
            return OSSCIR_E_INVALID;
        }
        t->id = s->next_id++;
        s->tickets[t->id] = t;
        s->queue.push_back(t);
        *ticket = t->id;
    }
    s->cv_work.notify_all();
    return OSSCIR_OK;
}

osscir_status osscir_poll(osscir_server_t s, uint64_t ticket, int timeout_ms, float* maps_out, osscir_stats* stats) {
    if (!s) return OSSCIR_E_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return OSSCIR_E_NOTFOUND;
    Ticket* t = it->second;
    if (!t->done) {
        if (timeout_ms < 0) s->cv_done.wait(lock, [t] { return t->done; });
        else s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [t] { return t->done; });
    }
    if (!t->done) return OSSCIR_E_TIMEOUT;
    s->tickets.erase(it);
    lock.unlock();
    if (maps_out && !t->maps.empty()) std::memcpy(maps_out, t->maps.data(), t->maps.size() * sizeof(float));
    if (stats) {
        stats->status = t->status;
        stats->iterations = t->status == OSSCIR_OK ? t->n_iters : 0;
        stats->dtpl = t->dtpl;
        stats->latency_ms = ms_between(t->t_submit, t->t_done);
        stats->queue_ms = ms_between(t->t_submit, t->t_start);
        stats->gpu_ms = t->gpu_ms;
    }
    const osscir_status st = t->status;
    delete t;
    return st;
}

osscir_status osscir_server_info(osscir_server_t s, int* running, int* queued, size_t* bytes_in_use) {
    if (!s) return OSSCIR_E_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    if (running) *running = s->running;
    if (queued) *queued = (int)s->queue.size();
    if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
    return OSSCIR_OK;
}

}  // extern "C"
