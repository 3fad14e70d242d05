// Served form of the library (include/osscir.h, "served form"): a worker
// thread admits queued reconstruction requests into slots under a device
// memory budget.  Admitted requests are spread over a few groups of about
// equal work; each group is a batch on its own stream that advances all its
// requests together, a few MOCCA iterations per round, through the batched
// kernels (one launch per kernel per iteration for the whole group), while the
// groups run side by side.  A group's batch is re-formed between its rounds as
// requests finish and new ones join (continuous batching at iteration
// granularity).  Contexts are cached by configuration and reused; a request's
// arithmetic is exactly that of the plain form.
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
               params.counts_model == o.params.counts_model &&
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
        mix(&params.counts_model, sizeof params.counts_model);
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

constexpr int kChunk = 4;      // MOCCA iterations per round (fewer if a request needs fewer)
constexpr int kInFlight = 2;   // rounds queued per group at a time
constexpr int kGroups = 4;     // batches running side by side, each on its own stream

struct Slot {
    osscir_ctx* ctx = nullptr;
    Config cfg;
    uint64_t key = 0;
    float* h_counts = nullptr;   // pinned
    float* h_maps = nullptr;     // pinned
    double* h_dtpl = nullptr;    // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    Ticket* running = nullptr;
    int group = 0;       // the batch it runs in
    double cost = 0.0;   // relative device time of one iteration
    int remaining = 0;   // iterations not yet enqueued
    bool tail = false;   // results copy-back enqueued
    bool failed = false;
    uint64_t last_used = 0;
    size_t bytes = 0;
};

// Device bytes a context of this configuration needs (exception table estimated).
size_t estimate_bytes(const Config& c) {
    const size_t L = (size_t)c.geom.n_views * c.geom.n_bins, P = (size_t)c.geom.n * c.geom.n;
    const size_t per_ray = 64 + 32 + 4 + 4 + 16 + 16 + 8 * 4 / 128 + 2;   // records, FP64 rays, chord, offsets, c, y, partials
    const size_t mu_pc = c.params.spc == 2 ? P * 16 + 12 * c.nE : 0;   // the caller's curves and a maps buffer
    // footprint tables: about 0.9 n footprint pairs per ray (0.82 n measured at 256 x 256), 6.9 bytes each
    // in the forward table and 7.5 in the back-projection's (with the rows' padding), and the view
    // groups' channel sums (at most 8 groups of 36 bytes per pixel)
    const size_t tables = (size_t)(0.9 * c.geom.n * (double)L * 14.4) + P * 288 + L * 12;
    // x, and xbar with its column-major copy: 48 bytes per pixel
    return L * per_ray + P * 48 + (size_t)c.nE * c.geom.n_bins * 16 + c.geom.n_bins * 16 + 12 * c.nE +
           c.geom.n_views * 8 + (L / 8) * 8 + mu_pc + tables + (1 << 16);
}

void release_slot(Slot* s) {
    if (s->ctx) osscir::ctx_destroy(s->ctx);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
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
    std::condition_variable cv_done;
    // Wake-ups of the worker: bumped by submissions, by destroy and by a host
    // callback that each stream runs when a round or a request's results are
    // done on the GPU, so an idle worker sleeps instead of polling its events.
    std::mutex mu_sig;
    std::condition_variable cv_sig;
    uint64_t sig = 0;
    void signal() {
        {
            std::lock_guard<std::mutex> g(mu_sig);
            ++sig;
        }
        cv_sig.notify_all();
    }
    std::deque<Ticket*> queue;
    std::unordered_map<uint64_t, Ticket*> tickets;
    std::list<Slot*> slots;
    size_t bytes_in_use = 0;
    int running = 0;
    bool stop = false;
    uint64_t next_id = 1, clock = 0;
    std::thread worker;
    // worker-thread state: per group its stream, batch and rounds in flight
    struct Group {
        cudaStream_t stream = nullptr;
        osscir::BatchRun* batch = nullptr;
        std::vector<osscir_ctx*> members;
        std::deque<cudaEvent_t> rounds;
        double load = 0.0;
    };
    Group groups[kGroups];
    std::deque<cudaEvent_t> spare;

    void run();
    Slot* acquire(Ticket* t);     // with mu held
    bool begin(Slot* s);          // worker thread, no lock
    bool enqueue_round(int g);    // worker thread, no lock
    bool enqueue_tail(Slot* s);   // worker thread, no lock
    void finish(Slot* s);         // with mu held
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
        for (Group& g : groups) g.members.clear();   // a new context may reuse the address: re-form the batches
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
    if (st == OSSCIR_OK) st = osscir::ctx_build_tables(s->ctx);   // counted in the context's bytes below
    const size_t L = (size_t)t->cfg.geom.n_views * t->cfg.geom.n_bins, P = (size_t)t->cfg.geom.n * t->cfg.geom.n;
    if (st == OSSCIR_OK && (cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess ||
                            cudaHostAlloc(&s->h_counts, L * 16, cudaHostAllocDefault) != cudaSuccess ||
                            cudaHostAlloc(&s->h_maps, P * 16, cudaHostAllocDefault) != cudaSuccess ||
                            cudaHostAlloc(&s->h_dtpl, sizeof(double), cudaHostAllocDefault) != cudaSuccess))
        st = OSSCIR_E_NOMEM;
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

// Copy the counts in and reset the state (the iterations follow in rounds).
// Host callback run in stream order after a round or a result copy: wake the worker.
void CUDART_CB gpu_progress(void* p) { static_cast<osscir_server*>(p)->signal(); }

bool osscir_server::begin(Slot* s) {
    Ticket* t = s->running;
    osscir_ctx* h = s->ctx;
    std::memcpy(s->h_counts, t->counts.data(), t->counts.size() * sizeof(float));
    cudaStream_t st = groups[s->group].stream;
    s->remaining = t->n_iters;
    s->tail = s->failed = false;
    h->iter = 0;
    return cudaEventRecord(s->ev0, st) == cudaSuccess &&
           cudaMemcpyAsync(h->c, s->h_counts, sizeof(float4) * h->L, cudaMemcpyHostToDevice, st) == cudaSuccess &&
           cudaMemsetAsync(h->y, 0, sizeof(float4) * h->L, st) == cudaSuccess &&
           cudaMemsetAsync(h->x, 0, sizeof(float4) * h->P, st) == cudaSuccess &&
           cudaMemsetAsync(h->xbar, 0, sizeof(float4) * 2 * h->P, st) == cudaSuccess &&
           cudaMemsetAsync(h->dtpl_out, 0, sizeof(double) * 2, st) == cudaSuccess;
}

// Results of a request whose iterations are all enqueued: maps and D_TPL back
// to pinned host memory, then its completion event.
bool osscir_server::enqueue_tail(Slot* s) {
    osscir_ctx* h = s->ctx;
    cudaStream_t stream = groups[s->group].stream;
    const bool ok =
        cudaMemcpyAsync(s->h_maps, h->x, sizeof(float4) * h->P, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
        cudaMemcpyAsync(s->h_dtpl, h->dtpl_out + 1, sizeof(double), cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
        cudaEventRecord(s->ev1, stream) == cudaSuccess &&
        cudaLaunchHostFunc(stream, gpu_progress, this) == cudaSuccess;
    s->tail = true;
    return ok;
}

// One round of group g: every running request of the group that still has
// iterations to do advances by k = min(kChunk, fewest remaining) iterations in
// the batched kernels; the group's batch is re-formed first if its members
// changed.  False if nothing was enqueued.
bool osscir_server::enqueue_round(int g) {
    Group& G = groups[g];
    std::vector<osscir_ctx*> active;
    std::vector<Slot*> act;
    int k = kChunk;
    for (Slot* s : slots)
        if (s->running && s->group == g && !s->failed && !s->tail && s->remaining > 0) {
            active.push_back(s->ctx);
            act.push_back(s);
            k = std::min(k, s->remaining);
        }
    if (act.empty()) return false;
    osscir_status st = OSSCIR_OK;
    if (active != G.members) {
        st = osscir::batchrun_set(G.batch, active, 1, G.stream);
        G.members = active;
    }
    if (st == OSSCIR_OK) st = osscir::batchrun_step(G.batch, k, G.stream);
    cudaEvent_t ev = nullptr;
    if (!spare.empty()) {
        ev = spare.front();
        spare.pop_front();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        ev = nullptr;
    }
    if (st == OSSCIR_OK && ev && cudaEventRecord(ev, G.stream) == cudaSuccess &&
        cudaLaunchHostFunc(G.stream, gpu_progress, this) == cudaSuccess) {
        G.rounds.push_back(ev);
    } else {
        if (ev) spare.push_back(ev);
        st = OSSCIR_E_CUDA;
    }
    for (Slot* s : act) {
        if (st != OSSCIR_OK) {
            s->failed = true;
            G.members.clear();   // the batch must be rebuilt before it is used again
            continue;
        }
        s->remaining -= k;
        if (s->remaining == 0 && !enqueue_tail(s)) s->failed = true;
    }
    return true;
}

void osscir_server::finish(Slot* s) {
    Ticket* t = s->running;
    const osscir_ctx* h = s->ctx;
    groups[s->group].load -= s->cost;
    if (s->failed) {
        cudaStreamSynchronize(groups[s->group].stream);
        t->status = OSSCIR_E_CUDA;
        t->t_done = clk::now();
        t->done = true;
        s->running = nullptr;
        --running;
        return;
    }
    s->ctx->iter = t->n_iters;
    t->maps.assign(s->h_maps, s->h_maps + (size_t)h->P * 4);
    osscir::ctx_maps_out_host(h, t->maps.data());
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
    bool dead = false;
    for (Group& g : groups) {
        dead = dead || cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess;
        g.batch = osscir::batchrun_new();
        dead = dead || !g.batch;
    }
    std::vector<Slot*> started;
    while (true) {
        started.clear();
        uint64_t seen;
        {
            std::lock_guard<std::mutex> g(mu_sig);
            seen = sig;   // any wake-up after this point ends the idle wait below at once
        }
        {
            std::unique_lock<std::mutex> lock(mu);
            if (stop && running == 0) break;
            // admissions, first come first served, while a slot and the memory budget allow
            while (!stop && !queue.empty() && running < max_slots) {
                Ticket* t = queue.front();
                Slot* s = dead ? reinterpret_cast<Slot*>(-1) : acquire(t);
                if (!s) break;   // wait for memory
                queue.pop_front();
                if (s == reinterpret_cast<Slot*>(-1)) {
                    if (dead) t->status = OSSCIR_E_CUDA;
                    t->t_start = t->t_done = clk::now();
                    t->done = true;
                    cv_done.notify_all();
                    continue;
                }
                s->running = t;
                s->last_used = ++clock;
                s->cost = osscir::batch_solve_cost(s->ctx);
                s->group = 0;
                for (int g = 1; g < kGroups; ++g)
                    if (groups[g].load < groups[s->group].load) s->group = g;
                groups[s->group].load += s->cost;
                t->t_start = clk::now();
                ++running;
                started.push_back(s);
            }
        }
        // CUDA work without the lock: the worker thread alone touches the stream and the batch
        bool acted = !started.empty();
        for (Slot* s : started)
            if (!begin(s)) s->failed = true;
        for (int g = 0; g < kGroups; ++g) {
            std::deque<cudaEvent_t>& rounds = groups[g].rounds;
            while (!rounds.empty()) {
                const cudaError_t q = cudaEventQuery(rounds.front());
                if (q == cudaErrorNotReady) break;
                spare.push_back(rounds.front());
                rounds.pop_front();
                acted = true;
            }
            while ((int)rounds.size() < kInFlight && enqueue_round(g)) acted = true;
        }
        std::vector<Slot*> done;
        for (Slot* s : slots) {
            if (!s->running) continue;
            if (!s->tail && (s->failed || s->remaining == 0)) {
                if (!enqueue_tail(s)) s->failed = true;
                acted = true;
            }
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
            // sleep until a submission, destroy, or a stream's callback; the 50 ms limit
            // only bounds the cost of a callback that could not be enqueued
            const bool busy = running > 0, idle = !stop && queue.empty();
            lock.unlock();
            std::unique_lock<std::mutex> ls(mu_sig);
            if (busy) cv_sig.wait_for(ls, std::chrono::milliseconds(50), [&] { return sig != seen; });
            else if (idle) cv_sig.wait(ls, [&] { return sig != seen; });
        }
    }
    for (Group& g : groups) {
        if (g.stream) cudaStreamSynchronize(g.stream);
        for (cudaEvent_t e : g.rounds) cudaEventDestroy(e);
        g.rounds.clear();
        osscir::batchrun_free(g.batch);
        g.batch = nullptr;
        if (g.stream) cudaStreamDestroy(g.stream);
        g.stream = nullptr;
    }
    for (cudaEvent_t e : spare) cudaEventDestroy(e);
    spare.clear();
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
    s->signal();
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
    if (req->params.inner > 1) return OSSCIR_E_INVALID;   // nested solves are not served
    if (req->spectra.n_windows != 0 && req->spectra.n_windows != 4) return OSSCIR_E_INVALID;   // four windows
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
        t->cfg.params.inner = 1;
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
    s->signal();
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
