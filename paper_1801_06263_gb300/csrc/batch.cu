// Batched form of the C-ABI (include/osscir.h): many independent solves
// advanced by one launch per kernel (per branch) per MOCCA step, over work
// lists of (solve, tile) items, captured once as a CUDA graph whose branches
// run concurrently; the autotuner that picks tile shapes, grid policy,
// work-list order and branch count by timing them on the batch itself; and the
// batch runner the served form drives.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "osscir_ctx.h"

using namespace osscir;

namespace {

osscir_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return OSSCIR_OK;
    if (e == cudaErrorMemoryAllocation) return OSSCIR_E_NOMEM;
    return OSSCIR_E_CUDA;
}

#define CK(expr)                                        \
    do {                                                \
        const cudaError_t e_ = (expr);                  \
        if (e_ != cudaSuccess) return from_cuda(e_);    \
    } while (0)

#define CKS(expr)                                       \
    do {                                                \
        const osscir_status s_ = (expr);                \
        if (s_ != OSSCIR_OK) return s_;                 \
    } while (0)

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

constexpr int kMaxBranches = 4;
constexpr osscir_batch_config kDefault = {4, 0, 0, 0, 0, 2, 0, 0, 1};

bool valid_config(const osscir_batch_config& c) {
    const auto pow2_in = [](int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; };
    const auto grid_ok = [](int g) { return g >= 0 && g <= (1 << 20); };
    const auto order_ok = [](int o) { return o >= 0 && o <= 2; };
    return pow2_in(c.proj_views, 1, 8) && pow2_in(c.bp_tile_x, 2, 32) && grid_ok(c.proj_grid) &&
           grid_ok(c.ray_grid) && grid_ok(c.bp_grid) && order_ok(c.proj_order) && order_ok(c.ray_order) &&
           order_ok(c.bp_order) && pow2_in(c.branches, 1, kMaxBranches);
}

SolveDesc make_desc(const osscir_ctx* h) {
    SolveDesc d{};
    d.C = h->gc;
    d.E = h->exc();
    d.rec = h->rec;
    d.views = h->views;
    d.S = h->spec();
    d.P = h->params;
    d.D = h->solve();
    d.dtpl_out = h->dtpl_out + 1;
    d.n_part = h->n_part;
    d.bp_groups = bp_view_groups(h->P, h->g64.n_views);
    d.T = h->fp_state == 1 ? h->fp() : FpTables{};
    return d;
}

// Whether every solve has its footprint tables (then the batch streams them;
// otherwise all solves take the on-the-fly kernels).
bool all_tables(const std::vector<osscir_ctx*>& ctx) {
    for (const osscir_ctx* h : ctx)
        if (h->fp_state != 1 || !h->bp_w) return false;
    return !ctx.empty();
}

// Build the footprint tables of every solve that has none yet.
osscir_status build_all_tables(const std::vector<osscir_ctx*>& ctx) {
    for (osscir_ctx* h : ctx) CKS(ctx_build_tables(h));
    return OSSCIR_OK;
}

// Relative device time of one iteration of a solve: footprint pairs (~ rays x
// image side) for the projection, rays x energies for the per-ray step, pixels
// x views for the back-projection, weighted by their measured costs per unit.
double solve_cost(const osscir_ctx* h) {
    const double L = (double)h->L, N = h->g64.n, P = (double)h->P;
    return L * N + 2.1 * L * h->nE + 1.8 * P * h->g64.n_views;
}

// Items per solve and the relative cost of one item, for kernel k (0 projection,
// 1 ray, 2 back-projection, 3 the group sums after a table back-projection)
// under configuration c; `tables`: the back-projection streams footprint tables.
void item_counts(const osscir_ctx* h, int k, const osscir_batch_config& c, bool tables, int* count, double* cost) {
    const int nb = h->g64.n_bins, nv = h->g64.n_views, N = h->g64.n;
    const int G = bp_view_groups(h->P, nv);
    if (k == 0) {
        *count = batch_proj_tiles(nb, nv, c.proj_views);
        *cost = (double)N;                       // pixels per ray ~ image side
    } else if (k == 1) {
        *count = batch_proj_tiles(nb, nv, kFwdThreads / 32);
        *cost = (double)h->nE;                   // energies per ray
    } else if (k == 2 && tables) {
        *count = bt_tiles(N) * G;                // (16 x 16 pixel tile, view group) blocks
        *cost = (double)nv / G;
    } else if (k == 2) {
        *count = batch_bp_items(N, c.bp_tile_x, G);
        *cost = (double)nv / G;                  // views per thread group
    } else {
        *count = tables ? (h->P + 255) / 256 : 0;
        *cost = (double)G;
    }
}

// Work list of kernel k over solves [first, first + n) of the descriptor array.
void build_items(const std::vector<osscir_ctx*>& ctx, int first, int n, int k, const osscir_batch_config& c,
                 bool tables, std::vector<int2>& out) {
    std::vector<int> count(n);
    std::vector<double> cost(n);
    for (int s = 0; s < n; ++s) item_counts(ctx[first + s], k, c, tables, &count[s], &cost[s]);
    const int order = k == 0 ? c.proj_order : (k == 1 ? c.ray_order : c.bp_order);
    out.clear();
    if (n == 0) return;
    if (order == 2) {
        const int most = *std::max_element(count.begin(), count.end());
        for (int t = 0; t < most; ++t)
            for (int s = 0; s < n; ++s)
                if (t < count[s]) out.push_back(make_int2(first + s, t));
        return;
    }
    std::vector<int> solves(n);
    std::iota(solves.begin(), solves.end(), 0);
    if (order == 1)
        std::stable_sort(solves.begin(), solves.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int s : solves)
        for (int t = 0; t < count[s]; ++t) out.push_back(make_int2(first + s, t));
}

// A batch laid out for the device: solves grouped by branch (about equal work
// per branch, largest first to the least loaded), their descriptors, and each
// branch's three work lists, as one byte image.
struct Plan {
    int branches = 1;
    bool tables = false;              // the back-projection streams every solve's tables
    size_t fpb_smem = 0;              // its dynamic shared memory: the largest solve's stages
    std::vector<osscir_ctx*> order;   // descriptor order
    int first[kMaxBranches] = {0, 0, 0, 0}, count[kMaxBranches] = {0, 0, 0, 0};
    size_t off[kMaxBranches][4] = {};
    int n_items[kMaxBranches][4] = {};
    std::vector<char> image;
};

void make_plan(const std::vector<osscir_ctx*>& ctx, const osscir_batch_config& c, Plan& p) {
    const int n = (int)ctx.size();
    p.branches = std::max(1, std::min(c.branches, n));
    std::vector<int> idx(n), owner(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return solve_cost(ctx[a]) > solve_cost(ctx[b]); });
    double load[kMaxBranches] = {0, 0, 0, 0};
    for (int i : idx) {
        int b = 0;
        for (int j = 1; j < p.branches; ++j)
            if (load[j] < load[b]) b = j;
        owner[i] = b;
        load[b] += solve_cost(ctx[i]);
    }
    p.order.clear();
    for (int b = 0; b < p.branches; ++b) {
        p.first[b] = (int)p.order.size();
        for (int i = 0; i < n; ++i)
            if (owner[i] == b) p.order.push_back(ctx[i]);
        p.count[b] = (int)p.order.size() - p.first[b];
    }
    p.tables = all_tables(ctx);
    p.fpb_smem = 0;
    if (p.tables)
        for (const osscir_ctx* h : ctx) p.fpb_smem = std::max(p.fpb_smem, (size_t)fpb_stage_bytes(h->bp_slots));
    size_t bytes = sizeof(SolveDesc) * n;
    std::vector<int2> lists[kMaxBranches][4];
    for (int b = 0; b < p.branches; ++b)
        for (int k = 0; k < 4; ++k) {
            build_items(p.order, p.first[b], p.count[b], k, c, p.tables, lists[b][k]);
            bytes = (bytes + 255) & ~size_t(255);
            p.off[b][k] = bytes;
            p.n_items[b][k] = (int)lists[b][k].size();
            bytes += sizeof(int2) * lists[b][k].size();
        }
    p.image.assign(std::max<size_t>(bytes, 1), 0);
    for (int i = 0; i < n; ++i) {
        const SolveDesc d = make_desc(p.order[i]);
        std::memcpy(p.image.data() + sizeof(SolveDesc) * i, &d, sizeof d);
    }
    for (int b = 0; b < p.branches; ++b)
        for (int k = 0; k < 4; ++k)
            if (!lists[b][k].empty())
                std::memcpy(p.image.data() + p.off[b][k], lists[b][k].data(), sizeof(int2) * lists[b][k].size());
}

inline const SolveDesc* plan_desc(const char* dev) { return reinterpret_cast<const SolveDesc*>(dev); }
inline const int2* plan_items(const Plan& p, const char* dev, int b, int k) {
    return reinterpret_cast<const int2*>(dev + p.off[b][k]);
}

cudaError_t launch_branch_kernel(const Plan& p, const char* dev, int b, int k, const osscir_batch_config& c,
                                 cudaStream_t st) {
    const SolveDesc* d = plan_desc(dev);
    const int2* it = plan_items(p, dev, b, k);
    const int n = p.n_items[b][k];
    if (k == 0) return launch_batch_proj(d, it, n, c.proj_views, c.proj_grid, st);
    if (k == 1) return launch_batch_ray(d, it, n, c.ray_grid, st);
    if (p.tables)
        return launch_batch_fpb(d, it, n, plan_items(p, dev, b, 3), p.n_items[b][3], c.bp_grid, p.fpb_smem, st);
    return launch_batch_bp(d, it, n, c.bp_tile_x, c.bp_grid, st);
}

// Streams and events a batch needs to capture its iteration with branches.
struct Lanes {
    cudaStream_t main = nullptr;
    cudaStream_t aux[kMaxBranches - 1] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    cudaEvent_t fork_at[kMaxBranches - 1] = {nullptr, nullptr, nullptr};
    cudaEvent_t join[kMaxBranches - 1] = {nullptr, nullptr, nullptr};

    cudaError_t create() {
        cudaError_t e = cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking);
        for (int i = 0; i < kMaxBranches - 1 && e == cudaSuccess; ++i)
            e = cudaStreamCreateWithFlags(&aux[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int i = 0; i < kMaxBranches - 1 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork_at[i], cudaEventDisableTiming);
        }
        return e;
    }
    void destroy() {
        if (main) cudaStreamSynchronize(main);
        for (auto& s : aux)
            if (s) cudaStreamDestroy(s);
        if (main) cudaStreamDestroy(main);
        if (fork) cudaEventDestroy(fork);
        for (auto& e : join)
            if (e) cudaEventDestroy(e);
        for (auto& e : fork_at)
            if (e) cudaEventDestroy(e);
        main = nullptr;
    }
};

// `iters` iterations of every solve into the stream being captured on L.main:
// in each iteration branch b launches projection, ray step, back-projection
// and its D_TPL reduction; branches other than 0 fork from L.main and join
// back after their last iteration.  With skew, branch b starts when branch
// b - 1 has finished its first projection, so the branches run different
// kernels side by side.  ev (optional) is recorded around branch 0's kernels
// of its last iteration.
cudaError_t enqueue_plan(const Plan& p, const char* dev, const osscir_batch_config& c, const Lanes& L,
                         const cudaEvent_t* ev, int iters = 1, bool skew = false) {
    cudaError_t e = cudaSuccess;
    auto stream_of = [&](int b) { return b == 0 ? L.main : L.aux[b - 1]; };
    if (p.branches > 1 && !skew) {
        e = cudaEventRecord(L.fork, L.main);
        for (int b = 1; b < p.branches && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(L.aux[b - 1], L.fork, 0);
    }
    for (int b = 0; b < p.branches && e == cudaSuccess; ++b) {
        cudaStream_t st = stream_of(b);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) {
            const bool timed = ev && b == 0 && it == iters - 1;
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                if (timed) e = cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal);
                if (e == cudaSuccess) e = launch_branch_kernel(p, dev, b, k, c, st);
                // the next branch starts after this branch's first projection
                if (e == cudaSuccess && skew && it == 0 && k == 0 && b + 1 < p.branches) {
                    e = cudaEventRecord(L.fork_at[b], st);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream_of(b + 1), L.fork_at[b], 0);
                }
            }
            if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
            if (e == cudaSuccess) e = launch_batch_dtpl(plan_desc(dev) + p.first[b], p.count[b], st);
        }
    }
    for (int b = 1; b < p.branches && e == cudaSuccess; ++b) {
        e = cudaEventRecord(L.join[b - 1], L.aux[b - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(L.main, L.join[b - 1], 0);
    }
    return e;
}

// Capture `iters` iterations as an executable graph.
osscir_status capture_plan(const Plan& p, const char* dev, const osscir_batch_config& c, const Lanes& L,
                           const cudaEvent_t* ev, cudaGraphExec_t* out, int iters = 1, bool skew = false) {
    *out = nullptr;
    CK(cudaStreamBeginCapture(L.main, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enqueue_plan(p, dev, c, L, ev, iters, skew);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(L.main, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return from_cuda(e != cudaSuccess ? e : e2);
    }
    const cudaError_t e3 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return from_cuda(e3);
}

}  // namespace

struct osscir_batch {
    int device = 0;
    int sms = 0;
    std::vector<osscir_ctx*> ctx;
    osscir_batch_config cfg{};
    Plan plan;
    char* dev = nullptr;   // descriptors and work lists
    size_t cap = 0;
    Lanes lanes;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

// Lay the batch out for configuration c and copy it to the device (synchronous).
osscir_status upload(osscir_batch* b, const osscir_batch_config& c) {
    make_plan(b->ctx, c, b->plan);
    const size_t bytes = b->plan.image.size();
    if (bytes > b->cap) {
        if (b->dev) cudaFree(b->dev);
        b->dev = nullptr;
        b->cap = 0;
        CK(cudaMalloc(reinterpret_cast<void**>(&b->dev), bytes));
        b->cap = bytes;
    }
    CK(cudaMemcpy(b->dev, b->plan.image.data(), bytes, cudaMemcpyHostToDevice));
    return OSSCIR_OK;
}

osscir_status rebuild(osscir_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    CKS(upload(b, b->cfg));
    return capture_plan(b->plan, b->dev, b->cfg, b->lanes, b->ev, &b->gexec);
}

void free_batch(osscir_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();   // launches of the batch's graph may still be queued on callers' streams
    b->lanes.destroy();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->dev) cudaFree(b->dev);
    delete b;
}

// ------------------------------------------------------------------ autotuner

// Mean device time (ms) of `reps` runs after one untimed run.  k = 0, 1, 2: that
// kernel alone over the whole batch (one branch); k = 3: a whole iteration graph.
osscir_status time_config(osscir_batch* b, int k, const osscir_batch_config& c, cudaEvent_t t0, cudaEvent_t t1,
                          float* ms) {
    CKS(upload(b, c));
    cudaGraphExec_t gx = nullptr;
    if (k == 3) CKS(capture_plan(b->plan, b->dev, c, b->lanes, nullptr, &gx));
    const int reps = 3;
    cudaStream_t st = b->lanes.main;
    auto run = [&]() { return k == 3 ? cudaGraphLaunch(gx, st) : launch_branch_kernel(b->plan, b->dev, 0, k, c, st); };
    cudaError_t e = run();
    if (e == cudaSuccess) e = cudaEventRecord(t0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run();
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    if (gx) cudaGraphExecDestroy(gx);
    CK(e);
    *ms /= reps;
    return OSSCIR_OK;
}

// Coordinate search per kernel with one branch: grid policy x order at the
// default tile, then the tile shape at the best of those.
osscir_status tune_kernel(osscir_batch* b, int k, int persistent_grid, cudaEvent_t t0, cudaEvent_t t1) {
    osscir_batch_config best = b->cfg;
    float best_ms = 3.0e38f;
    osscir_batch_config c = best;
    int* cgrid = k == 0 ? &c.proj_grid : (k == 1 ? &c.ray_grid : &c.bp_grid);
    int* corder = k == 0 ? &c.proj_order : (k == 1 ? &c.ray_order : &c.bp_order);
    for (int g : {0, persistent_grid})
        for (int o = 0; o < 3; ++o) {
            *cgrid = g;
            *corder = o;
            float ms;
            CKS(time_config(b, k, c, t0, t1, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    if (k == 0 || (k == 2 && !b->plan.tables)) {
        c = best;
        const int views[4] = {1, 2, 4, 8};
        const int txs[5] = {2, 4, 8, 16, 32};
        for (int i = 0; i < (k == 0 ? 4 : 5); ++i) {
            if (k == 0) {
                if (views[i] == best.proj_views) continue;
                c.proj_views = views[i];
                int per_sm = 0;
                CK(batch_resident_ctas(0, 32 * views[i], &per_sm));
                if (c.proj_grid > 0) c.proj_grid = std::max(1, per_sm) * b->sms;
            } else {
                if (txs[i] == best.bp_tile_x) continue;
                c.bp_tile_x = txs[i];
            }
            float ms;
            CKS(time_config(b, k, c, t0, t1, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    b->cfg = best;
    return OSSCIR_OK;
}

// Whole iterations with 1, 2 and 4 branches at the tuned kernel settings.
osscir_status tune_branches(osscir_batch* b, cudaEvent_t t0, cudaEvent_t t1) {
    osscir_batch_config best = b->cfg, c = b->cfg;
    float best_ms = 3.0e38f;
    for (int br = 1; br <= kMaxBranches && br <= (int)b->ctx.size(); br *= 2) {
        c.branches = br;
        float ms;
        CKS(time_config(b, 3, c, t0, t1, &ms));
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    b->cfg = best;
    return OSSCIR_OK;
}

osscir_status autotune(osscir_batch* b) {
    // every solve's state (x_n, xbar_n, y_n) is saved and put back afterwards;
    // g, b, S, the D_TPL partials and D_TPL itself are recomputed by the next iteration
    size_t total = 0;
    for (const osscir_ctx* h : b->ctx) total += sizeof(float4) * (3 * (size_t)h->P + h->L) + sizeof(double);
    char* save = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&save), total));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    osscir_status s = OSSCIR_OK;
    cudaStream_t st = b->lanes.main;
    auto copy_state = [&](bool out) -> cudaError_t {
        size_t off = 0;
        for (osscir_ctx* h : b->ctx) {
            void* buf[4] = {h->x, h->xbar, h->y, h->dtpl_out + 1};
            const size_t sz[4] = {sizeof(float4) * h->P, sizeof(float4) * 2 * h->P, sizeof(float4) * h->L,
                                  sizeof(double)};   // xbar with its column-major copy
            for (int i = 0; i < 4; ++i) {
                const cudaError_t e = out ? cudaMemcpyAsync(save + off, buf[i], sz[i], cudaMemcpyDeviceToDevice, st)
                                          : cudaMemcpyAsync(buf[i], save + off, sz[i], cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return e;
                off += sz[i];
            }
        }
        return cudaStreamSynchronize(st);
    };
    cudaError_t e = copy_state(true);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) s = from_cuda(e);
    make_plan(b->ctx, b->cfg, b->plan);   // whether the back-projection streams tables
    const bool tables = b->plan.tables;
    const int threads[3] = {32 * kDefault.proj_views, kFwdThreads, tables ? kBTThreads : kBpMaxThreads};
    for (int k = 0; k < 3 && s == OSSCIR_OK; ++k) {
        int per_sm = 0;
        e = (k == 2 && tables) ? batch_resident_ctas(3, threads[k], &per_sm, b->plan.fpb_smem)
                               : batch_resident_ctas(k, threads[k], &per_sm);
        if (e != cudaSuccess) {
            s = from_cuda(e);
            break;
        }
        s = tune_kernel(b, k, std::max(1, per_sm) * b->sms, t0, t1);
    }
    if (s == OSSCIR_OK) s = tune_branches(b, t0, t1);
    e = copy_state(false);
    if (s == OSSCIR_OK && e != cudaSuccess) s = from_cuda(e);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(save);
    return s;
}

}  // namespace

// ------------------------------------------------------------------ batch runner (served form)

namespace osscir {

struct BatchRun {
    std::vector<osscir_ctx*> ctx;
    Plan plan;
    char* dev = nullptr;
    size_t cap = 0;
    char* stage[2] = {nullptr, nullptr};   // pinned staging, used alternately
    size_t cap_stage[2] = {0, 0};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    bool stage_used[2] = {false, false};
    int next = 0;
    Lanes lanes;
    bool lanes_ok = false;
    cudaGraphExec_t gexec = nullptr;    // one iteration
    cudaGraphExec_t ground = nullptr;   // kRound iterations, branches skewed
};

constexpr int kRound = 4;

BatchRun* batchrun_new() { return new (std::nothrow) BatchRun(); }

void batchrun_free(BatchRun* r) {
    if (!r) return;
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    if (r->ground) cudaGraphExecDestroy(r->ground);
    r->lanes.destroy();
    cudaDeviceSynchronize();
    if (r->dev) cudaFree(r->dev);
    for (int i = 0; i < 2; ++i) {
        if (r->stage[i]) cudaFreeHost(r->stage[i]);
        if (r->stage_ev[i]) cudaEventDestroy(r->stage_ev[i]);
    }
    delete r;
}

double batch_solve_cost(const osscir_ctx* h) { return solve_cost(h); }

osscir_status batchrun_set(BatchRun* r, const std::vector<osscir_ctx*>& ctx, int branches, cudaStream_t st) {
    r->ctx = ctx;
    if (ctx.empty()) return OSSCIR_OK;
    CKS(build_all_tables(ctx));   // new solves only (each built once, on its own stream)
    if (branches < 1 || branches > kMaxBranches || (branches & (branches - 1))) return OSSCIR_E_INVALID;
    if (!r->lanes_ok) {
        CK(r->lanes.create());
        r->lanes_ok = true;
    }
    osscir_batch_config c = kDefault;
    c.branches = branches;
    make_plan(ctx, c, r->plan);
    const size_t bytes = r->plan.image.size();
    // device image: grown in stream order, so changing the batch never stalls the device
    if (bytes > r->cap) {
        const size_t n = std::max(bytes, 2 * r->cap);
        if (r->dev) CK(cudaFreeAsync(r->dev, st));
        r->dev = nullptr;
        r->cap = 0;
        CK(cudaMallocAsync(reinterpret_cast<void**>(&r->dev), n, st));
        r->cap = n;
    }
    // staging buffer: wait until the copy that last read it has run
    const int b = r->next;
    r->next ^= 1;
    if (!r->stage_ev[b]) CK(cudaEventCreateWithFlags(&r->stage_ev[b], cudaEventDisableTiming));
    if (r->stage_used[b]) CK(cudaEventSynchronize(r->stage_ev[b]));
    if (bytes > r->cap_stage[b]) {
        if (r->stage[b]) CK(cudaFreeHost(r->stage[b]));
        r->stage[b] = nullptr;
        r->cap_stage[b] = 0;
        CK(cudaHostAlloc(reinterpret_cast<void**>(&r->stage[b]), bytes, cudaHostAllocDefault));
        r->cap_stage[b] = bytes;
    }
    std::memcpy(r->stage[b], r->plan.image.data(), bytes);
    CK(cudaMemcpyAsync(r->dev, r->stage[b], bytes, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(r->stage_ev[b], st));
    r->stage_used[b] = true;
    // an executable graph still in flight is released when it completes
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    if (r->ground) cudaGraphExecDestroy(r->ground);
    r->gexec = r->ground = nullptr;
    CKS(capture_plan(r->plan, r->dev, c, r->lanes, nullptr, &r->gexec));
    return capture_plan(r->plan, r->dev, c, r->lanes, nullptr, &r->ground, kRound, r->plan.branches > 1);
}

osscir_status batchrun_step(BatchRun* r, int n_iters, cudaStream_t st) {
    if (r->ctx.empty() || n_iters <= 0) return OSSCIR_OK;
    if (!r->gexec || !r->ground) return OSSCIR_E_INVALID;
    int i = 0;
    for (; i + kRound <= n_iters; i += kRound) CK(cudaGraphLaunch(r->ground, st));
    for (; i < n_iters; ++i) CK(cudaGraphLaunch(r->gexec, st));
    for (osscir_ctx* h : r->ctx) h->iter += n_iters;
    return OSSCIR_OK;
}

}  // namespace osscir

extern "C" {

osscir_status osscir_batch_create(const osscir_t* solves, int n, int autotune_flag, osscir_batch_t* out) {
    if (!out) return OSSCIR_E_INVALID;
    *out = nullptr;
    if (!solves || n < 1 || n > 4096 || (autotune_flag != 0 && autotune_flag != 1)) return OSSCIR_E_INVALID;
    std::vector<osscir_ctx*> v(solves, solves + n);
    for (osscir_ctx* h : v)
        if (!h) return OSSCIR_E_INVALID;
    std::vector<osscir_ctx*> sorted = v;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return OSSCIR_E_INVALID;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    for (osscir_ctx* h : v)   // nested solves (inner > 1) step on their own; the batched kernels take four windows
        if (h->device != dev || h->inner > 1 || h->nw != 4) return OSSCIR_E_INVALID;
    // work already queued on the solves (on any stream) must be done before the
    // autotuner saves their state
    CK(cudaDeviceSynchronize());
    CKS(build_all_tables(v));

    osscir_batch* b = new (std::nothrow) osscir_batch();
    if (!b) return OSSCIR_E_NOMEM;
    b->device = dev;
    b->ctx = std::move(v);
    b->cfg = kDefault;
    osscir_status s = from_cuda(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    if (s == OSSCIR_OK) s = from_cuda(b->lanes.create());
    for (int i = 0; i < 4 && s == OSSCIR_OK; ++i) s = from_cuda(cudaEventCreate(&b->ev[i]));
    if (s == OSSCIR_OK && autotune_flag) s = autotune(b);
    if (s == OSSCIR_OK) s = rebuild(b);
    if (s != OSSCIR_OK) {
        free_batch(b);
        return s;
    }
    *out = b;
    return OSSCIR_OK;
}

osscir_status osscir_batch_destroy(osscir_batch_t b) {
    free_batch(b);
    return OSSCIR_OK;
}

osscir_status osscir_batch_step(osscir_batch_t b, int n_iters, void* stream) {
    if (!b || n_iters < 0) return OSSCIR_E_INVALID;
    for (int i = 0; i < n_iters; ++i) CK(cudaGraphLaunch(b->gexec, as_stream(stream)));
    for (osscir_ctx* h : b->ctx) h->iter += n_iters;
    return OSSCIR_OK;
}

osscir_status osscir_batch_get_config(osscir_batch_t b, osscir_batch_config* out) {
    if (!b || !out) return OSSCIR_E_INVALID;
    *out = b->cfg;
    return OSSCIR_OK;
}

osscir_status osscir_batch_set_config(osscir_batch_t b, const osscir_batch_config* cfg) {
    if (!b || !cfg || !valid_config(*cfg)) return OSSCIR_E_INVALID;
    CK(cudaDeviceSynchronize());   // no launch of the old work lists may still be in flight
    b->cfg = *cfg;
    return rebuild(b);
}

osscir_status osscir_batch_last_kernel_ms(osscir_batch_t b, float* ms, void* stream) {
    if (!b || !ms) return OSSCIR_E_INVALID;
    CK(cudaStreamSynchronize(as_stream(stream)));
    for (int k = 0; k < 3; ++k) CK(cudaEventElapsedTime(ms + k, b->ev[k], b->ev[k + 1]));
    return OSSCIR_OK;
}

}  // extern "C"
