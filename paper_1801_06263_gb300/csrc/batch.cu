// Batched form of the C-ABI (include/osscir.h): many independent solves
// advanced by one launch per kernel per MOCCA step, over work lists of
// (solve, tile) items, captured once as a CUDA graph; plus the autotuner that
// picks tile shapes, grid policy and work-list order by timing them on the
// batch itself.
#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "osscir_ctx.h"

using namespace osscir;

struct osscir_batch {
    int device = 0;
    int sms = 0;
    std::vector<osscir_ctx*> ctx;
    osscir_batch_config cfg{};
    SolveDesc* desc = nullptr;   // device [n]
    int2* items[3] = {nullptr, nullptr, nullptr};   // projection, ray, back-projection work lists
    int n_items[3] = {0, 0, 0};
    size_t cap_items[3] = {0, 0, 0};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

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

constexpr osscir_batch_config kDefault = {4, 0, 0, 0, 0, 8, 0, 0};

bool valid_config(const osscir_batch_config& c) {
    const auto pow2_in = [](int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; };
    const auto grid_ok = [](int g) { return g >= 0 && g <= (1 << 20); };
    const auto order_ok = [](int o) { return o >= 0 && o <= 2; };
    return pow2_in(c.proj_views, 1, 8) && pow2_in(c.bp_tile_x, 4, 32) && grid_ok(c.proj_grid) &&
           grid_ok(c.ray_grid) && grid_ok(c.bp_grid) && order_ok(c.proj_order) && order_ok(c.ray_order) &&
           order_ok(c.bp_order);
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
    return d;
}

// Items per solve and the relative cost of one item, for kernel k (0 projection,
// 1 ray, 2 back-projection) under configuration c.
void item_counts(const osscir_batch* b, int k, const osscir_batch_config& c, std::vector<int>& count,
                 std::vector<double>& cost) {
    const int n = (int)b->ctx.size();
    count.assign(n, 0);
    cost.assign(n, 0.0);
    for (int s = 0; s < n; ++s) {
        const osscir_ctx* h = b->ctx[s];
        const int nb = h->g64.n_bins, nv = h->g64.n_views, N = h->g64.n;
        if (k == 0) {
            count[s] = batch_proj_tiles(nb, nv, c.proj_views);
            cost[s] = (double)N;                         // pixels per ray ~ image side
        } else if (k == 1) {
            count[s] = batch_proj_tiles(nb, nv, kFwdThreads / 32);
            cost[s] = (double)h->nE;                     // energy passes per ray
        } else {
            const int G = bp_view_groups(h->P, nv);
            count[s] = batch_bp_items(N, c.bp_tile_x, G);
            cost[s] = (double)nv / G;                    // views per thread group
        }
    }
}

void build_items(const osscir_batch* b, int k, const osscir_batch_config& c, std::vector<int2>& out) {
    std::vector<int> count;
    std::vector<double> cost;
    item_counts(b, k, c, count, cost);
    const int order = k == 0 ? c.proj_order : (k == 1 ? c.ray_order : c.bp_order);
    const int n = (int)count.size();
    std::vector<int> solves(n);
    std::iota(solves.begin(), solves.end(), 0);
    out.clear();
    if (order == 1)
        std::stable_sort(solves.begin(), solves.end(), [&](int a, int bb) { return cost[a] > cost[bb]; });
    if (order == 2) {
        const int most = *std::max_element(count.begin(), count.end());
        for (int t = 0; t < most; ++t)
            for (int s = 0; s < n; ++s)
                if (t < count[s]) out.push_back(make_int2(s, t));
        return;
    }
    for (int s : solves)
        for (int t = 0; t < count[s]; ++t) out.push_back(make_int2(s, t));
}

osscir_status upload_items(osscir_batch* b, int k, const std::vector<int2>& v) {
    if (v.size() > (size_t)0x7fffffff) return OSSCIR_E_INVALID;
    if (v.size() > b->cap_items[k]) {
        if (b->items[k]) cudaFree(b->items[k]);
        b->items[k] = nullptr;
        b->cap_items[k] = 0;
        CK(cudaMalloc(reinterpret_cast<void**>(&b->items[k]), sizeof(int2) * v.size()));
        b->cap_items[k] = v.size();
    }
    if (!v.empty()) CK(cudaMemcpy(b->items[k], v.data(), sizeof(int2) * v.size(), cudaMemcpyHostToDevice));
    b->n_items[k] = (int)v.size();
    return OSSCIR_OK;
}

osscir_status build_all_items(osscir_batch* b) {
    std::vector<int2> v;
    for (int k = 0; k < 3; ++k) {
        build_items(b, k, b->cfg, v);
        CKS(upload_items(b, k, v));
    }
    return OSSCIR_OK;
}

cudaError_t launch_kernel(const osscir_batch* b, int k, const osscir_batch_config& c, cudaStream_t st) {
    if (k == 0) return launch_batch_proj(b->desc, b->items[0], b->n_items[0], c.proj_views, c.proj_grid, st);
    if (k == 1) return launch_batch_ray(b->desc, b->items[1], b->n_items[1], c.ray_grid, st);
    return launch_batch_bp(b->desc, b->items[2], b->n_items[2], c.bp_tile_x, c.bp_grid, st);
}

cudaError_t enqueue_iteration(const osscir_batch* b, cudaStream_t st) {
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaEventRecordWithFlags(b->ev[k], st, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
        e = launch_kernel(b, k, b->cfg, st);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = cudaEventRecordWithFlags(b->ev[3], st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    return launch_batch_dtpl(b->desc, (int)b->ctx.size(), st);
}

void drop_graph(osscir_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

osscir_status capture(osscir_batch* b) {
    drop_graph(b);
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enqueue_iteration(b, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return from_cuda(e);
    }
    CK(e2);
    b->graph = g;
    CK(cudaGraphInstantiate(&b->gexec, g, 0));
    return OSSCIR_OK;
}

void free_batch(osscir_batch* b) {
    if (!b) return;
    if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
    drop_graph(b);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    for (auto& p : b->items)
        if (p) cudaFree(p);
    if (b->desc) cudaFree(b->desc);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

// ------------------------------------------------------------------ autotuner

// Mean device time (ms) of `reps` launches of kernel k under configuration c,
// after one untimed launch, on the batch's own stream.
osscir_status time_kernel(osscir_batch* b, int k, const osscir_batch_config& c, cudaEvent_t t0, cudaEvent_t t1,
                          float* ms) {
    std::vector<int2> v;
    build_items(b, k, c, v);
    CKS(upload_items(b, k, v));
    const int reps = 3;
    CK(launch_kernel(b, k, c, b->cap_stream));
    CK(cudaEventRecord(t0, b->cap_stream));
    for (int r = 0; r < reps; ++r) CK(launch_kernel(b, k, c, b->cap_stream));
    CK(cudaEventRecord(t1, b->cap_stream));
    CK(cudaEventSynchronize(t1));
    CK(cudaEventElapsedTime(ms, t0, t1));
    *ms /= reps;
    return OSSCIR_OK;
}

// Coordinate search per kernel: grid policy x order at the default tile, then
// the tile shape at the best of those.
osscir_status tune_kernel(osscir_batch* b, int k, int persistent_grid, cudaEvent_t t0, cudaEvent_t t1) {
    osscir_batch_config best = b->cfg;
    float best_ms = 3.0e38f;
    int* grid = k == 0 ? &best.proj_grid : (k == 1 ? &best.ray_grid : &best.bp_grid);
    int* order = k == 0 ? &best.proj_order : (k == 1 ? &best.ray_order : &best.bp_order);
    osscir_batch_config c = best;
    int* cgrid = k == 0 ? &c.proj_grid : (k == 1 ? &c.ray_grid : &c.bp_grid);
    int* corder = k == 0 ? &c.proj_order : (k == 1 ? &c.ray_order : &c.bp_order);
    for (int g : {0, persistent_grid})
        for (int o = 0; o < 3; ++o) {
            *cgrid = g;
            *corder = o;
            float ms;
            CKS(time_kernel(b, k, c, t0, t1, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                *grid = g;
                *order = o;
            }
        }
    if (k != 1) {
        c = best;
        const int tiles[4] = {1, 2, 4, 8};
        const int txs[4] = {4, 8, 16, 32};
        for (int i = 0; i < 4; ++i) {
            if (k == 0) {
                if (tiles[i] == best.proj_views) continue;
                c.proj_views = tiles[i];
                int per_sm = 0;
                CK(batch_resident_ctas(0, 32 * tiles[i], &per_sm));
                if (c.proj_grid > 0) c.proj_grid = std::max(1, per_sm) * b->sms;
            } else {
                if (txs[i] == best.bp_tile_x) continue;
                c.bp_tile_x = txs[i];
            }
            float ms;
            CKS(time_kernel(b, k, c, t0, t1, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    b->cfg = best;
    return OSSCIR_OK;
}

osscir_status autotune(osscir_batch* b) {
    // every solve's state (x_n, xbar_n, y_n) is saved and put back afterwards;
    // g, b, S and the D_TPL partials are recomputed by the next iteration
    size_t total = 0;
    for (const osscir_ctx* h : b->ctx) total += sizeof(float4) * (2 * (size_t)h->P + h->L);
    char* save = nullptr;
    CK(cudaMalloc(reinterpret_cast<void**>(&save), total));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    osscir_status s = OSSCIR_OK;
    auto copy_state = [&](bool out) -> cudaError_t {
        size_t off = 0;
        for (osscir_ctx* h : b->ctx) {
            void* buf[3] = {h->x, h->xbar, h->y};
            const size_t sz[3] = {sizeof(float4) * h->P, sizeof(float4) * h->P, sizeof(float4) * h->L};
            for (int i = 0; i < 3; ++i) {
                const cudaError_t e = out ? cudaMemcpyAsync(save + off, buf[i], sz[i], cudaMemcpyDeviceToDevice,
                                                            b->cap_stream)
                                          : cudaMemcpyAsync(buf[i], save + off, sz[i], cudaMemcpyDeviceToDevice,
                                                            b->cap_stream);
                if (e != cudaSuccess) return e;
                off += sz[i];
            }
        }
        return cudaStreamSynchronize(b->cap_stream);
    };
    cudaError_t e = copy_state(true);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) s = from_cuda(e);
    const int threads[3] = {32 * kDefault.proj_views, kFwdThreads, kBpMaxThreads};
    for (int k = 0; k < 3 && s == OSSCIR_OK; ++k) {
        int per_sm = 0;
        e = batch_resident_ctas(k, threads[k], &per_sm);
        if (e != cudaSuccess) {
            s = from_cuda(e);
            break;
        }
        s = tune_kernel(b, k, std::max(1, per_sm) * b->sms, t0, t1);
    }
    e = copy_state(false);
    if (s == OSSCIR_OK && e != cudaSuccess) s = from_cuda(e);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(save);
    return s;
}

}  // namespace

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
    for (osscir_ctx* h : v)
        if (h->device != dev) return OSSCIR_E_INVALID;

    osscir_batch* b = new (std::nothrow) osscir_batch();
    if (!b) return OSSCIR_E_NOMEM;
    b->device = dev;
    b->ctx = std::move(v);
    b->cfg = kDefault;
    auto fail = [&](osscir_status s) {
        free_batch(b);
        return s;
    };
    auto ck = [&](cudaError_t e) { return from_cuda(e); };
    osscir_status s = ck(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    if (s == OSSCIR_OK) s = ck(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 4 && s == OSSCIR_OK; ++i) s = ck(cudaEventCreate(&b->ev[i]));
    if (s == OSSCIR_OK) s = ck(cudaMalloc(reinterpret_cast<void**>(&b->desc), sizeof(SolveDesc) * n));
    if (s == OSSCIR_OK) {
        std::vector<SolveDesc> d(n);
        for (int i = 0; i < n; ++i) d[i] = make_desc(b->ctx[i]);
        s = ck(cudaMemcpy(b->desc, d.data(), sizeof(SolveDesc) * n, cudaMemcpyHostToDevice));
    }
    if (s == OSSCIR_OK && autotune_flag) s = autotune(b);
    if (s == OSSCIR_OK) s = build_all_items(b);
    if (s == OSSCIR_OK) s = capture(b);
    if (s != OSSCIR_OK) return fail(s);
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
    CKS(build_all_items(b));
    return capture(b);
}

osscir_status osscir_batch_last_kernel_ms(osscir_batch_t b, float* ms, void* stream) {
    if (!b || !ms) return OSSCIR_E_INVALID;
    CK(cudaStreamSynchronize(as_stream(stream)));
    for (int k = 0; k < 3; ++k) CK(cudaEventElapsedTime(ms + k, b->ev[k], b->ev[k + 1]));
    return OSSCIR_OK;
}

}  // extern "C"
