// C-ABI of the library (include/osscir.h): context creation, validation,
// per-geometry tables, and the per-iteration CUDA graph.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "osscir_ctx.h"

using namespace osscir;

namespace {

thread_local size_t g_dalloc_bytes_sink = 0;
thread_local size_t* g_dalloc_bytes = &g_dalloc_bytes_sink;

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    const size_t bytes = sizeof(T) * (count ? count : 1);
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e == cudaSuccess) *g_dalloc_bytes += bytes;
    return e;
}

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

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void free_ctx(osscir_ctx* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->gexec_in) cudaGraphExecDestroy(h->gexec_in);
    if (h->graph_in) cudaGraphDestroy(h->graph_in);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    void* ptrs[] = {h->rec, h->r64, h->views, h->chord, h->exc_off, h->exc_ent, h->s4, h->N4, h->mu,
                    h->g, h->c, h->y, h->x, h->xbar, h->dtpl_part, h->dtpl_out, h->model};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete h;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

osscir_status validate(const osscir_geometry* g, const osscir_spectra* sp, const float* mu,
                       const osscir_params* pa) {
    if (!g || !sp || !mu || !pa || !sp->s || !sp->N) return OSSCIR_E_INVALID;
    if (g->n < 1 || g->n > 8192 || g->n_views < 1 || g->n_bins < 1) return OSSCIR_E_INVALID;
    if ((long long)g->n_views * g->n_bins > (1LL << 30)) return OSSCIR_E_INVALID;
    if (!finite_pos(g->pixel_mm) || !finite_pos(g->bin_mm) || !finite_pos(g->sid_mm) || !finite_pos(g->sdd_mm))
        return OSSCIR_E_INVALID;
    if (!std::isfinite(g->arc_deg) || !std::isfinite(g->start_deg)) return OSSCIR_E_INVALID;
    const double rc = g->n * g->pixel_mm * std::sqrt(2.0) / 2.0;
    if (!(g->sid_mm > rc) || !(g->sdd_mm > g->sid_mm)) return OSSCIR_E_INVALID;
    if (sp->n_energies < 1 || sp->n_energies > 256) return OSSCIR_E_INVALID;
    const int nE = sp->n_energies;
    for (int b = 0; b < g->n_bins; ++b) {
        for (int w = 0; w < 4; ++w) {
            double sum = 0.0;
            for (int i = 0; i < nE; ++i) {
                const float v = sp->s[((size_t)b * nE + i) * 4 + w];
                if (!std::isfinite(v) || v < 0.f) return OSSCIR_E_INVALID;
                sum += v;
            }
            if (std::fabs(sum - 1.0) > 1e-4) return OSSCIR_E_INVALID;
            if (!finite_pos(sp->N[(size_t)b * 4 + w])) return OSSCIR_E_INVALID;
        }
    }
    for (int i = 0; i < 3 * nE; ++i)   // a transformed basis (mu-PC) may have negative curves
        if (!std::isfinite(mu[i])) return OSSCIR_E_INVALID;
    if (!finite_pos(pa->lambda) || !(pa->lambda < 3.0e38)) return OSSCIR_E_INVALID;
    if (pa->model != 0 && pa->model != 1) return OSSCIR_E_INVALID;
    if (pa->spc != 0 && pa->spc != 1) return OSSCIR_E_INVALID;
    if (pa->counts_model != 0 && pa->counts_model != 1) return OSSCIR_E_INVALID;
    if (pa->inner < 0 || pa->inner > 1000000) return OSSCIR_E_INVALID;
    if (pa->use_box)
        for (int m = 0; m < 3; ++m)
            if (std::isnan(pa->lo[m]) || std::isnan(pa->hi[m]) || !(pa->lo[m] <= pa->hi[m]) ||
                pa->lo[m] == INFINITY || pa->hi[m] == -INFINITY)
                return OSSCIR_E_INVALID;
    return OSSCIR_OK;
}

osscir_status build(osscir_ctx* h, const osscir_geometry* g, const osscir_spectra* sp, const float* mu,
                    const osscir_params* pa) {
    g_dalloc_bytes = &h->bytes;
    CK(cudaGetDevice(&h->device));
    const int n = g->n;
    h->P = n * n;
    h->L = g->n_views * g->n_bins;
    h->nE = sp->n_energies;
    GeomD& G = h->g64;
    G.n = n;
    G.h = g->pixel_mm;
    G.x0 = -0.5 * n * g->pixel_mm;
    G.n_views = g->n_views;
    G.n_bins = g->n_bins;
    G.arc_deg = g->arc_deg;
    G.start_deg = g->start_deg;
    G.bin_mm = g->bin_mm;
    G.sid = g->sid_mm;
    G.sdd = g->sdd_mm;
    G.thr = 1e-9 * g->pixel_mm;
    const double r_img = n * g->pixel_mm * std::sqrt(2.0) / 2.0;
    GeomC& C = h->gc;
    C.grid = GridF{n, (float)g->pixel_mm, (float)G.x0};
    C.n_views = g->n_views;
    C.n_bins = g->n_bins;
    C.sid = (float)g->sid_mm;
    C.scale = (float)(g->sdd_mm / g->bin_mm);
    C.mid = (float)(0.5 * (g->n_bins - 1));
    C.margin_mm = (float)(1e-5 * r_img + 1e-3 * g->pixel_mm);
    C.margin_bins = 0.01f;
    h->params.lambda = (float)pa->lambda;
    h->params.model = pa->model;
    h->params.spc = pa->spc;
    h->exp_model = pa->counts_model;
    h->inner = pa->inner > 1 ? pa->inner : 1;
    h->params.use_box = pa->use_box;
    for (int m = 0; m < 3; ++m) {
        h->params.lo[m] = pa->lo[m];
        h->params.hi[m] = pa->hi[m];
    }

    const int L = h->L, P = h->P, nE = h->nE;
    h->n_part = dtpl_partials(g->n_bins, g->n_views);
    CK(dalloc(&h->rec, 2 * (size_t)L));   // weight halves, then step halves
    CK(dalloc(&h->r64, L));
    CK(dalloc(&h->views, g->n_views));
    CK(dalloc(&h->chord, L));
    CK(dalloc(&h->exc_off, L + 1));
    CK(dalloc(&h->s4, (size_t)nE * g->n_bins));
    CK(dalloc(&h->N4, g->n_bins));
    CK(dalloc(&h->mu, 3 * nE));
    CK(dalloc(&h->g, L));
    CK(dalloc(&h->c, L));
    CK(dalloc(&h->y, L));
    CK(dalloc(&h->x, P));
    CK(dalloc(&h->xbar, P));
    CK(dalloc(&h->dtpl_part, h->n_part));
    CK(dalloc(&h->dtpl_out, 2));
    if (h->inner > 1) CK(dalloc(&h->model, (size_t)kModelStride * L));
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : h->ev) CK(cudaEventCreate(&e));
    CK(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
    cudaStream_t st = h->cap_stream;

    // spectral tables: s reordered to [nE][n_bins] float4 so consecutive rays read consecutive entries
    {
        std::vector<float> s4((size_t)nE * g->n_bins * 4);
        for (int b = 0; b < g->n_bins; ++b)
            for (int i = 0; i < nE; ++i)
                for (int w = 0; w < 4; ++w)
                    s4[((size_t)i * g->n_bins + b) * 4 + w] = sp->s[((size_t)b * nE + i) * 4 + w];
        CK(cudaMemcpy(h->s4, s4.data(), s4.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->N4, sp->N, sizeof(float) * 4 * g->n_bins, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->mu, mu, sizeof(float) * 3 * nE, cudaMemcpyHostToDevice));
    }
    // per-ray records, then the footprint pairs decided in FP64
    CK(launch_ray_setup(G, r_img, h->rec, h->r64, h->views, st));
    CK(launch_exc_pass(C, G, h->rec, h->r64, h->exc_off, nullptr, nullptr, st));
    std::vector<int> cnt(L + 1, 0);
    CK(cudaMemcpyAsync(cnt.data(), h->exc_off, sizeof(int) * L, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    long long run = 0;
    for (int l = 0; l < L; ++l) {
        const int c0 = cnt[l];
        cnt[l] = (int)run;
        run += c0;
    }
    if (run > (1LL << 31) - 1) return OSSCIR_E_NOMEM;
    cnt[L] = (int)run;
    h->exc_n = (int)run;
    CK(cudaMemcpyAsync(h->exc_off, cnt.data(), sizeof(int) * (L + 1), cudaMemcpyHostToDevice, st));
    CK(dalloc(&h->exc_ent, run));
    CK(launch_exc_pass(C, G, h->rec, h->r64, nullptr, h->exc_off, h->exc_ent, st));
    CK(launch_chord(C, h->exc(), h->rec, h->chord, st));
    CK(cudaMemsetAsync(h->c, 0, sizeof(float4) * L, st));
    CK(cudaMemsetAsync(h->y, 0, sizeof(float4) * L, st));
    CK(cudaMemsetAsync(h->x, 0, sizeof(float4) * P, st));
    CK(cudaMemsetAsync(h->xbar, 0, sizeof(float4) * P, st));
    CK(cudaMemsetAsync(h->dtpl_out, 0, sizeof(double) * 2, st));
    CK(cudaStreamSynchronize(st));
    return OSSCIR_OK;
}

// One MOCCA iteration as launches on a stream (captured into a graph once).
// One iteration on st: projection, per-ray step, back-projection; the D_TPL
// reduction needs only the per-ray partials, so it runs on a side branch
// beside the back-projection and joins before the iteration ends.  For a
// nested solve the outer iteration also keeps the rays' models, and an inner
// one (inner_step) replaces the per-ray step by the dual step on them.
cudaError_t enqueue_iteration(osscir_ctx* h, cudaStream_t st, bool inner_step) {
    cudaError_t e = cudaEventRecordWithFlags(h->ev[0], st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    e = launch_mocca_proj(h->gc, h->exc(), h->rec, h->solve(), st);
    if (e != cudaSuccess) return e;
    e = cudaEventRecordWithFlags(h->ev[1], st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    if (inner_step) {
        e = launch_mocca_ray_inner(h->gc, h->rec, h->solve(), st);
        if (e != cudaSuccess) return e;
        e = cudaEventRecordWithFlags(h->ev[2], st, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
        e = launch_mocca_bp(h->gc, h->exc(), h->rec, h->views, h->params, h->solve(), st);
        if (e != cudaSuccess) return e;
        return cudaEventRecordWithFlags(h->ev[3], st, cudaEventRecordExternal);
    }
    e = h->inner > 1 ? launch_mocca_ray_keep(h->gc, h->rec, h->spec(), h->params, h->solve(), st)
                     : launch_mocca_ray(h->gc, h->rec, h->spec(), h->params, h->solve(), st);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(h->fork, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamWaitEvent(h->side_stream, h->fork, 0);
    if (e != cudaSuccess) return e;
    e = launch_dtpl_reduce(h->dtpl_part, h->n_part, h->dtpl_out + 1, h->side_stream);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(h->join, h->side_stream);
    if (e != cudaSuccess) return e;
    e = cudaEventRecordWithFlags(h->ev[2], st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    e = launch_mocca_bp(h->gc, h->exc(), h->rec, h->views, h->params, h->solve(), st);
    if (e != cudaSuccess) return e;
    e = cudaEventRecordWithFlags(h->ev[3], st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(st, h->join, 0);
}

osscir_status capture(osscir_ctx* h, bool inner_step, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enqueue_iteration(h, h->cap_stream, inner_step);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return from_cuda(e);
    }
    CK(e2);
    *graph = g;
    CK(cudaGraphInstantiate(exec, g, 0));
    return OSSCIR_OK;
}

osscir_status ensure_graph(osscir_ctx* h) {
    if (!h->gexec) {
        const osscir_status s = capture(h, false, &h->graph, &h->gexec);
        if (s != OSSCIR_OK) return s;
    }
    if (h->inner > 1 && !h->gexec_in) return capture(h, true, &h->graph_in, &h->gexec_in);
    return OSSCIR_OK;
}

}  // namespace

namespace osscir {

osscir_status ctx_create(const osscir_geometry* geom, const osscir_spectra* spectra, const float* mu,
                         const osscir_params* params, osscir_ctx** out) {
    *out = nullptr;
    const osscir_status v = validate(geom, spectra, mu, params);
    if (v != OSSCIR_OK) return v;
    osscir_ctx* h = new (std::nothrow) osscir_ctx();
    if (!h) return OSSCIR_E_NOMEM;
    const osscir_status s = build(h, geom, spectra, mu, params);
    g_dalloc_bytes = &g_dalloc_bytes_sink;
    if (s != OSSCIR_OK) {
        free_ctx(h);
        return s;
    }
    *out = h;
    return OSSCIR_OK;
}

void ctx_destroy(osscir_ctx* h) { free_ctx(h); }

osscir_status ctx_validate(const osscir_geometry* geom, const osscir_spectra* spectra, const float* mu,
                           const osscir_params* params) {
    return validate(geom, spectra, mu, params);
}

osscir_status ctx_ensure_graph(osscir_ctx* h) { return ensure_graph(h); }

}  // namespace osscir

extern "C" {

const char* osscir_status_string(osscir_status s) {
    switch (s) {
        case OSSCIR_OK: return "ok";
        case OSSCIR_E_INVALID: return "invalid argument";
        case OSSCIR_E_NOMEM: return "out of memory";
        case OSSCIR_E_CUDA: return "CUDA error";
        case OSSCIR_E_TIMEOUT: return "timeout";
        case OSSCIR_E_DIVERGED: return "diverged";
        case OSSCIR_E_BUSY: return "busy";
        case OSSCIR_E_NOTFOUND: return "not found";
        default: return "unknown status";
    }
}

osscir_status osscir_create(const osscir_geometry* geom, const osscir_spectra* spectra, const float* mu,
                            const osscir_params* params, osscir_t* out) {
    if (!out) return OSSCIR_E_INVALID;
    return osscir::ctx_create(geom, spectra, mu, params, out);
}

osscir_status osscir_destroy(osscir_t h) {
    free_ctx(h);
    return OSSCIR_OK;
}

osscir_status osscir_info(osscir_t h, int* n_pixels, int* n_rays, int* n_fp64_pairs) {
    if (!h) return OSSCIR_E_INVALID;
    if (n_pixels) *n_pixels = h->P;
    if (n_rays) *n_rays = h->L;
    if (n_fp64_pairs) *n_fp64_pairs = h->exc_n;
    return OSSCIR_OK;
}

osscir_status osscir_forward(osscir_t h, const float* x, float* g, void* stream) {
    if (!h || !x || !g) return OSSCIR_E_INVALID;
    CK(launch_forward4(h->gc, h->exc(), h->rec, reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(g),
                       as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_backproject(osscir_t h, const float* rf, float* img, void* stream) {
    if (!h || !rf || !img) return OSSCIR_E_INVALID;
    CK(launch_backproject4(h->gc, h->exc(), h->rec, h->views, reinterpret_cast<const float4*>(rf),
                           reinterpret_cast<float4*>(img), as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_simulate(osscir_t h, const float* f, float* chat, void* stream) {
    if (!h || !f || !chat) return OSSCIR_E_INVALID;
    CK(launch_counts(h->gc, h->exc(), h->rec, h->spec(), reinterpret_cast<const float4*>(f),
                     reinterpret_cast<float4*>(chat), nullptr, nullptr, as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_set_counts(osscir_t h, const float* c, void* stream) {
    if (!h || !c) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(h->c, c, sizeof(float4) * h->L, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(h->y, 0, sizeof(float4) * h->L, st));
    CK(cudaMemsetAsync(h->x, 0, sizeof(float4) * h->P, st));
    CK(cudaMemsetAsync(h->xbar, 0, sizeof(float4) * h->P, st));
    h->iter = 0;
    h->phase = 0;
    return OSSCIR_OK;
}

osscir_status osscir_mocca_step(osscir_t h, int n_iters, void* stream) {
    if (!h || n_iters < 0) return OSSCIR_E_INVALID;
    if (n_iters == 0) return OSSCIR_OK;
    const osscir_status s = ensure_graph(h);
    if (s != OSSCIR_OK) return s;
    for (int i = 0; i < n_iters; ++i) {
        CK(cudaGraphLaunch(h->phase == 0 ? h->gexec : h->gexec_in, as_stream(stream)));
        h->iter += 1;
        h->phase = (h->phase + 1) % h->inner;
    }
    return OSSCIR_OK;
}

osscir_status osscir_reconstruct(osscir_t h, const float* c_host, int n_iters, float* maps_out_host,
                                 void* stream) {
    if (!h || !c_host || !maps_out_host || n_iters < 0) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(h->c, c_host, sizeof(float4) * h->L, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->y, 0, sizeof(float4) * h->L, st));
    CK(cudaMemsetAsync(h->x, 0, sizeof(float4) * h->P, st));
    CK(cudaMemsetAsync(h->xbar, 0, sizeof(float4) * h->P, st));
    h->iter = 0;
    h->phase = 0;
    const osscir_status s = osscir_mocca_step(h, n_iters, stream);
    if (s != OSSCIR_OK) return s;
    CK(cudaMemcpyAsync(maps_out_host, h->x, sizeof(float4) * h->P, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return OSSCIR_OK;
}

osscir_status osscir_last_kernel_ms(osscir_t h, float* ms, void* stream) {
    if (!h || !ms) return OSSCIR_E_INVALID;
    if (!h->gexec) return OSSCIR_E_INVALID;
    CK(cudaStreamSynchronize(as_stream(stream)));
    for (int k = 0; k < 3; ++k) CK(cudaEventElapsedTime(ms + k, h->ev[k], h->ev[k + 1]));
    return OSSCIR_OK;
}

osscir_status osscir_get_maps(osscir_t h, float* x_out, void* stream) {
    if (!h || !x_out) return OSSCIR_E_INVALID;
    CK(cudaMemcpyAsync(x_out, h->x, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_get_state(osscir_t h, float* x, float* xbar, float* y, int* iter, void* stream) {
    if (!h || !x || !xbar || !y) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(x, h->x, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(xbar, h->xbar, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(y, h->y, sizeof(float4) * h->L, cudaMemcpyDeviceToDevice, st));
    if (iter) *iter = h->iter;
    return OSSCIR_OK;
}

osscir_status osscir_set_state(osscir_t h, const float* x, const float* xbar, const float* y, int iter,
                               void* stream) {
    if (!h || !x || !xbar || !y || iter < 0) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(h->x, x, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->xbar, xbar, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->y, y, sizeof(float4) * h->L, cudaMemcpyDeviceToDevice, st));
    h->iter = iter;
    h->phase = 0;
    return OSSCIR_OK;
}

osscir_status osscir_dtpl(osscir_t h, int which, double* out, void* stream) {
    if (!h || !out || (which != 0 && which != 1)) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    if (which == 0) {
        CK(launch_counts(h->gc, h->exc(), h->rec, h->spec(), h->x, nullptr, h->c, h->dtpl_part, st));
        CK(launch_dtpl_reduce(h->dtpl_part, h->n_part, h->dtpl_out, st));
    }
    CK(cudaMemcpyAsync(out, h->dtpl_out + which, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!std::isfinite(*out)) return OSSCIR_E_DIVERGED;
    return OSSCIR_OK;
}

osscir_status osscir_footprint_rays(osscir_t h, int l0, int n, int cap, int* cnt, int* idx, float* wt,
                                    void* stream) {
    if (!h || !cnt || (cap > 0 && (!idx || !wt)) || l0 < 0 || n < 0 || cap < 0 || l0 + n > h->L)
        return OSSCIR_E_INVALID;
    if (n == 0) return OSSCIR_OK;
    CK(launch_footprint_rays(h->gc, h->exc(), h->rec, l0, n, cap, cnt, idx, wt, as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_footprint_pixels(osscir_t h, int k0, int n, int cap, int* cnt, int* idx, float* wt,
                                      void* stream) {
    if (!h || !cnt || (cap > 0 && (!idx || !wt)) || k0 < 0 || n < 0 || cap < 0 || k0 + n > h->P)
        return OSSCIR_E_INVALID;
    if (n == 0) return OSSCIR_OK;
    CK(launch_footprint_pixels(h->gc, h->exc(), h->rec, h->views, k0, n, cap, cnt, idx, wt, as_stream(stream)));
    return OSSCIR_OK;
}

}  // extern "C"
