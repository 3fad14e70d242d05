// C-ABI of the library (include/osscir.h): context creation, validation,
// per-geometry tables, and the per-iteration CUDA graph.
#include <algorithm>
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
    void* ptrs[] = {h->rec,     h->r64,    h->views,     h->chord,    h->exc_off,    h->exc_ent,  h->s4,
                    h->N4,      h->mu,     h->mu_in,     h->g,        h->c,          h->y,        h->x,
                    h->xbar,    h->xo,     h->dtpl_part, h->dtpl_out, h->bad_counts, h->model,    h->fwd_row,
                    h->fwd_cnt, h->fwd_k0, h->fwd_w, h->fwd_d, h->bp_span, h->bp_row,  h->bp_w,
                    h->bp_slot, h->bp_roff,   h->bp_rays, h->bp_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete h;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Measured counts must be finite and >= 0 (Eq. DTPL takes c log c).  c holds L
// rays of `stride` floats, of which the first W are the windows (the rest is padding).
bool counts_valid(const float* c, size_t L, int stride, int W) {
    for (size_t l = 0; l < L; ++l)
        for (int w = 0; w < W; ++w) {
            const float v = c[l * stride + w];
            if (!(v >= 0.0f) || !std::isfinite(v)) return false;
        }
    return true;
}

// The same check on device counts: any invalid value sets *bad (never cleared here).
__global__ void k_check_counts(const float* __restrict__ c, int L, int stride, int W, int* bad) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
        bool ok = true;
        for (int w = 0; w < W; ++w) {
            const float v = c[(size_t)l * stride + w];
            ok = ok && v >= 0.0f && isfinite(v);
        }
        if (!ok) *bad = 1;
    }
}

// Eigen-decomposition of a symmetric 3x3 matrix A (row-major) by cyclic Jacobi
// rotations (Golub and Van Loan, Sec. 8.5): A = V diag(w) V^T, V's columns the
// eigenvectors.
void sym3_eigen(const double A[9], double w[3], double V[9]) {
    double a[3][3] = {{A[0], A[1], A[2]}, {A[3], A[4], A[5]}, {A[6], A[7], A[8]}};
    double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > 1e-32 * dia)) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {   // A <- A J (columns p, q)
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {   // A <- J^T A (rows p, q)
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {   // V <- V J
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) {
        w[i] = a[i][i];
        for (int j = 0; j < 3; ++j) V[i * 3 + j] = v[i][j];
    }
}

// mu-PC (Sec. 1 and 2): a material basis whose attenuation curves are
// orthonormal over the energy grid (Euclidean inner product), with the symmetric
// choice M = (mu mu^T)^(-1/2), so mu' = M mu and, for unchanged line integrals
// (mu'^T f' = mu^T f), f' = M^-1 f.  Writes M (row-major, symmetric) and mu' in
// FP64; false if mu mu^T is singular to working precision.
bool mu_pc_basis(const float* mu, int nE, double M[9], std::vector<double>& mu_t) {
    double Gm[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int e = 0; e < nE; ++e) acc += (double)mu[i * nE + e] * (double)mu[j * nE + e];
            Gm[i * 3 + j] = acc;
        }
    double w[3], V[9];
    sym3_eigen(Gm, w, V);
    const double wmax = std::max(w[0], std::max(w[1], w[2]));
    for (int k = 0; k < 3; ++k)
        if (!(w[k] > 1e-14 * wmax) || !std::isfinite(w[k])) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += V[i * 3 + k] * V[j * 3 + k] / std::sqrt(w[k]);
            M[i * 3 + j] = acc;
        }
    mu_t.assign((size_t)3 * nE, 0.0);
    for (int i = 0; i < 3; ++i)
        for (int e = 0; e < nE; ++e)
            mu_t[(size_t)i * nE + e] = M[i * 3 + 0] * mu[e] + M[i * 3 + 1] * mu[nE + e] + M[i * 3 + 2] * mu[2 * nE + e];
    return true;
}

// Maps from the mu-PC basis to the caller's: f = M f' per pixel (FP64 arithmetic).
struct Basis3 {
    double m[9];
};
__global__ void k_maps_out(const float4* __restrict__ x, Basis3 B, float4* __restrict__ out, int P) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const float4 v = x[k];
    const double a = v.x, b = v.y, c = v.z;
    out[k] = make_float4((float)(B.m[0] * a + B.m[1] * b + B.m[2] * c), (float)(B.m[3] * a + B.m[4] * b + B.m[5] * c),
                         (float)(B.m[6] * a + B.m[7] * b + B.m[8] * c), 0.f);
}

// Energy windows of a spectra struct (0 means the default four).
int n_windows(const osscir_spectra* sp) { return sp->n_windows == 0 ? 4 : sp->n_windows; }

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
    const int nE = sp->n_energies, W = n_windows(sp);
    if (W != 4 && W != 5) return OSSCIR_E_INVALID;
    if (W != 4 && pa->inner > 1) return OSSCIR_E_INVALID;   // nested MOCCA keeps four-window models
    for (int b = 0; b < g->n_bins; ++b) {
        for (int w = 0; w < W; ++w) {
            double sum = 0.0;
            for (int i = 0; i < nE; ++i) {
                const float v = sp->s[((size_t)b * nE + i) * W + w];
                if (!std::isfinite(v) || v < 0.f) return OSSCIR_E_INVALID;
                sum += v;
            }
            if (std::fabs(sum - 1.0) > 1e-4) return OSSCIR_E_INVALID;
            if (!finite_pos(sp->N[(size_t)b * W + w])) return OSSCIR_E_INVALID;
        }
    }
    for (int i = 0; i < 3 * nE; ++i)   // a transformed basis (mu-PC) may have negative curves
        if (!std::isfinite(mu[i])) return OSSCIR_E_INVALID;
    if (!finite_pos(pa->lambda) || !(pa->lambda < 3.0e38)) return OSSCIR_E_INVALID;
    if (pa->model < 0 || pa->model > 3) return OSSCIR_E_INVALID;
    if (pa->spc < 0 || pa->spc > 2) return OSSCIR_E_INVALID;
    if (pa->spc == 2) {
        double M[9];
        std::vector<double> mu_t;
        if (!mu_pc_basis(mu, nE, M, mu_t)) return OSSCIR_E_INVALID;
    }
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
    h->nw = n_windows(sp);
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
    h->params.spc = pa->spc == 2 ? 1 : pa->spc;   // mu-PC runs the diagonal SPC in its basis
    h->basis = pa->spc == 2;
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
    const int W = h->nw, F4 = h->wf4();
    CK(dalloc(&h->s4, (size_t)nE * g->n_bins * F4));
    CK(dalloc(&h->N4, (size_t)g->n_bins * F4));
    CK(dalloc(&h->mu, 3 * nE));
    if (h->basis) {
        CK(dalloc(&h->mu_in, 3 * nE));
        CK(dalloc(&h->xo, P));
    }
    CK(dalloc(&h->g, L));
    CK(dalloc(&h->c, (size_t)L * F4));
    CK(dalloc(&h->y, (size_t)L * F4));
    CK(dalloc(&h->x, P));
    CK(dalloc(&h->xbar, 2 * (size_t)P));   // row-major, then the column-major copy
    CK(dalloc(&h->dtpl_part, h->n_part));
    CK(dalloc(&h->dtpl_out, 2));
    CK(dalloc(&h->bad_counts, 2));
    if (h->inner > 1) CK(dalloc(&h->model, (size_t)kModelStride * L));
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : h->ev) CK(cudaEventCreate(&e));
    CK(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
    cudaStream_t st = h->cap_stream;

    // spectral tables: s reordered to [nE][n_bins] window vectors (4 F4 floats, zero padded)
    // so consecutive rays read consecutive entries
    {
        const int S = 4 * F4;
        std::vector<float> s4((size_t)nE * g->n_bins * S, 0.0f), N4((size_t)g->n_bins * S, 0.0f);
        for (int b = 0; b < g->n_bins; ++b)
            for (int i = 0; i < nE; ++i)
                for (int w = 0; w < W; ++w)
                    s4[((size_t)i * g->n_bins + b) * S + w] = sp->s[((size_t)b * nE + i) * W + w];
        for (int b = 0; b < g->n_bins; ++b)
            for (int w = 0; w < W; ++w) N4[(size_t)b * S + w] = sp->N[(size_t)b * W + w];
        CK(cudaMemcpy(h->s4, s4.data(), s4.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->N4, N4.data(), N4.size() * sizeof(float), cudaMemcpyHostToDevice));
        if (h->basis) {
            std::vector<double> mu_t;
            if (!mu_pc_basis(mu, nE, h->Mb, mu_t)) return OSSCIR_E_INVALID;
            std::vector<float> mu32(mu_t.begin(), mu_t.end());
            CK(cudaMemcpy(h->mu, mu32.data(), sizeof(float) * 3 * nE, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(h->mu_in, mu, sizeof(float) * 3 * nE, cudaMemcpyHostToDevice));
        } else {
            CK(cudaMemcpy(h->mu, mu, sizeof(float) * 3 * nE, cudaMemcpyHostToDevice));
        }
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
    CK(cudaMemsetAsync(h->c, 0, sizeof(float4) * L * F4, st));
    CK(cudaMemsetAsync(h->y, 0, sizeof(float4) * L * F4, st));
    CK(cudaMemsetAsync(h->x, 0, sizeof(float4) * P, st));
    CK(cudaMemsetAsync(h->xbar, 0, sizeof(float4) * 2 * P, st));
    CK(cudaMemsetAsync(h->dtpl_out, 0, sizeof(double) * 2, st));
    CK(cudaMemsetAsync(h->bad_counts, 0, 2 * sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return OSSCIR_OK;
}

void free_tables(osscir_ctx* h) {
    void* ptrs[] = {h->fwd_row, h->fwd_cnt, h->fwd_k0, h->fwd_w, h->fwd_d, h->bp_span, h->bp_row,
                    h->bp_w,    h->bp_slot, h->bp_roff,   h->bp_rays, h->bp_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->fwd_row = nullptr;
    h->fwd_cnt = nullptr;
    h->fwd_k0 = nullptr;
    h->fwd_w = nullptr;
    h->fwd_d = nullptr;
    h->bp_span = nullptr;
    h->bp_row = nullptr;
    h->bp_w = nullptr;
    h->bp_slot = nullptr;
    h->bp_roff = nullptr;
    h->bp_rays = nullptr;
    h->bp_part = nullptr;
    h->bytes -= h->fp_bytes;
    h->fp_bytes = 0;
}

// Device array of the prefix sums of n counts (in place on the host copy), with
// its total appended; false if the total does not fit 32 bits.
bool prefix_rows(std::vector<uint32_t>& v, size_t n) {
    uint64_t run = 0;
    for (size_t i = 0; i < n; ++i) {
        const uint64_t c = v[i];
        v[i] = (uint32_t)run;
        run += c;
    }
    if (run > 0xffffffffull) return false;
    v[n] = (uint32_t)run;
    return true;
}

// Build the footprint tables (FpTables) once per context, before the first
// iteration graph is captured.  If the device has no room for them the context
// keeps the on-the-fly projections (the same results, computed again every
// iteration).
osscir_status build_tables(osscir_ctx* h) {
    if (h->fp_state != 0) return OSSCIR_OK;
    cudaStream_t st = h->cap_stream;
    const GeomC& C = h->gc;
    const size_t nbg = (C.n_bins + 31) / 32, n_fw = (size_t)C.n_views * nbg;
    const int G = bp_view_groups(h->P, C.n_views);
    size_t before = h->bytes;
    g_dalloc_bytes = &h->bytes;
    auto fail = [&](cudaError_t e) -> osscir_status {
        g_dalloc_bytes = &g_dalloc_bytes_sink;
        h->fp_bytes = h->bytes - before;
        free_tables(h);
        if (e == cudaErrorMemoryAllocation) {   // no room: keep the on-the-fly projections
            cudaGetLastError();
            h->fp_state = -1;
            return OSSCIR_OK;
        }
        return from_cuda(e);
    };
#define CKT(expr)                                    \
    do {                                             \
        const cudaError_t e_ = (expr);               \
        if (e_ != cudaSuccess) return fail(e_);      \
    } while (0)
    // forward: per-ray counts and per-warp rows, then the pairs
    CKT(dalloc(&h->fwd_cnt, (size_t)h->L));
    CKT(dalloc(&h->fwd_row, n_fw + 1));
    CKT(launch_fp_fwd_count(C, h->exc(), h->rec, h->fwd_cnt, h->fwd_row, st));
    std::vector<uint32_t> rows(n_fw + 1, 0);
    CKT(cudaMemcpyAsync(rows.data(), h->fwd_row, sizeof(uint32_t) * n_fw, cudaMemcpyDeviceToHost, st));
    CKT(cudaStreamSynchronize(st));
    for (size_t i = 0; i < n_fw; ++i) rows[i] = (rows[i] + 1) & ~1u;   // even: entries are read two at a time
    if (!prefix_rows(rows, n_fw)) return fail(cudaErrorMemoryAllocation);
    CKT(cudaMemcpyAsync(h->fwd_row, rows.data(), sizeof(uint32_t) * (n_fw + 1), cudaMemcpyHostToDevice, st));
    CKT(dalloc(&h->fwd_w, (size_t)rows[n_fw] * 32));
    CKT(dalloc(&h->fwd_d, (size_t)rows[n_fw] * 32));
    CKT(dalloc(&h->fwd_k0, (size_t)h->L));
    {
        int* bad = nullptr;   // a pixel step outside 16 bits: keep the on-the-fly projections
        CKT(dalloc(&bad, 1));
        int bad_h = 0;
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_fp_fwd_fill(C, h->exc(), h->rec, h->fwd_row, h->fwd_w, h->fwd_d, h->fwd_k0,
                                                     bad, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(bad);
        h->bytes -= sizeof(int);
        CKT(e);
        if (bad_h) return fail(cudaErrorMemoryAllocation);
    }
    // back-projection (blocked): per tile and view the union of candidate bins; the
    // chunk size (views per staged chunk) so that two stage buffers fit in 48 KB;
    // then per-pixel counts and per-warp rows of each (block, chunk), then the pairs
    const int n_t = bt_tiles(C.grid.n), per = (C.n_views + G - 1) / G;
    CKT(dalloc(&h->bp_span, (size_t)n_t * C.n_views));
    CKT(launch_fpb_span(C, h->views, h->bp_span, st));
    std::vector<uint32_t> span((size_t)n_t * C.n_views);
    CKT(cudaMemcpyAsync(span.data(), h->bp_span, sizeof(uint32_t) * span.size(), cudaMemcpyDeviceToHost, st));
    CKT(cudaStreamSynchronize(st));
    int chunk = 0, slots = 0;
    auto group_range = [&](int g, int& v0, int& v1) {
        v0 = std::min(C.n_views, g * per);
        v1 = std::min(C.n_views, v0 + per);
    };
    for (int cand = kBTMaxChunk; cand >= 1 && !chunk; cand /= 2) {
        int most = 0;
        for (int t = 0; t < n_t; ++t)
            for (int g = 0; g < G; ++g) {
                int v0, v1;
                group_range(g, v0, v1);
                for (int u0 = v0; u0 < v1; u0 += cand) {
                    int sum = 0;
                    for (int u = u0; u < std::min(v1, u0 + cand); ++u)
                        sum += (int)(span[(size_t)t * C.n_views + u] >> 16);
                    most = std::max(most, sum);
                }
            }
        const int padded = (most + 3) / 4 * 4;   // stage buffers of 44-byte slots stay 16-byte aligned
        if (fpb_stage_bytes(padded) <= 48 * 1024) {
            chunk = cand;
            slots = padded;
        }
    }
    if (chunk > 0) {
        const int nch = (per + chunk - 1) / chunk;
        const size_t n_e = (size_t)n_t * G * nch;
        // each entry's staged rays, view after view, in slot order
        std::vector<uint32_t> roff(n_e + 1, 0);
        std::vector<int> rays;
        for (int t = 0; t < n_t; ++t)
            for (int g = 0; g < G; ++g) {
                int v0, v1;
                group_range(g, v0, v1);
                for (int c = 0; c < nch; ++c) {
                    roff[((size_t)t * G + g) * nch + c] = (uint32_t)rays.size();
                    const int u0 = std::min(v1, v0 + c * chunk), u1 = std::min(v1, u0 + chunk);
                    for (int u = u0; u < u1; ++u) {
                        const uint32_t sp = span[(size_t)t * C.n_views + u];
                        for (uint32_t i = 0; i < (sp >> 16); ++i) rays.push_back(u * C.n_bins + (int)(sp & 0xffffu) + (int)i);
                    }
                }
            }
        roff[n_e] = (uint32_t)rays.size();
        CKT(dalloc(&h->bp_roff, n_e + 1));
        CKT(dalloc(&h->bp_rays, rays.size()));
        CKT(cudaMemcpyAsync(h->bp_roff, roff.data(), sizeof(uint32_t) * (n_e + 1), cudaMemcpyHostToDevice, st));
        CKT(cudaMemcpyAsync(h->bp_rays, rays.data(), sizeof(int) * rays.size(), cudaMemcpyHostToDevice, st));
        CKT(dalloc(&h->bp_row, n_e * (kBTThreads / 32) + 1));
        CKT(launch_fpb_count(C, h->exc(), h->rec, h->views, G, chunk, nch, h->bp_row, st));
        const size_t n_w = n_e * (kBTThreads / 32);
        std::vector<uint32_t> brow(n_w + 1, 0);
        CKT(cudaMemcpyAsync(brow.data(), h->bp_row, sizeof(uint32_t) * n_w, cudaMemcpyDeviceToHost, st));
        CKT(cudaStreamSynchronize(st));
        for (size_t i = 0; i < n_w; ++i) brow[i] = (brow[i] + 1) & ~1u;   // even: entries are read two at a time
        if (!prefix_rows(brow, n_w)) return fail(cudaErrorMemoryAllocation);
        CKT(cudaMemcpyAsync(h->bp_row, brow.data(), sizeof(uint32_t) * (n_w + 1), cudaMemcpyHostToDevice, st));
        CKT(dalloc(&h->bp_w, (size_t)brow[n_w] * 32));
        CKT(dalloc(&h->bp_slot, (size_t)brow[n_w] * 32));
        CKT(dalloc(&h->bp_part, (size_t)G * 9 * h->P));
        // rows a pixel does not fill: no slot (0xffff), weight 0
        CKT(cudaMemsetAsync(h->bp_slot, 0xff, sizeof(uint16_t) * (size_t)brow[n_w] * 32, st));
        CKT(cudaMemsetAsync(h->bp_w, 0, sizeof(float) * (size_t)brow[n_w] * 32, st));
        CKT(launch_fpb_fill(C, h->exc(), h->rec, h->views, h->bp_span, G, chunk, nch, h->bp_row, h->bp_w,
                            h->bp_slot, st));
        h->bp_chunk = chunk;
        h->bp_nch = nch;
        h->bp_slots = slots;
    }
    CKT(cudaStreamSynchronize(st));
#undef CKT
    g_dalloc_bytes = &g_dalloc_bytes_sink;
    h->bp_groups = G;
    h->fp_bytes = h->bytes - before;
    h->fp_tab = h->fp();
    h->fp_state = 1;
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
    e = launch_mocca_proj(h->gc, h->exc(), h->rec, h->solve(), st, 0, -1, h->fp_or_null());
    if (e != cudaSuccess) return e;
    e = cudaEventRecordWithFlags(h->ev[1], st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    if (inner_step) {
        e = launch_mocca_ray_inner(h->gc, h->rec, h->solve(), st);
        if (e != cudaSuccess) return e;
        e = cudaEventRecordWithFlags(h->ev[2], st, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
        e = launch_mocca_bp(h->gc, h->exc(), h->rec, h->views, h->params, h->solve(), st, h->fp_or_null());
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
    e = launch_mocca_bp(h->gc, h->exc(), h->rec, h->views, h->params, h->solve(), st, h->fp_or_null());
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
    const osscir_status ts = build_tables(h);   // before the capture: the launches take the tables
    if (ts != OSSCIR_OK) return ts;
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

osscir_status ctx_build_tables(osscir_ctx* h) { return build_tables(h); }

cudaError_t ctx_maps_out(const osscir_ctx* h, const float4* x, float4* out, cudaStream_t st) {
    if (!h->basis) return cudaMemcpyAsync(out, x, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st);
    Basis3 B;
    for (int i = 0; i < 9; ++i) B.m[i] = h->Mb[i];
    k_maps_out<<<(h->P + 255) / 256, 256, 0, st>>>(x, B, out, h->P);
    return cudaGetLastError();
}

void ctx_maps_out_host(const osscir_ctx* h, float* maps) {
    if (!h->basis) return;
    const double* M = h->Mb;
    for (int k = 0; k < h->P; ++k) {
        float* v = maps + (size_t)4 * k;
        const double a = v[0], b = v[1], c = v[2];
        v[0] = (float)(M[0] * a + M[1] * b + M[2] * c);
        v[1] = (float)(M[3] * a + M[4] * b + M[5] * c);
        v[2] = (float)(M[6] * a + M[7] * b + M[8] * c);
        v[3] = 0.f;
    }
}

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

osscir_status osscir_memory(osscir_t h, size_t* device_bytes, size_t* table_bytes) {
    if (!h) return OSSCIR_E_INVALID;
    if (device_bytes) *device_bytes = h->bytes;
    if (table_bytes) *table_bytes = h->fp_state == 1 ? h->fp_bytes : 0;
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
    CK(launch_counts(h->gc, h->exc(), h->rec, h->spec_in(), reinterpret_cast<const float4*>(f),
                     reinterpret_cast<float4*>(chat), nullptr, nullptr, as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_set_counts(osscir_t h, const float* c, void* stream) {
    if (!h || !c) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    const size_t ray_bytes = sizeof(float4) * h->wf4() * h->L;
    CK(cudaMemcpyAsync(h->c, c, ray_bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(h->bad_counts, 0, sizeof(int), st));
    k_check_counts<<<std::min((h->L + 255) / 256, 1024), 256, 0, st>>>(
        reinterpret_cast<const float*>(h->c), h->L, 4 * h->wf4(), h->nw, h->bad_counts);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(h->y, 0, ray_bytes, st));
    CK(cudaMemsetAsync(h->x, 0, sizeof(float4) * h->P, st));
    CK(cudaMemsetAsync(h->xbar, 0, sizeof(float4) * 2 * h->P, st));
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

osscir_status osscir_mocca_partial(osscir_t h, int v0, int v1, float* chan, void* stream) {
    if (!h || !chan || v0 < 0 || v1 > h->gc.n_views || v0 >= v1 || h->inner > 1) return OSSCIR_E_INVALID;
    const osscir_status ts = build_tables(h);
    if (ts != OSSCIR_OK) return ts;
    cudaStream_t st = as_stream(stream);
    const SolveD D = h->solve();
    CK(launch_mocca_proj(h->gc, h->exc(), h->rec, D, st, v0, v1, h->fp_or_null()));
    CK(launch_mocca_ray(h->gc, h->rec, h->spec(), h->params, D, st, v0, v1));
    const int nbg = (h->gc.n_bins + 31) / 32;   // D_TPL partials per view
    CK(launch_dtpl_reduce(h->dtpl_part + (size_t)v0 * nbg, (v1 - v0) * nbg, h->dtpl_out + 1, st));
    CK(launch_mocca_bp_partial(h->gc, h->exc(), h->rec, h->views, h->params, D, v0, v1, chan, st,
                               h->fp_or_null()));
    return OSSCIR_OK;
}

osscir_status osscir_mocca_apply(osscir_t h, const float* chan, void* stream) {
    if (!h || !chan || h->inner > 1) return OSSCIR_E_INVALID;
    CK(launch_mocca_apply(h->gc, h->params, h->solve(), chan, as_stream(stream)));
    h->iter += 1;
    return OSSCIR_OK;
}

osscir_status osscir_reconstruct(osscir_t h, const float* c_host, int n_iters, float* maps_out_host,
                                 void* stream) {
    if (!h || !c_host || !maps_out_host || n_iters < 0) return OSSCIR_E_INVALID;
    if (!counts_valid(c_host, h->L, 4 * h->wf4(), h->nw)) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    const size_t ray_bytes = sizeof(float4) * h->wf4() * h->L;
    CK(cudaMemcpyAsync(h->c, c_host, ray_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->y, 0, ray_bytes, st));
    CK(cudaMemsetAsync(h->x, 0, sizeof(float4) * h->P, st));
    CK(cudaMemsetAsync(h->xbar, 0, sizeof(float4) * 2 * h->P, st));
    h->iter = 0;
    h->phase = 0;
    const osscir_status s = osscir_mocca_step(h, n_iters, stream);
    if (s != OSSCIR_OK) return s;
    const float4* xs = h->x;
    if (h->basis) {
        CK(ctx_maps_out(h, h->x, h->xo, st));
        xs = h->xo;
    }
    CK(cudaMemcpyAsync(maps_out_host, xs, sizeof(float4) * h->P, cudaMemcpyDeviceToHost, st));
    double d = 0.0;   // D_TPL at the last expansion point (the value the iterations computed)
    int kerr = 0;
    if (n_iters > 0) CK(cudaMemcpyAsync(&d, h->dtpl_out + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&kerr, h->bad_counts + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (kerr) return OSSCIR_E_CUDA;
    if (!std::isfinite(d)) return OSSCIR_E_DIVERGED;
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
    CK(ctx_maps_out(h, h->x, reinterpret_cast<float4*>(x_out), as_stream(stream)));
    return OSSCIR_OK;
}

osscir_status osscir_get_state(osscir_t h, float* x, float* xbar, float* y, int* iter, void* stream) {
    if (!h || !x || !xbar || !y) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(x, h->x, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(xbar, h->xbar, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(y, h->y, sizeof(float4) * h->wf4() * h->L, cudaMemcpyDeviceToDevice, st));
    if (iter) *iter = h->iter;
    return OSSCIR_OK;
}

osscir_status osscir_set_state(osscir_t h, const float* x, const float* xbar, const float* y, int iter,
                               void* stream) {
    if (!h || !x || !xbar || !y || iter < 0) return OSSCIR_E_INVALID;
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(h->x, x, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->xbar, xbar, sizeof(float4) * h->P, cudaMemcpyDeviceToDevice, st));
    CK(launch_xbar_columns(h->gc.grid.n, h->xbar, st));
    CK(cudaMemcpyAsync(h->y, y, sizeof(float4) * h->wf4() * h->L, cudaMemcpyDeviceToDevice, st));
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
    int bad[2] = {0, 0};
    CK(cudaMemcpyAsync(out, h->dtpl_out + which, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(bad, h->bad_counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad[1]) return OSSCIR_E_CUDA;
    if (bad[0]) return OSSCIR_E_INVALID;
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
