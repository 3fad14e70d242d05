// The reconstruction context behind osscir_t (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "../../include/osscir.h"
#include "osscir_launch.h"

struct osscir_ctx {
    int device = 0;
    size_t bytes = 0;   // device bytes allocated by this context
    osscir::GeomD g64{};
    osscir::GeomC gc{};
    int P = 0, L = 0, nE = 0;
    int nw = 4;   // energy windows W (4 or 5)
    osscir::StepParams params{};
    // per-geometry tables
    osscir::RayRec* rec = nullptr;
    osscir::Ray64* r64 = nullptr;
    osscir::ViewF* views = nullptr;
    float* chord = nullptr;
    int* exc_off = nullptr;
    int2* exc_ent = nullptr;
    int exc_n = 0;
    // spectral tables
    float4* s4 = nullptr;   // [nE][n_bins] window vectors
    float4* N4 = nullptr;   // [n_bins] window vectors
    float* mu = nullptr;      // [3][nE] the curves the iteration uses (mu-PC: the transformed ones)
    float* mu_in = nullptr;   // [3][nE] the caller's curves, kept apart only for mu-PC (else null)
    // mu-PC (spc = 2): the iteration runs in the basis f' = M^-1 f with M = (mu mu^T)^(-1/2)
    // (symmetric); maps leave the library as f = M f'.  xo: [P] staging for the maps.
    int basis = 0;
    double Mb[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    float4* xo = nullptr;
    // solver state
    float4* g = nullptr;
    float4* c = nullptr;   // [L] window vectors
    float4* y = nullptr;   // [L] window vectors
    float4* x = nullptr;
    float4* xbar = nullptr;
    double* dtpl_part = nullptr;
    double* dtpl_out = nullptr;   // [0]: at x (on request), [1]: at the last expansion point
    int* bad_counts = nullptr;    // [0]: set by the check of the counts osscir_set_counts loads (0: valid);
                                  // [1]: set by a kernel whose bounded wait for its own copies ran out
    int n_part = 0;
    int exp_model = 0;   // counts model: 0 softexp (Eq. finalModel), 1 exp (Eq. fullModel)
    int iter = 0;
    // nested MOCCA: iterations per kept local model, the position in the cycle
    // (0: the next iteration is an outer one) and the models [L][kModelStride]
    int inner = 1, phase = 0;
    float4* model = nullptr;
    // footprint tables (built before the first plain iteration; see FpTables)
    int fp_state = 0;   // 0 not built yet, 1 built, -1 not used (no room on the device)
    uint32_t* fwd_row = nullptr;
    int* fwd_cnt = nullptr;
    int* fwd_k0 = nullptr;
    float* fwd_w = nullptr;   // null: the forward projection stays on the fly
    int16_t* fwd_d = nullptr;
    uint32_t* bp_span = nullptr;
    uint32_t* bp_row = nullptr;
    float* bp_w = nullptr;   // null: the back-projection stays on the fly
    uint16_t* bp_slot = nullptr;
    uint32_t* bp_roff = nullptr;
    int* bp_rays = nullptr;
    float* bp_part = nullptr;
    int bp_groups = 1, bp_chunk = 0, bp_nch = 0, bp_slots = 0;
    size_t fp_bytes = 0;
    osscir::FpTables fp() const {
        return osscir::FpTables{fwd_row, fwd_cnt, fwd_k0,  fwd_w,   fwd_d,     bp_span, bp_row, bp_w,
                                bp_slot, bp_roff, bp_rays,   bp_part, bp_groups, bp_chunk, bp_nch, bp_slots};
    }
    const osscir::FpTables* fp_or_null() const { return fp_state == 1 ? &fp_tab : nullptr; }
    osscir::FpTables fp_tab{};
    // per-iteration graph
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph_in = nullptr;        // inner iteration of nested MOCCA
    cudaGraphExec_t gexec_in = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // recorded around the kernels inside the graph
    cudaStream_t side_stream = nullptr;                 // D_TPL reduction beside the back-projection
    cudaEvent_t fork = nullptr, join = nullptr;

    osscir::ExcTable exc() const { return osscir::ExcTable{exc_off, exc_ent}; }
    osscir::SpecD spec() const { return osscir::SpecD{nE, s4, N4, mu, exp_model, nw}; }
    // the spectral tables with the caller's attenuation curves (for maps in the caller's basis)
    osscir::SpecD spec_in() const { return osscir::SpecD{nE, s4, N4, mu_in ? mu_in : mu, exp_model, nw}; }
    // float4 per ray of the window arrays c, y (and of the caller's counts): 1 for 4 windows, 2 for 5
    int wf4() const { return nw > 4 ? 2 : 1; }
    osscir::SolveD solve() const {
        return osscir::SolveD{g, c, y, x, xbar, chord, dtpl_part, model, bad_counts ? bad_counts + 1 : nullptr};
    }
};

namespace osscir {

// Validate the inputs, allocate the device state and build the per-geometry
// tables on the current device (synchronises).  On error *out is null.
osscir_status ctx_create(const osscir_geometry* geom, const osscir_spectra* spectra, const float* mu,
                         const osscir_params* params, osscir_ctx** out);
void ctx_destroy(osscir_ctx* h);
osscir_status ctx_validate(const osscir_geometry* geom, const osscir_spectra* spectra, const float* mu,
                           const osscir_params* params);
// Maps x (the iteration's basis, device [P]) to the caller's basis in out (device [P]);
// a plain copy unless the context runs mu-PC.
cudaError_t ctx_maps_out(const osscir_ctx* h, const float4* x, float4* out, cudaStream_t st);
// The same on host maps [P][4] in place (FP64 arithmetic).
void ctx_maps_out_host(const osscir_ctx* h, float* maps);
// Capture the per-iteration graph(s) once.
osscir_status ctx_ensure_graph(osscir_ctx* h);
// Build the footprint tables if they are not built yet (synchronises the
// context's own stream); a device without room leaves the on-the-fly kernels.
osscir_status ctx_build_tables(osscir_ctx* h);

// Batch runner for the served form: the batched kernels over a set of contexts
// that changes over time, with all updates in stream order on one stream.
struct BatchRun;
BatchRun* batchrun_new();
void batchrun_free(BatchRun* r);   // synchronises the device
// Make ctx the batch, split into `branches` (1, 2 or 4) graph branches
// (descriptors, work lists and the iteration graphs are rebuilt; device
// buffers grow with stream-ordered allocation on st).
osscir_status batchrun_set(BatchRun* r, const std::vector<osscir_ctx*>& ctx, int branches, cudaStream_t st);
// Relative device time of one MOCCA iteration of a context (for load balancing).
double batch_solve_cost(const osscir_ctx* h);
// Enqueue n_iters MOCCA iterations of every solve of the batch on st.
osscir_status batchrun_step(BatchRun* r, int n_iters, cudaStream_t st);

}  // namespace osscir
