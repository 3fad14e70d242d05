// Host-side declarations of the kernel launchers (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "osscir_internal.cuh"

namespace osscir {

// FP64 ray: foot point (x, y) nearest the origin and unit direction (z, w).
struct __align__(32) Ray64 {
    double x, y, z, w;
};

// FP64 geometry as given at creation (planes at x0 + i h, x0 = -n h / 2).
struct GeomD {
    int n;
    double h, x0;
    int n_views, n_bins;
    double arc_deg, start_deg, bin_mm, sid, sdd;
    double thr;   // footprint threshold: 1e-9 h
};

// Spectral tables on the device.
struct SpecD {
    int n_energies;
    const float4* s4;   // [nE][n_bins] window vectors (win_f4 float4 each): s_{w,b,i}
    const float4* N4;   // [n_bins] window vectors: N_{w,b}
    const float* mu;    // [3][nE]
    int exp_model;      // 0: softexp (Eq. finalModel), 1: exp for every energy (Eq. fullModel)
    int n_windows;      // W: 4 or 5 (the per-ray arrays c, y, chat hold win_f4<W> float4 per ray)
};

// MOCCA per-solve parameters.
struct StepParams {
    float lambda;
    int model;       // 0: eigen-clipped Hessian, 1: W = 0, 2: Gauss-Newton sum_w c_w a_w a_w^T, 3: W = diag(c)
    int spc;         // 0: m-block-diagonal SPC, 1: diagonal SPC
    int use_box;
    float lo[3], hi[3];
};

// MOCCA per-solve device state.
struct SolveD {
    float4* g;          // [L] line integrals of the three maps at xbar
    const float4* c;    // [L] measured counts
    float4* y;          // [L] dual
    float4* x;          // [P] x_n
    float4* xbar;       // [2P] 2 x_n - x_{n-1}: pixel iy n + ix, then a column-major copy at P + ix n + iy
    const float* chord; // [L] (X 1)_l
    double* dtpl_part;  // [fwd blocks]
    float4* model;      // [L][kModelStride] local models kept for nested MOCCA, or null
    int* err;           // set to 1 by a kernel whose bounded wait for its own copies ran out (else untouched)
};

// Per-ray local model kept by an outer iteration of nested MOCCA (float4 slots):
//   0..2 alpha_{w,m} for m = 0, 1, 2 (over w);  3 (g0, flag: 1 solve, 0 keep y);
//   4, 5 r as the hi and lo floats of a double-float;  6 Sigma^-1;  7..10 the rows of
//   B, the map of the dual prox y' = r + B (u - r).
constexpr int kModelStride = 11;

constexpr int kFwdThreads = 128;
constexpr int kBpTileX = 16, kBpTileY = 8;            // plain back-projection tile
constexpr int kBpPixX = 2, kBpPixY = 32;              // MOCCA back-projection pixel tile (2 x 32: measured fastest)
constexpr int kBpPix = kBpPixX * kBpPixY;
constexpr int kBpMaxThreads = 512;                    // kBpPix x up to 8 view groups
// Blocked back-projection table: a block is a tile of kBTX x kBTY pixels (one
// per thread) and one view group; its views go in chunks of at most kBTMaxChunk.
constexpr int kBTX = 16, kBTY = 16, kBTThreads = kBTX * kBTY, kBTMaxChunk = 16;
inline int bt_tiles(int n) { return ((n + kBTX - 1) / kBTX) * ((n + kBTY - 1) / kBTY); }

// Footprint tables of one geometry: the pairs (l, k) of X with their weights,
// in the order each projector visits them.
//   Forward (ray-major): warp w = (view v, 32-bin group bx), w = v nbg + bx with
//   nbg = ceil(n_bins / 32), lane r = bin 32 bx + r.  Ray l has fwd_cnt[l] pairs
//   in the visiting order of ray_weights; its j-th pair is the weight fwd_w[i]
//   and the pixel k_j = fwd_k0[l] + sum_{i <= j} fwd_d[i] (fwd_d: the 16-bit step
//   from the previous pixel, 0 for the first), at i = (fwd_row[w] + j - j mod 2)
//   32 + 2 r + j mod 2: two pairs side by side, so a lane reads two with one load
//   (6 bytes a pair).  fwd_row is the prefix sum of the warps' largest counts,
//   each rounded up to even.
//   Back-projection (blocked): block b = t G + g (tile t, view group g of G =
//   bp_groups); the group's views (the split of k_mocca_bp) in chunks of
//   bp_chunk views, bp_nch chunks per group, entry e = b bp_nch + c.  bp_span
//   [t n_views + u] = tlo | span << 16: the union of the tile's candidate bins in
//   view u.  An entry's rays, view after view (ray (u, tlo + i)), are its stage
//   slots: bp_rays[bp_roff[e] + slot], at most bp_slots of them.  The rows of
//   warp w of entry e, bp_row[8 e + w] .. bp_row[8 e + w + 1] (an even number, so
//   that a lane reads two rows with one load), are aligned per view: view u of
//   the chunk takes as many rows as the warp's largest pair count in u.  Thread
//   r's pairs (stage slot, weight) in the order of bp_pixel_sum sit at rows j of
//   their view, (bp_slot, bp_w)[(row + j - j mod 2) 32 + 2 (r mod 32) + j mod 2];
//   the rows a pixel does not fill hold the slot 0xffff.
//   bp_part: [G][9][P] scratch for the groups' channel sums.
struct FpTables {
    const uint32_t* fwd_row;   // [n_views nbg + 1]
    const int* fwd_cnt;        // [L]
    const int* fwd_k0;         // [L] first pixel of each ray
    const float* fwd_w;        // null: the forward projection is computed on the fly
    const int16_t* fwd_d;
    const uint32_t* bp_span;   // [bt_tiles(n) n_views]
    const uint32_t* bp_row;    // [n_entries 8 + 1]
    const float* bp_w;         // null: the back-projection is computed on the fly
    const uint16_t* bp_slot;
    const uint32_t* bp_roff;   // [n_entries + 1]
    const int* bp_rays;
    float* bp_part;            // [bp_groups][9][P]
    int bp_groups, bp_chunk, bp_nch, bp_slots;
};
// Shared memory of the blocked back-projection's two stage buffers of `slots` slots.
int fpb_stage_bytes(int slots);

// View groups per pixel for the MOCCA back-projection: enough threads to fill
// the GPU several times over, at most 8, and at least one view per group.
inline int bp_view_groups(int n_pixels, int n_views) {
    int G = n_pixels <= 131072 ? 8 : (n_pixels <= 524288 ? 4 : 2);
    while (G > 1 && G > n_views) G >>= 1;
    return G;
}

cudaError_t launch_ray_setup(const GeomD& G, double r_img, RayRec* rec, Ray64* r64, ViewF* views,
                             cudaStream_t st);
cudaError_t launch_exc_pass(const GeomC& C, const GeomD& G, const RayRec* rec, const Ray64* r64, int* count,
                            const int* off, int2* ent, cudaStream_t st);
cudaError_t launch_chord(const GeomC& C, const ExcTable& E, const RayRec* rec, float* chord, cudaStream_t st);
cudaError_t launch_footprint_rays(const GeomC& C, const ExcTable& E, const RayRec* rec, int l0, int n, int cap,
                                  int* cnt, int* pix, float* wt, cudaStream_t st);
cudaError_t launch_footprint_pixels(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                    int k0, int n, int cap, int* cnt, int* ray, float* wt, cudaStream_t st);

cudaError_t launch_forward4(const GeomC& C, const ExcTable& E, const RayRec* rec, const float4* x, float4* g,
                            cudaStream_t st);
cudaError_t launch_backproject4(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                const float4* rf, float4* img, cudaStream_t st);
cudaError_t launch_counts(const GeomC& C, const ExcTable& E, const RayRec* rec, const SpecD& S, const float4* f,
                          float4* chat, const float4* c, double* dtpl_part, cudaStream_t st);
// The ray-driven kernels over the views [v0, v1) (v1 < 0: all views); with
// footprint tables T the projections stream them (same results bit for bit).
cudaError_t launch_mocca_proj(const GeomC& C, const ExcTable& E, const RayRec* rec, const SolveD& D,
                              cudaStream_t st, int v0 = 0, int v1 = -1, const FpTables* T = nullptr);
cudaError_t launch_mocca_ray(const GeomC& C, RayRec* rec, const SpecD& S, const StepParams& P, const SolveD& D,
                             cudaStream_t st, int v0 = 0, int v1 = -1);
// Outer iteration of nested MOCCA: the per-ray step that also keeps each ray's model in D.model.
cudaError_t launch_mocca_ray_keep(const GeomC& C, RayRec* rec, const SpecD& S, const StepParams& P,
                                  const SolveD& D, cudaStream_t st);
// Inner iteration of nested MOCCA: the dual step on the kept models.
cudaError_t launch_mocca_ray_inner(const GeomC& C, RayRec* rec, const SolveD& D, cudaStream_t st);
cudaError_t launch_mocca_bp(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                            const StepParams& P, const SolveD& D, cudaStream_t st, const FpTables* T = nullptr);
cudaError_t launch_dtpl_reduce(const double* part, int n, double* out, cudaStream_t st);
// View split of one iteration: the back-projection of the views [v0, v1) into
// the nine per-pixel channels chan [9][P] (no primal step), and the primal step
// from channels summed over all view ranges.
cudaError_t launch_mocca_bp_partial(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                    const StepParams& P, const SolveD& D, int v0, int v1, float* chan,
                                    cudaStream_t st, const FpTables* T = nullptr);
// Footprint table construction: counts (forward: per ray, and per warp the slot
// rows; back-projection: slot rows per entry), then the fills from the row offsets.
cudaError_t launch_fp_fwd_count(const GeomC& C, const ExcTable& E, const RayRec* rec, int* cnt,
                                uint32_t* warp_rows, cudaStream_t st);
// Writes the column-major copy of xbar ([2P]: P + ix n + iy) from its row-major half.
cudaError_t launch_xbar_columns(int n, float4* xbar, cudaStream_t st);
// Fills fwd_w, fwd_d and fwd_k0; sets *bad if a pixel step does not fit in 16 bits.
cudaError_t launch_fp_fwd_fill(const GeomC& C, const ExcTable& E, const RayRec* rec, const uint32_t* fwd_row,
                               float* fwd_w, int16_t* fwd_d, int* fwd_k0, int* bad, cudaStream_t st);
cudaError_t launch_fpb_span(const GeomC& C, const ViewF* views, uint32_t* span, cudaStream_t st);
cudaError_t launch_fpb_count(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views, int G,
                             int chunk, int nch, uint32_t* warp_rows, cudaStream_t st);
cudaError_t launch_fpb_fill(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                            const uint32_t* span, int G, int chunk, int nch, const uint32_t* bp_row, float* bp_w,
                            uint16_t* bp_slot, cudaStream_t st);
cudaError_t launch_mocca_apply(const GeomC& C, const StepParams& P, const SolveD& D, const float* chan,
                               cudaStream_t st);

// Ray-driven kernels: blocks of 32 bins x (kFwdThreads / 32) views.
inline dim3 fwd_grid(int n_bins, int n_views) {
    return dim3((n_bins + 31) / 32, (n_views + kFwdThreads / 32 - 1) / (kFwdThreads / 32));
}
// D_TPL partial sums: one per (view, group of 32 bins), i.e. per warp of the ray-driven kernels.
inline int dtpl_partials(int n_bins, int n_views) { return n_views * ((n_bins + 31) / 32); }

// ------------------------------------------------------------------ batched kernels

// One solve of a batch as the batched kernels see it (device array, one per solve).
struct SolveDesc {
    GeomC C;
    ExcTable E;
    RayRec* rec;
    const ViewF* views;
    SpecD S;
    StepParams P;
    SolveD D;
    double* dtpl_out;   // D_TPL at the last expansion point
    int n_part;         // dtpl_partials(n_bins, n_views)
    int bp_groups;      // bp_view_groups(P, n_views), a divisor of 8
    FpTables T;         // the solve's footprint tables (null pointers: the projections run on the fly)
};

constexpr int kBatchProjMaxThreads = 256;   // up to 8 views x 32 bins per projection block

// Work-list sizes per solve.  Projection: tiles of 32 bins x vb views; ray
// kernel: 32 bins x 4 views; back-projection: 8 / G pixel tiles of kBpPix pixels
// (tx wide) per item.
inline int batch_proj_tiles(int n_bins, int n_views, int vb) {
    return ((n_bins + 31) / 32) * ((n_views + vb - 1) / vb);
}
inline int batch_bp_items(int n, int tx, int G) {
    const int ty = kBpPix / tx, tiles = ((n + tx - 1) / tx) * ((n + ty - 1) / ty), per = 8 / G;
    return (tiles + per - 1) / per;
}

// grid <= 0: one CTA per work item; otherwise that many persistent CTAs.
cudaError_t launch_batch_proj(const SolveDesc* sd, const int2* items, int n_items, int vb, int grid,
                              cudaStream_t st);
cudaError_t launch_batch_ray(const SolveDesc* sd, const int2* items, int n_items, int grid, cudaStream_t st);
cudaError_t launch_batch_bp(const SolveDesc* sd, const int2* items, int n_items, int tx, int grid,
                            cudaStream_t st);
cudaError_t launch_batch_dtpl(const SolveDesc* sd, int n_solves, cudaStream_t st);
// Back-projection of solves with footprint tables: items (solve, table block),
// then fin_items (solve, block of 256 pixels) for the group sums and a7; smem:
// the largest solve's two stage buffers (fpb_stage_bytes).
cudaError_t launch_batch_fpb(const SolveDesc* sd, const int2* items, int n_items, const int2* fin_items,
                             int n_fin, int grid, size_t smem, cudaStream_t st);
// Resident CTAs per SM of a batched kernel (0 projection, 1 ray, 2 back-projection
// on the fly, 3 back-projection from tables with smem bytes of dynamic shared memory).
cudaError_t batch_resident_ctas(int kernel, int threads, int* per_sm, size_t smem = 0);

}  // namespace osscir
