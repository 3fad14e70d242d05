/*
 * osscir: one-step spectral CT image reconstruction of three basis-material
 * maps by MOCCA with m-block-diagonal step-preconditioning, on one GB300 GPU.
 *
 * Method: Sidky, Barber, Gilat-Schmidt, Pan, "Three material decomposition
 * for spectral computed tomography enabled by block-diagonal
 * step-preconditioning" (arXiv:1801.06263), Sec. 2.  Notation:
 *   f_{k,m}   material maps, pixel k = iy * n + ix, material m = 0 (PMMA), 1 (Al), 2 (Gd)
 *   l         ray (view v, detector bin b), l = v * n_bins + b
 *   w         energy window: W = 4 windows (the paper's overlapping realistic
 *             responses, Sec. 3) or W = 5 (the ideal non-overlapping responses
 *             of the earlier one-step work that Sec. 1 contrasts them with)
 *   X_{l,k}   length (mm) of ray l inside pixel k
 *   c^_{w,l}  counts model N_{w,l} sum_i s_{w,l,i} softexp(-sum_{m,k} mu_{m,i} X_{l,k} f_{k,m})  (Eq. finalModel)
 *   D_TPL     transmission-Poisson Kullback-Leibler data discrepancy                        (Eq. DTPL)
 *
 * Conventions for every entry point:
 *   - The return value is an osscir_status; 0 is success, negative is an error;
 *     no call aborts the process.
 *   - Arguments documented as "device" are device pointers that the CALLER owns
 *     (for example PyTorch tensors); they must stay valid until the enqueued
 *     work finishes.  Arguments documented as "host" are read during the call
 *     and copied; the caller may free them on return.
 *   - Work on device pointers is enqueued on the given stream (0 = the legacy
 *     default stream) and is asynchronous unless stated.  The context must be
 *     used from one host thread at a time.
 *   - Every float4-shaped array is `float[count][4]`, 16-byte aligned, with the
 *     three materials (or four windows) in the first components.
 *   - Per-ray window arrays (counts c and c^, the dual y) are `float[L][WS]`,
 *     16-byte aligned, with WS = 4 for four windows and WS = 8 for five: the
 *     windows in the first W components, the rest padding (ignored on input,
 *     written as zero on output).  Written "float[L][WS]" below.
 */
#ifndef OSSCIR_H_
#define OSSCIR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int osscir_status;
#define OSSCIR_OK 0
#define OSSCIR_E_INVALID (-1)  /* an argument failed validation                          */
#define OSSCIR_E_NOMEM (-2)    /* a device or host allocation failed                      */
#define OSSCIR_E_CUDA (-3)     /* a CUDA call or kernel launch failed                     */
#define OSSCIR_E_TIMEOUT (-4)  /* osscir_poll: the request is still running               */
#define OSSCIR_E_DIVERGED (-5) /* a solve produced a non-finite D_TPL                     */
#define OSSCIR_E_BUSY (-6)     /* admission refused: memory budget or slots exhausted     */
#define OSSCIR_E_NOTFOUND (-7) /* unknown ticket                                          */

typedef struct osscir_ctx *osscir_t;

/* Fan-beam geometry with a flat detector (Sec. 3 names a bench-top system; the
 * geometry itself is not given in the paper).  Image: n x n square pixels of side
 * pixel_mm centred on the rotation axis, pixel (ix, iy) covering
 * [x0 + ix h, x0 + (ix+1) h) x [x0 + iy h, x0 + (iy+1) h), x0 = -n h / 2.
 * View v: source angle start_deg + v * arc_deg / n_views (counter-clockwise),
 * source at distance sid_mm from the axis, detector line at distance sdd_mm from
 * the source, bin b centred at (b - (n_bins-1)/2) * bin_mm.  Requires
 * sid_mm > n * pixel_mm / sqrt(2) (the source outside the image) and sdd_mm > sid_mm. */
typedef struct {
    int n;
    double pixel_mm;
    int n_views;
    double arc_deg, start_deg;
    int n_bins;
    double bin_mm, sid_mm, sdd_mm;
} osscir_geometry;

/* Normalised spectral response and incident photons of Eq. (fullModel) over W
 * windows (W = n_windows; 0 means 4):
 *   s  host float[n_bins][n_energies][W]: s_{w,b,i} >= 0 with sum_i s_{w,b,i} = 1 (within 1e-4)
 *   N  host float[n_bins][W]:             N_{w,b} > 0 (photons per ray and window)
 * The response depends on the detector bin, not on the view.  W = 5 is taken by
 * the single-solve entry points; the batched and served forms and nested
 * solves (inner > 1) take four windows only (OSSCIR_E_INVALID otherwise). */
typedef struct {
    int n_energies; /* 1 .. 256 */
    const float *s;
    const float *N;
    int n_windows;  /* 0 or 4: four windows; 5: five */
} osscir_spectra;

/* Solver parameters.  lambda is the step-size ratio of the step-preconditioner
 * (Sec. 2 leaves it to tuning).  model = 0 uses the per-ray Hessian of Sec. 2 with
 * its negative eigenvalues removed as the curvature of the local quadratic;
 * model = 1 uses zero curvature (a preconditioned gradient step); model = 2 the
 * Hessian's first term alone, sum_w c_w alpha_w alpha_w^T (Gauss-Newton: the
 * term weighted by the residual is dropped, so no eigenvalue is negative);
 * model = 3 the separable W = diag(c) on the window line integrals (equal to
 * model 2's curvature on the range of K).  Models 2 and 3 are readings of the
 * local quadratic that Sec. 2 defers to Barber et al. 2016.  use_box = 1
 * constrains every iterate to lo <= f <= hi per material (the convex constraint
 * set of the one-step framework, Sec. 1); bounds may be infinite, so lo = 0,
 * hi = +inf is nonnegativity; 0 leaves f unconstrained (Sec. 2: the softexp
 * model avoids the need for constraints).  spc = 0 selects the
 * m-block-diagonal step-preconditioner of Sec. 2; spc = 1 the diagonal one of
 * Pock and Chambolle that it replaces (Sigma_wl = (1/lambda) / sum_mk |K|,
 * T_mk = lambda / sum_wl |K|, Sec. 2); spc = 2 the mu-PC of Sec. 1 and 2: the
 * library changes the material basis to one whose attenuation curves are
 * orthonormal over the energy grid (Euclidean inner product; the symmetric
 * choice M = (mu mu^T)^(-1/2), computed in FP64 at creation, mu' = M mu),
 * iterates with the diagonal SPC on f' = M^-1 f, and returns maps in the
 * caller's basis (f = M f') from osscir_get_maps, osscir_reconstruct and the
 * served form; osscir_simulate takes maps in the caller's basis, while the
 * solver state of osscir_get_state / osscir_set_state stays in the iteration's
 * basis.  mu mu^T singular to working precision is OSSCIR_E_INVALID.  counts_model = 0 is
 * the softexp counts model of Eq. (finalModel); counts_model = 1 the standard
 * model of Eq. (fullModel) with exp for every energy (the paper's softexp
 * replaces it so that negative line integrals do not make the counts blow up);
 * it applies to osscir_simulate and osscir_dtpl as well as to the iteration.
 * inner = k > 1 (at most 1e6; 0 means 1) runs the nested inner/outer form that
 * Sec. 3 mentions and sets aside: one outer iteration, the single-loop
 * iteration, builds each ray's local convex model (alpha, the clipped Hessian,
 * the residual r, Sigma^-1 and g0 = X xbar) and keeps it; the next k - 1 inner
 * iterations are primal-dual steps on that fixed model (the dual prox at
 * u = y + Sigma alpha (X xbar - g0); the stored alpha in K and in T), without
 * evaluating the spectral model.  k = 1 is the single-loop method.  Nested
 * solves are stepped with osscir_mocca_step only (not in a batch or server). */
typedef struct {
    double lambda;
    int model;
    int use_box;
    float lo[3], hi[3];
    int spc;
    int counts_model;
    int inner;
} osscir_params;

/* Human-readable name of a status code (static string). */
const char *osscir_status_string(osscir_status s);

/* Create a reconstruction context on the current CUDA device (Sec. 2, the data
 * model's fixed inputs: geometry X, spectra s and N, attenuation mu).
 *   geom, spectra, params: host structs, copied.
 *   mu: host float[3][n_energies], mu_{m,i} in 1/mm per unit of f (Eq. matdecomp), finite
 *       (a transformed basis such as mu-PC's may be negative), copied.
 *   out: receives the handle.
 * Builds the per-geometry ray tables and footprint tables on the device and
 * synchronises before returning.  Errors: OSSCIR_E_INVALID (geometry outside
 * its limits, non-finite or negative inputs, sum_i s != 1), OSSCIR_E_NOMEM,
 * OSSCIR_E_CUDA.  On error *out is NULL and nothing is leaked. */
osscir_status osscir_create(const osscir_geometry *geom, const osscir_spectra *spectra, const float *mu,
                            const osscir_params *params, osscir_t *out);

/* Release every device and host resource of the context (synchronises). NULL is a no-op. */
osscir_status osscir_destroy(osscir_t h);

/* Sizes of the context: pixels P = n*n, rays L = n_views*n_bins, and the
 * number of footprint pairs decided in FP64 (any pointer may be NULL). */
osscir_status osscir_info(osscir_t h, int *n_pixels, int *n_rays, int *n_fp64_pairs);

/* Device memory held by the context (host size_t, either pointer may be NULL):
 * device_bytes all of it, table_bytes the part taken by the footprint tables,
 * which the context builds before its first iteration (0 before that, and 0 if
 * the device had no room for them: the projections are then recomputed every
 * iteration, with the same results).  The paper has no counterpart. */
osscir_status osscir_memory(osscir_t h, size_t *device_bytes, size_t *table_bytes);

/* Forward projection g_l = sum_k X_{l,k} x_k of four channels (the X of Eq. fullModel).
 *   x: device float[P][4] (input), g: device float[L][4] (output). */
osscir_status osscir_forward(osscir_t h, const float *x, float *g, void *stream);

/* Back-projection (the adjoint X^T) img_k = sum_l X_{l,k} rf_l of four channels.
 *   rf: device float[L][4] (input), img: device float[P][4] (output). */
osscir_status osscir_backproject(osscir_t h, const float *rf, float *img, void *stream);

/* Expected counts c^(f) of Eq. (finalModel) for material maps f.
 *   f: device float[P][4] (first three components used), chat: device float[L][WS] (output). */
osscir_status osscir_simulate(osscir_t h, const float *f, float *chat, void *stream);

/* Load measured counts c_{w,l} (Eq. DTPL) and reset the solver state to
 * x_0 = xbar_0 = 0, y_0 = 0, iteration 0.
 *   c: device float[L][WS], c >= 0 and finite (copied on the stream).
 * The counts are checked on the device, on the stream, after the copy; the
 * call itself does not wait for the check.  The next osscir_dtpl returns
 * OSSCIR_E_INVALID if any count was negative or not finite (the iterations in
 * between run on those counts and their results are meaningless). */
osscir_status osscir_set_counts(osscir_t h, const float *c, void *stream);

/* Run n_iters MOCCA iterations (Sec. 1: local convex quadratic, removal of
 * negative curvature, one preconditioned CPPD step; Sec. 2: the m-block-diagonal
 * Sigma and T).  Library-owned state; asynchronous on the stream.  With
 * params.inner = k > 1 the iterations continue the nested cycle across calls:
 * the first after osscir_create, osscir_set_counts, osscir_set_state or
 * osscir_reconstruct is an outer one, then every k-th. */
osscir_status osscir_mocca_step(osscir_t h, int n_iters, void *stream);

/* One MOCCA iteration split by views, for one solve shared by several GPUs
 * (the forward and back-projections, which Sec. 1 and 2 name as the cost, are
 * sums over rays, so the rays can be partitioned).  Every GPU holds a context
 * of the same problem (geometry, spectra, mu, parameters, counts) in the same
 * state.  osscir_mocca_partial runs the ray side of the iteration for the rays
 * of the views [v0, v1) only: the forward projection at xbar, the counts model,
 * the clipped curvature and the dual step (updating the duals of those rays),
 * then back-projects those rays' nine per-pixel channels, K^T y' and the block
 * step matrix P_k (T^-1_k = P_k / lambda), into chan.  It does not change the
 * maps.  The caller sums chan over a partition of the views into ranges (one
 * all-reduce of 9 P floats per iteration); osscir_mocca_apply then takes every
 * pixel's primal step (the 3x3 solve of the m-block SPC, the optional box,
 * the extrapolation) from the summed channels and counts the iteration.  With
 * the views of all ranges summed, the iterates equal osscir_mocca_step's up to
 * the order of the floating-point additions.
 *   v0, v1: 0 <= v0 < v1 <= n_views;
 *   chan:   device float[9][P] (channel-major: channels 0-2 K^T y' for the three
 *           materials, 3-8 P_k packed as 00 01 02 11 12 22), written by partial,
 *           read by apply.
 * Asynchronous on the stream.  After osscir_mocca_partial, osscir_dtpl(h, 1)
 * returns the D_TPL terms of the rays of [v0, v1) only (the ranges' values add
 * up to the whole).  Errors: OSSCIR_E_INVALID (bad range, NULL chan, a nested
 * solve: inner > 1), OSSCIR_E_CUDA. */
osscir_status osscir_mocca_partial(osscir_t h, int v0, int v1, float *chan, void *stream);
osscir_status osscir_mocca_apply(osscir_t h, const float *chan, void *stream);

/* End-to-end reconstruction with host buffers: copies the counts c (host
 * float[L][WS], c >= 0; pinned memory makes the copy asynchronous DMA) to the
 * device, resets the state as osscir_set_counts does, runs n_iters MOCCA
 * iterations and copies the maps x_n to maps_out (host float[P][4]).
 * Synchronises the stream before returning.  Errors: OSSCIR_E_INVALID (NULL
 * arguments, n_iters < 0, or a count that is negative or not finite, checked
 * on the host before anything is enqueued), OSSCIR_E_DIVERGED (the D_TPL of
 * the last iteration is not finite; maps_out holds the non-finite maps),
 * OSSCIR_E_CUDA. */
osscir_status osscir_reconstruct(osscir_t h, const float *c_host, int n_iters, float *maps_out_host,
                                 void *stream);

/* Device time of the last MOCCA iteration's three main kernels, measured with
 * CUDA events recorded inside the iteration's graph (host float[3]): ms[0]
 * the ray-driven forward projection, ms[1] the per-ray spectral model,
 * curvature and dual step (after an inner iteration of a nested solve: its dual
 * step on the kept models), ms[2] the pixel-driven back-projection, block
 * step-preconditioner and primal step.  Synchronises the stream. */
osscir_status osscir_last_kernel_ms(osscir_t h, float *ms, void *stream);

/* Copy the current material maps x_n to x_out: device float[P][4] (in the
 * caller's material basis; see spc = 2). */
osscir_status osscir_get_maps(osscir_t h, float *x_out, void *stream);

/* Checkpoint / resume of the solver state (x_n, xbar_n, y_n, n).  All arrays
 * are device pointers: x, xbar float[P][4], y float[L][WS].  get copies out,
 * set copies in; resuming from a saved state reproduces the uninterrupted
 * iterates bit for bit.  iter: host int.  The kept local models of a nested
 * solve are not part of the state: the first iteration after set is an outer one. */
osscir_status osscir_get_state(osscir_t h, float *x, float *xbar, float *y, int *iter, void *stream);
osscir_status osscir_set_state(osscir_t h, const float *x, const float *xbar, const float *y, int iter,
                               void *stream);

/* D_TPL (Eq. DTPL) of the loaded counts: which = 0 evaluates it at the current
 * maps x_n (one extra forward projection); which = 1 returns the value the last
 * iteration computed at its expansion point xbar (for a nested solve, the last
 * outer iteration: inner iterations do not evaluate the counts model).
 * Synchronises the stream; out: host double.  Errors: OSSCIR_E_INVALID also
 * when the counts loaded by the last osscir_set_counts failed its check;
 * OSSCIR_E_DIVERGED when the value is not finite. */
osscir_status osscir_dtpl(osscir_t h, int which, double *out, void *stream);

/* Footprint dumps for verification: for rays [l0, l0+n) (or pixels [k0, k0+n))
 * the pixels (rays) with nonzero X_{l,k} as the forward (back-)projection uses
 * them, and their weights.  cnt: device int[n]; idx: device int[n][cap];
 * wt: device float[n][cap]; entries beyond cap are counted but not stored
 * (with cap = 0 only the counts are written and idx, wt may be NULL). */
osscir_status osscir_footprint_rays(osscir_t h, int l0, int n, int cap, int *cnt, int *idx, float *wt,
                                    void *stream);
osscir_status osscir_footprint_pixels(osscir_t h, int k0, int n, int cap, int *cnt, int *idx, float *wt,
                                      void *stream);

/* Seeded Poisson noise: c[i] ~ Poisson(chat[i]) for i < n, the noise of the
 * paper's simulated data (Sec. 3), drawn on the device without a context.
 * chat, c: device float[n] (for example [L][4] counts, n = 4 L); chat >= 0
 * (0, negative or NaN means give 0); counts are exact below 2^24.  Sample i
 * depends only on (seed, i, chat[i]): uniforms from Philox4x32-10 (Salmon et
 * al. 2011) at counter (i, t, 0, 0) under key (seed mod 2^32, seed / 2^32);
 * means below 10 by inversion, larger by the transformed rejection of Hormann
 * (1993).  Asynchronous on stream.  Errors: OSSCIR_E_INVALID (n < 0, NULL
 * buffers), OSSCIR_E_CUDA. */
osscir_status osscir_poisson_noise(const float *chat, int n, uint64_t seed, float *c, void *stream);

/* ------------------------------------------------------------------ batched form
 * Many independent solves, each its own context (any geometry, spectra, mu,
 * parameters; counts loaded with osscir_set_counts), advanced together: each
 * MOCCA step of the batch is one launch per kernel over a work list of
 * (solve, tile) items from all solves, captured once as one CUDA graph.  The
 * MOCCA iteration of Sec. 2 is unchanged: every solve's iterates, D_TPL and
 * iteration count are bit-identical to what osscir_mocca_step gives the same
 * context alone, for any batch composition and any configuration below.
 *
 * The batch refers to its contexts; they must outlive it and must not be
 * stepped on their own or destroyed while it exists.  Counts and state may be
 * reloaded (osscir_set_counts, osscir_set_state) between batch steps, in
 * stream order.  Per-solve results are read with the per-context calls
 * (osscir_get_maps, osscir_get_state, osscir_dtpl(h, 1, ...)). */
typedef struct osscir_batch *osscir_batch_t;

/* Launch configuration of a batch (the paper has no counterpart: it sets how
 * work is spread over the GPU, never what is computed).
 *   proj_views:  views per projection block (1, 2, 4 or 8; 32 bins each);
 *   proj_grid, ray_grid, bp_grid: 0 = one CTA per work item (flat grid),
 *                > 0 = that many persistent CTAs striding over the items;
 *   bp_tile_x:   width of the 64-pixel back-projection tile (2, 4, 8, 16 or 32);
 *   *_order:     work-list order of each kernel: 0 solve by solve, 1 the
 *                solves with the costliest items first, 2 solves interleaved
 *                item by item;
 *   branches:    1, 2 or 4 (at most the number of solves): the solves are
 *                split into that many groups of about equal work, each with
 *                its own launches, as parallel branches of the iteration graph
 *                (so one group's projection can overlap another's per-ray
 *                step). */
typedef struct {
    int proj_views;
    int proj_grid;
    int proj_order;
    int ray_grid;
    int ray_order;
    int bp_tile_x;
    int bp_grid;
    int bp_order;
    int branches;
} osscir_batch_config;

/* Build a batch over n (1 .. 4096) distinct contexts of the current device
 * (synchronises the device first).  autotune = 0 takes the default
 * configuration; autotune = 1 times candidate configurations on the batch
 * itself (a few launches each, restoring every solve's state afterwards) and
 * keeps the fastest.  Errors:
 * OSSCIR_E_INVALID (NULL or repeated handles, contexts of another device),
 * OSSCIR_E_NOMEM, OSSCIR_E_CUDA. */
osscir_status osscir_batch_create(const osscir_t *solves, int n, int autotune, osscir_batch_t *out);

/* Release the batch (not its contexts; synchronises).  NULL is a no-op. */
osscir_status osscir_batch_destroy(osscir_batch_t b);

/* Enqueue n_iters (>= 0) MOCCA iterations of every solve on stream. */
osscir_status osscir_batch_step(osscir_batch_t b, int n_iters, void *stream);

/* The configuration in use; set replaces it (validated as documented above,
 * else OSSCIR_E_INVALID) and rebuilds the work lists and the graph (it
 * synchronises the device first). */
osscir_status osscir_batch_get_config(osscir_batch_t b, osscir_batch_config *out);
osscir_status osscir_batch_set_config(osscir_batch_t b, const osscir_batch_config *cfg);

/* Device time (ms) of the projection, ray and back-projection launches of
 * the last batch iteration enqueued on stream (synchronises the stream); with
 * several branches, those of the first branch. */
osscir_status osscir_batch_last_kernel_ms(osscir_batch_t b, float ms[3], void *stream);

/* ------------------------------------------------------------------ served form
 * A server owns a worker thread and a stream on the device that is current
 * when it is created.  Requests (complete reconstruction problems with host
 * data) are queued by osscir_submit and admitted while a slot is free and the
 * device memory of all cached contexts stays within the budget.  Admitted
 * requests are spread over up to four groups of about equal work; each group
 * advances all its requests together, a few MOCCA iterations per round,
 * through the batched kernels (one launch per kernel per iteration for the
 * group) on its own stream, and the groups run side by side.  A group's batch
 * is re-formed between its rounds, so requests that arrive while others are on
 * the GPU join at the next round and finished ones leave (continuous
 * batching).  Contexts of finished requests stay cached and are reused by later
 * requests with the same geometry, spectra, mu and parameters; the least
 * recently used idle ones are released when memory is needed.  A request's
 * result does not depend on what else runs: it equals the plain form's bit for
 * bit. */
typedef struct osscir_server *osscir_server_t;

typedef struct {
    osscir_geometry geom;
    osscir_spectra spectra; /* host arrays, copied at submit */
    const float *mu;        /* host float[3][n_energies], copied at submit */
    osscir_params params;
    const float *counts;    /* host float[L][4], measured counts c >= 0, copied at submit */
    int n_iters;            /* MOCCA iterations from x_0 = 0 */
} osscir_request;

typedef struct {
    osscir_status status; /* OSSCIR_OK, OSSCIR_E_DIVERGED (non-finite D_TPL) or an error */
    int iterations;
    double dtpl;          /* D_TPL at the last expansion point */
    double latency_ms;    /* submit to result ready (host clock) */
    double queue_ms;      /* submit to work enqueued on the GPU */
    double gpu_ms;        /* device time from its first work to its results (the
                             rounds it shares with other requests included) */
} osscir_stats;

/* Create a server.  hbm_budget_bytes: device memory the server's contexts may
 * hold; max_slots: requests running at once (1 .. 256). */
osscir_status osscir_server_create(size_t hbm_budget_bytes, int max_slots, osscir_server_t *out);

/* Stop the server: queued requests are dropped, running ones finish, every
 * resource is released (synchronises). NULL is a no-op. */
osscir_status osscir_server_destroy(osscir_server_t s);

/* Queue a request; *ticket identifies it.  Errors: OSSCIR_E_INVALID (as
 * osscir_create, or counts < 0 / non-finite, n_iters < 0), OSSCIR_E_BUSY (the
 * request alone needs more device memory than the budget). */
osscir_status osscir_submit(osscir_server_t s, const osscir_request *req, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: no limit) for a request.  When done, copies the
 * maps x_n to maps_out (host float[P][4], may be NULL), fills stats (may be
 * NULL), forgets the ticket and returns the request's status.  Returns
 * OSSCIR_E_TIMEOUT if it is still queued or running (the ticket stays valid)
 * and OSSCIR_E_NOTFOUND for an unknown ticket. */
osscir_status osscir_poll(osscir_server_t s, uint64_t ticket, int timeout_ms, float *maps_out, osscir_stats *stats);

/* Requests running and queued, and device bytes held by the server's contexts
 * (any pointer may be NULL). */
osscir_status osscir_server_info(osscir_server_t s, int *running, int *queued, size_t *bytes_in_use);

/* The transmission-Poisson data discrepancy of expected counts chat against
 * measured counts c, computed without allocating any memory and without a
 * context.  The paper has no
 * counterpart: this serves callers that must not call cudaMalloc after
 * start-up, for example a server whose memory arena claims the device at
 * launch, or a latency-bound loop that cannot accept the synchronisation an
 * allocation may cause; osscir_dtpl needs a context, and creating one allocates.
 *   chat, c: device float[n_rays][4];  out: device double (written on the stream).
 *   n_rays: 1 .. 4,194,304 (larger values return OSSCIR_E_INVALID).
 *   Five-window arrays float[L][8] pass as n_rays = 2 L when their padding is
 *   zero (a term with c = c^ = 0 is zero).
 * Scratch: a fixed 128 KiB array of per-block partial sums inside the library's
 * device memory, held by every GPU that loads the library until the process
 * exits.  The first call on a device looks up that array's device address (with
 * the device current); make that first call before any stream capture.  Every
 * call overwrites the partials it reads, so nothing carries over between calls,
 * but all calls share the one array: calls that overlap on the GPU (different
 * streams, or different host threads on the same device) race and give wrong
 * results; serialise them on one stream. */
osscir_status osscir_dtpl_counts_static(const float *chat, const float *c, int n_rays, double *out,
                                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OSSCIR_H_ */
