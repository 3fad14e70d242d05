// Per-iteration kernels of MOCCA with the m-block-diagonal SPC (Sec. 2) and the
// plain projectors behind osscir_forward / osscir_backproject / osscir_simulate.
//
// One iteration is three launches (plus a tiny deterministic reduction):
//   k_mocca_proj (ray-driven):  g = X xbar for the three maps;
//   k_mocca_ray (per ray):      the counts model
//       of Eq. (finalModel) summed over energies (compensated), D_TPL of
//       Eq. (DTPL), alpha_w = sum_i A_wi mu_i (K = alpha X, Eq. aeq), the per-ray
//       Hessian of Sec. 2 in g with its negative eigenvalues removed (FP64, for
//       the Hessians that are not positive definite), the dual step matrix
//       Sigma^-1 = lambda |alpha_w| (X 1)_l, the exact preconditioned dual prox
//       y' = y - Sigma (W + Sigma)^-1 (y - r) (taken in an orthonormal basis of
//       the range of alpha, see ray_dual), and the per-ray products b = alpha^T y'
//       and S = sum_w alpha_w alpha_w^T / |alpha_w|.
//   k_mocca_bp (pixel-driven):  v_k = sum_l X_lk b_l (= K^T y') and
//       P_k = sum_l X_lk S_l (so T^-1_k = P_k / lambda, the m-block SPC), the
//       3x3 solve (double-float), the primal step (optionally onto a box) and the
//       extrapolation xbar' = 2 x' - x.
#include "osscir_internal.cuh"
#include "osscir_launch.h"

namespace osscir {
namespace {

constexpr int kMaxEnergies = 256;
constexpr int kSmemStride = 12;   // per energy: mu0 mu1 mu2 | m00 m01 m02 m11 m12 m22 | pad
constexpr int kDFold = 16;        // energies per plain FP32 partial of D_w

__device__ __forceinline__ void neumaier(float& s, float& c, float t) {
    const float u = s + t;
    c += (fabsf(s) >= fabsf(t)) ? ((s - u) + t) : ((t - u) + s);
    s = u;
}

// One term of Eq. (DTPL), c^ - c - c log(c^/c) = c (u - log(1 + u)) with
// u = (c^ - c) / c; a series is used for small |u| (cancellation), c = 0 gives c^.
__device__ __forceinline__ float dtpl_term(float chat, float c) {
    if (!(c > 0.0f)) return chat;
    const float u = (chat - c) / c;
    if (fabsf(u) < 0.0625f) {
        const float p = 0.5f - u * (1.0f / 3.0f - u * (0.25f - u * (0.2f - u * (1.0f / 6.0f - u * (1.0f / 7.0f - u * 0.125f)))));
        return c * u * u * p;
    }
    return chat - c - c * logf(chat / c);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// Ray-driven kernels give each warp 32 consecutive detector bins (one per lane)
// of one view, and a block vb consecutive views (one per warp), so the block's
// slice of the energy-major spectral table is shared by its warps.  (bx, by)
// is the block's tile: bins [32 bx, 32 bx + 32), views [vb by, vb by + vb).
__device__ __forceinline__ int warp_view(int by, int vb) { return by * vb + (threadIdx.x >> 5); }

__device__ __forceinline__ int ray_at(const GeomC& C, int bx, int by, int vb) {
    const int b = bx * 32 + (threadIdx.x & 31);
    const int v = warp_view(by, vb);
    return (b < C.n_bins && v < C.n_views) ? v * C.n_bins + b : -1;
}

__device__ __forceinline__ int ray_of_thread(const GeomC& C) {
    return ray_at(C, blockIdx.x, blockIdx.y, kFwdThreads / 32);
}

// The same tiling over the views [v0, v1) only: view v0 + (by vb + warp).
__device__ __forceinline__ int ray_in_views(const GeomC& C, int bx, int by, int vb, int v0, int v1) {
    const int b = bx * 32 + (threadIdx.x & 31);
    const int v = v0 + warp_view(by, vb);
    return (b < C.n_bins && v < v1) ? v * C.n_bins + b : -1;
}

// The warp's D_TPL partial, stored at (view, 32-bin group) whatever the block
// shape, so the fixed-order reduction sees the same sequence for any tiling.
__device__ __forceinline__ void warp_partial(const GeomC& C, int bx, int v, double val, double* part,
                                             int v_end = -1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
    if ((threadIdx.x & 31) == 0 && v < (v_end < 0 ? C.n_views : v_end)) part[v * ((C.n_bins + 31) >> 5) + bx] = val;
}

__device__ __forceinline__ void load_mu_smem(const SpecD& S, float* sm) {
    const int nE = S.n_energies;
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        const float m0 = S.mu[i], m1 = S.mu[nE + i], m2 = S.mu[2 * nE + i];
        float* q = sm + kSmemStride * i;
        q[0] = m0; q[1] = m1; q[2] = m2;
        q[3] = m0 * m0; q[4] = m0 * m1; q[5] = m0 * m2;
        q[6] = m1 * m1; q[7] = m1 * m2; q[8] = m2 * m2;
        q[9] = q[10] = q[11] = 0.f;
    }
}

// softexp(x), softexp'(x), softexp''(x) (Sec. 2): exp below 0, x + 1 above;
// with expm the standard model's exp everywhere (Eq. fullModel).
__device__ __forceinline__ void sexp3(float x, bool expm, float& e0, float& e1, float& e2) {
    if (x <= 0.0f || expm) {
        e0 = expf(x);
        e1 = e0;
        e2 = e0;
    } else {
        e0 = x + 1.0f;
        e1 = 1.0f;
        e2 = 0.0f;
    }
}

// Back-projection table entries are read once per iteration: streaming loads
// that allocate no L1 line (measured about 2 % faster at 256x256 and 1 % at
// 512x512; the forward table's entries loaded so were 10 % slower and keep
// ordinary loads).
__device__ __forceinline__ float2 ld_stream(const float2* p) {
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ ushort2 ld_stream(const ushort2* p) {
    unsigned u;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(u) : "l"(p));
    return make_ushort2((unsigned short)(u & 0xffffu), (unsigned short)(u >> 16));
}

// Half of a ray record (32 bytes, 32-byte aligned) in one 256-bit load.
struct RecHalf {
    float4 a, b;
};
__device__ __forceinline__ RecHalf ldg_half(const float4* p) {
    RecHalf r;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r.a.x), "=f"(r.a.y), "=f"(r.a.z), "=f"(r.a.w), "=f"(r.b.x), "=f"(r.b.y), "=f"(r.b.z), "=f"(r.b.w)
        : "l"(p));
    return r;
}

template <class Visit>
__device__ __forceinline__ void ray_pixels(const GeomC& C, const ExcTable& E, const float4& r0, float ex, float ey,
                                           int l, Visit&& visit) {
    ray_weights(r0, ex, ey, C.grid, C.margin_mm, E, l, visit);
}

template <class Visit>
__device__ __forceinline__ void pixel_rays(const GeomC& C, const ExcTable& E, const RayRec* rec,
                                           const ViewF* views, int ix, int iy, Visit&& visit) {
    for (int v = 0; v < C.n_views; ++v) {
        int blo, bhi;
        pixel_bin_range(C, views[v], ix, iy, blo, bhi);
        for (int b = blo; b <= bhi; ++b) {
            const int l = v * C.n_bins + b;
            const float4 r0 = __ldg(&rec[l].r0);
            const float4 r1 = __ldg(&rec[l].r1);
            const float w = x_weight(r0, r1.x, r1.y, C.grid, E, l, ix, iy);
            if (w != 0.0f) visit(l, w, r1);
        }
    }
}

// Line sums of the interleaved maps along one ray, summed in two levels: an FP32
// partial over at most kFold pixels is folded into the running total.  The rounding
// error then grows with kFold + n / kFold terms instead of n (about 700 pixels per
// ray at 512 x 512), which keeps the counts model within 1e-5 relative even on the
// most attenuated rays.
constexpr int kFold = 16;
struct LineSum {
    float4 part = make_float4(0.f, 0.f, 0.f, 0.f), total = make_float4(0.f, 0.f, 0.f, 0.f);
    int n = 0;
    __device__ __forceinline__ void add(float w, const float4& v) {
        part.x = fmaf(w, v.x, part.x);
        part.y = fmaf(w, v.y, part.y);
        part.z = fmaf(w, v.z, part.z);
        part.w = fmaf(w, v.w, part.w);
        if (++n == kFold) {
            total.x += part.x, total.y += part.y, total.z += part.z, total.w += part.w;
            part = make_float4(0.f, 0.f, 0.f, 0.f);
            n = 0;
        }
    }
    __device__ __forceinline__ float4 sum() const {
        return make_float4(total.x + part.x, total.y + part.y, total.z + part.z, total.w + part.w);
    }
};

// ------------------------------------------------------------------ plain projectors

__global__ void __launch_bounds__(kFwdThreads) k_forward4(GeomC C, ExcTable E, const RayRec* rec, const float4* x,
                                                          float4* g) {
    const int l = ray_of_thread(C);
    if (l < 0) return;
    const float4 r0 = rec[l].r0, r1 = rec[l].r1;
    LineSum acc;
    ray_pixels(C, E, r0, r1.x, r1.y, l, [&](int k, float w) { acc.add(w, __ldg(x + k)); });
    g[l] = acc.sum();
}

__global__ void k_backproject4(GeomC C, ExcTable E, const RayRec* rec, const ViewF* views, const float4* rf,
                               float4* img) {
    const int ix = blockIdx.x * kBpTileX + threadIdx.x, iy = blockIdx.y * kBpTileY + threadIdx.y;
    if (ix >= C.grid.n || iy >= C.grid.n) return;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    pixel_rays(C, E, rec, views, ix, iy, [&](int l, float w, const float4&) {
        const float4 v = __ldg(rf + l);
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
        acc.z = fmaf(w, v.z, acc.z);
        acc.w = fmaf(w, v.w, acc.w);
    });
    img[iy * C.grid.n + ix] = acc;
}

// c^(f) (Eq. finalModel) for every ray; with c != nullptr also the D_TPL block partials.
// W windows; chat and c hold win_f4<W>() float4 per ray.
template <int W>
__global__ void __launch_bounds__(kFwdThreads) k_counts(GeomC C, ExcTable E, const RayRec* rec, SpecD S,
                                                        const float4* f, float4* chat, const float4* c,
                                                        double* part) {
    constexpr int F4 = win_f4<W>();
    __shared__ float sm[kSmemStride * kMaxEnergies];
    load_mu_smem(S, sm);
    __syncthreads();
    const int l = ray_of_thread(C);
    double dsum = 0.0;
    if (l >= 0) {
        const float4 r0 = rec[l].r0, r1 = rec[l].r1;
        LineSum acc;
        ray_pixels(C, E, r0, r1.x, r1.y, l, [&](int k, float w) { acc.add(w, __ldg(f + k)); });
        const float4 gs = acc.sum();
        const float g0 = gs.x, g1 = gs.y, g2 = gs.z;
        const int b = l % C.n_bins, nb = C.n_bins;
        float Ds[W], Dc[W];
#pragma unroll
        for (int w = 0; w < W; ++w) Ds[w] = Dc[w] = 0.f;
        for (int i = 0; i < S.n_energies; ++i) {
            const float* q = sm + kSmemStride * i;
            const float p = fmaf(q[2], g2, fmaf(q[1], g1, q[0] * g0));
            float e0, e1, e2;
            sexp3(-p, S.exp_model != 0, e0, e1, e2);
            float sv[W];
            win_load<W, true>(S.s4 + F4 * ((size_t)i * nb + b), sv);
#pragma unroll
            for (int w = 0; w < W; ++w) neumaier(Ds[w], Dc[w], sv[w] * e0);
        }
        float Nv[W], ch[W];
        win_load<W, true>(S.N4 + F4 * b, Nv);
#pragma unroll
        for (int w = 0; w < W; ++w) ch[w] = Nv[w] * (Ds[w] + Dc[w]);
        if (chat) win_store<W>(chat + F4 * (size_t)l, ch);
        if (c) {
            float cv[W];
            win_load<W>(c + F4 * (size_t)l, cv);
#pragma unroll
            for (int w = 0; w < W; ++w) dsum += (double)dtpl_term(ch[w], cv[w]);
        }
    }
    if (part) warp_partial(C, blockIdx.x, warp_view(blockIdx.y, kFwdThreads / 32), dsum, part);
}

// ------------------------------------------------------------------ double-float arithmetic
//
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2),
// about 48 significant bits, computed on the FP32 pipe: on this GPU the FP64
// pipe runs at 1/64 of the FP32 rate, so for the ill-conditioned parts of the
// dual step and for the pixel step two-float arithmetic is several times
// cheaper than FP64.  The
// error-free transformations are Knuth's TwoSum and Dekker's exact product in
// its FMA form (Dekker 1971); additions are the accurate ("IEEE-style")
// double-word sum of Hida, Li and Bailey (2001), which keeps its accuracy under
// cancellation; the reciprocal is one Newton step from the FP32 reciprocal.
// Every operation is spelled with _rn intrinsics so that the compiler cannot
// contract or reassociate them.
struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_fast2sum(float a, float b) {   // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfl df_2prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    const dfl s = df_2sum(x.hi, y.hi), t = df_2sum(x.lo, y.lo);
    const dfl u = df_fast2sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast2sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, dfl{-y.hi, -y.lo}); }

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const dfl p = df_2prod(x.hi, y.hi);
    return df_fast2sum(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}

__device__ __forceinline__ dfl df_mulf(dfl x, float y) {
    const dfl p = df_2prod(x.hi, y);
    return df_fast2sum(p.hi, __fmaf_rn(x.lo, y, p.lo));
}

__device__ __forceinline__ float df_f(dfl x) { return __fadd_rn(x.hi, x.lo); }

// 1 / x: r + r (1 - x r) with r the FP32 reciprocal of x.hi.
__device__ __forceinline__ dfl df_rcp(dfl x) {
    const float r = __frcp_rn(x.hi);
    const dfl e = df_sub(dfl{1.0f, 0.0f}, df_mulf(x, r));
    return df_add(dfl{r, 0.0f}, df_mulf(e, r));
}

// ------------------------------------------------------------------ FP64 3x3 / 4x4 algebra

// Symmetric 3x3 stored as (00, 01, 02, 11, 12, 22).

// Unit eigenvector of H for the simple eigenvalue lam: the largest cross
// product of two rows of H - lam I.  Returns false if all are (near) zero.
__device__ __forceinline__ bool eigvec3(const double h[6], double lam, double v[3]) {
    const double a00 = h[0] - lam, a11 = h[3] - lam, a22 = h[5] - lam;
    // rows r0 = (a00, h1, h2), r1 = (h1, a11, h4), r2 = (h2, h4, a22)
    const double c0x = fma(h[1], h[4], -h[2] * a11), c0y = fma(h[2], h[1], -a00 * h[4]), c0z = fma(a00, a11, -h[1] * h[1]);
    const double c1x = fma(h[1], a22, -h[2] * h[4]), c1y = fma(h[2], h[2], -a00 * a22), c1z = fma(a00, h[4], -h[1] * h[2]);
    const double c2x = fma(a11, a22, -h[4] * h[4]), c2y = fma(h[4], h[2], -h[1] * a22), c2z = fma(h[1], h[4], -a11 * h[2]);
    const double n0 = fma(c0x, c0x, fma(c0y, c0y, c0z * c0z));
    const double n1 = fma(c1x, c1x, fma(c1y, c1y, c1z * c1z));
    const double n2 = fma(c2x, c2x, fma(c2y, c2y, c2z * c2z));
    double bx = c0x, by = c0y, bz = c0z, best = n0;
    if (n1 > best) { bx = c1x; by = c1y; bz = c1z; best = n1; }
    if (n2 > best) { bx = c2x; by = c2y; bz = c2z; best = n2; }
    const double sc = fabs(h[0]) + fabs(h[3]) + fabs(h[5]) + fabs(h[1]) + fabs(h[2]) + fabs(h[4]) + fabs(lam);
    if (!(best > 1e-60 * sc * sc * sc * sc)) return false;
    const double in = rsqrt(best);
    v[0] = bx * in;
    v[1] = by * in;
    v[2] = bz * in;
    return true;
}

// Cyclic Jacobi, used only when the closed form meets a (near) repeated root.
__device__ void clip_psd3_jacobi(double h[6]) {
    double a[3][3] = {{h[0], h[1], h[2]}, {h[1], h[3], h[4]}, {h[2], h[4], h[5]}};
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 10; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > 1e-30 * dia)) break;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int p = t == 2 ? 1 : 0, q = t == 0 ? 1 : 2, r = 3 - p - q;
            const double apq = a[p][q];
            if (apq == 0.0) continue;
            const double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = rsqrt(1.0 + tt * tt), s = tt * c;
            a[p][p] -= tt * apq;
            a[q][q] += tt * apq;
            a[p][q] = a[q][p] = 0.0;
            const double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double vp = V[i][p], vq = V[i][q];
                V[i][p] = c * vp - s * vq;
                V[i][q] = s * vp + c * vq;
            }
        }
    }
    const double l0 = fmax(a[0][0], 0.0), l1 = fmax(a[1][1], 0.0), l2 = fmax(a[2][2], 0.0);
    const int idx[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int i = idx[e][0], j = idx[e][1];
        h[e] = l0 * V[i][0] * V[j][0] + l1 * V[i][1] * V[j][1] + l2 * V[i][2] * V[j][2];
    }
}


// sqrt of a positive double-float: s = sqrt(hi) corrected by one Newton step,
// s + (x - s^2) / (2 s) (Karp and Markstein 1997), the correction in FP32.
__device__ __forceinline__ dfl df_sqrt(dfl x) {
    const float s = __fsqrt_rn(x.hi);
    const float e = df_f(df_sub(x, df_2prod(s, s)));
    return df_fast2sum(s, __fmul_rn(e, __fdiv_rn(0.5f, s)));
}

__device__ __forceinline__ dfl df_neg(dfl x) { return dfl{-x.hi, -x.lo}; }

// Negative-curvature removal of H (FP64, packed) as its terms: returns 0 if H is
// positive semi-definite (H+ = H), 1 if one eigenvalue is negative (H+ = H - lam
// v v^T), 2 if two are (H+ = lam v v^T, lam the positive one), 3 if all three are
// (H+ = 0), and 4 if the closed form met a near repeated root (H+ in h, by Jacobi).
__device__ int clip_terms(double h[6], double& lam, double v[3]) {
    const double m2 = fma(h[0], h[3], -h[1] * h[1]);
    const double det = fma(h[0], fma(h[3], h[5], -h[4] * h[4]),
                           fma(-h[1], fma(h[1], h[5], -h[4] * h[2]), h[2] * fma(h[1], h[4], -h[3] * h[2])));
    if (h[0] > 0.0 && m2 > 0.0 && det > 0.0) return 0;
    const double p1 = fma(h[1], h[1], fma(h[2], h[2], h[4] * h[4]));
    if (p1 == 0.0) {   // diagonal
        h[0] = fmax(h[0], 0.0);
        h[3] = fmax(h[3], 0.0);
        h[5] = fmax(h[5], 0.0);
        return 4;
    }
    // One negative eigenvalue (det < 0 with a positive diagonal entry, so not all
    // three are negative), the common case: the eigenvalue by Newton steps on the
    // characteristic polynomial p(l) = det(H - l I) = -l^3 + tr l^2 - c2 l + det from
    // l = det / c2 (the eigenvalue itself when it is small against the others).
    // p and p' are FP64 and each step's ratio p / p' FP32, so the iterates settle on
    // the FP64 zero of p; if they do not within eight steps, the closed form below.
    if (det < 0.0 && (h[0] > 0.0 || h[3] > 0.0 || h[5] > 0.0)) {
        const double tr = h[0] + h[3] + h[5];
        const double c2 = fma(h[0], h[3], -h[1] * h[1]) + fma(h[0], h[5], -h[2] * h[2]) + fma(h[3], h[5], -h[4] * h[4]);
        if (c2 > 0.0) {
            double l = (double)__fdiv_rn((float)det, (float)c2);
            bool settled = false;
            for (int it = 0; it < 8 && !settled; ++it) {
                const double p = fma(fma(tr - l, l, -c2), l, det);
                const double dp = fma(fma(-3.0, l, 2.0 * tr), l, -c2);
                const double step = (double)__fdiv_rn((float)p, (float)dp);
                l -= step;
                settled = fabs(step) <= 1e-14 * fabs(l);
            }
            if (settled && l < 0.0) {
                lam = l;
                if (eigvec3(h, lam, v)) return 1;
            }
        }
    }
    const double q = (h[0] + h[3] + h[5]) / 3.0;
    const double a0 = h[0] - q, a3 = h[3] - q, a5 = h[5] - q;
    const double p = sqrt(fma(a0, a0, fma(a3, a3, fma(a5, a5, 2.0 * p1))) / 6.0);
    const double ip = 1.0 / p;
    const double b0 = a0 * ip, b1 = h[1] * ip, b2 = h[2] * ip, b3 = a3 * ip, b4 = h[4] * ip, b5 = a5 * ip;
    double r = 0.5 * fma(b0, fma(b3, b5, -b4 * b4), fma(-b1, fma(b1, b5, -b4 * b2), b2 * fma(b1, b4, -b3 * b2)));
    r = fmin(fmax(r, -1.0), 1.0);
    const double phi = acos(r) / 3.0;
    const double lhi = fma(2.0 * p, cos(phi), q);
    const double llo = fma(2.0 * p, cos(phi + 2.0943951023931954923), q);   // + 2 pi / 3
    const double lmid = 3.0 * q - lhi - llo;
    const int neg = (lhi < 0.0) + (lmid < 0.0) + (llo < 0.0);
    if (neg == 0) return 0;
    if (neg == 3) return 3;
    lam = neg == 1 ? llo : lhi;
    if (!eigvec3(h, lam, v)) {
        clip_psd3_jacobi(h);
        return 4;
    }
    return neg;
}

// Dual step of one ray that meets the image (see the file header).
//   al: window-effective attenuations alpha (FP32), sinv: Sigma^-1 (FP32),
//   cw: counts (FP32, exact), r: residuals (double-float), Bt: sum_i beta_i mu_i mu_i^T
//   with beta_i = softexp''_i sum_w r_w s_wi / D_w (FP32, packed), y: dual.
// With G = (alpha^T alpha)^-1 alpha^T and W = G^T H+ G, the prox
//   y' = y - Sigma (W + Sigma)^-1 (y - r)
// is taken in an orthonormal basis of the range of alpha.  With R the Cholesky
// factor of alpha^T alpha (R^T R = alpha^T alpha, upper triangular) and
// Q = alpha R^-1 (orthonormal columns), W = Q M Q^T with M = R^-T H+ R^-1, and by
// the push-through identity y' = r + Q z, (I + M S) z = M Q^T Sigma^-1 (y - r),
// S = Q^T Sigma^-1 Q.  alpha^T alpha has a condition number near 1e7, so it, R
// and Q are double-float; the anisotropy of alpha then sits in R, and M =
// Q^T diag(c) Q - R^-T Bt R^-1 (= R^-T H R^-1), its Sylvester test and the 3x3
// solve are FP32 (to FP32 accuracy in y' relative to y - r, measured against the
// FP64 prox).  M has the inertia of H; when its test fails, H is formed in
// double-float, the FP64 eigen-clip finds its negative part, and M takes the
// same correction in this basis: M - lam w w^T with w = R^-T v (one negative
// eigenvalue), lam w w^T (two), 0 (three).  Returns y' in yo; with KEEP the
// prox's linear map y' = r + Bm (u - r), Bm = Q (I + M S)^-1 M Q^T Sigma^-1.
template <bool KEEP, int W>
__device__ void ray_dual(const float (&al)[W][3], const float (&sinv)[W], const float (&cw)[W], const dfl (&r)[W],
                         const float Bt[6], const float (&y)[W], float (&yo)[W], float (&Bm)[W][W]) {
    const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    const int sidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};   // packed index of (i, j)
    auto degenerate = [&]() {   // alpha without full rank: no curvature term, y' = r
#pragma unroll
        for (int w = 0; w < W; ++w) yo[w] = df_f(r[w]);
        if (KEEP)
            for (int w = 0; w < W; ++w)
                for (int j = 0; j < W; ++j) Bm[w][j] = 0.0f;
    };
    // A = alpha^T alpha (the products of two floats are exact)
    dfl A[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        dfl acc = df_2prod(al[0][ij[e][0]], al[0][ij[e][1]]);
#pragma unroll
        for (int w = 1; w < W; ++w) acc = df_add(acc, df_2prod(al[w][ij[e][0]], al[w][ij[e][1]]));
        A[e] = acc;
    }
    // Cholesky A = R^T R; a pivot that is not positive: alpha is degenerate
    if (!(A[0].hi > 0.0f) || !isfinite(A[0].hi)) {
        degenerate();
        return;
    }
    const dfl r00 = df_sqrt(A[0]), i00 = df_rcp(r00);
    const dfl r01 = df_mul(A[1], i00), r02 = df_mul(A[2], i00);
    const dfl t11 = df_sub(A[3], df_mul(r01, r01));
    if (!(t11.hi > 0.0f) || !isfinite(t11.hi)) {
        degenerate();
        return;
    }
    const dfl r11 = df_sqrt(t11), i11 = df_rcp(r11);
    const dfl r12 = df_mul(df_sub(A[4], df_mul(r01, r02)), i11);
    const dfl t22 = df_sub(df_sub(A[5], df_mul(r02, r02)), df_mul(r12, r12));
    if (!(t22.hi > 0.0f) || !isfinite(t22.hi)) {
        degenerate();
        return;
    }
    const dfl i22 = df_rcp(df_sqrt(t22));
    // R^-1 = [[i00, u01, u02], [0, i11, u12], [0, 0, i22]]
    const dfl u01 = df_neg(df_mul(df_mul(r01, i00), i11));
    const dfl u12 = df_neg(df_mul(df_mul(r12, i11), i22));
    const dfl u02 = df_mul(df_sub(df_mul(r01, r12), df_mul(r02, r11)), df_mul(df_mul(i00, i11), i22));
    const float Ri[3][3] = {{df_f(i00), df_f(u01), df_f(u02)}, {0.0f, df_f(i11), df_f(u12)}, {0.0f, 0.0f, df_f(i22)}};
    // Q = alpha R^-1, rounded to FP32
    float q[W][3];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        q[w][0] = df_f(df_mulf(i00, al[w][0]));
        q[w][1] = df_f(df_add(df_mulf(u01, al[w][0]), df_mulf(i11, al[w][1])));
        q[w][2] = df_f(df_add(df_add(df_mulf(u02, al[w][0]), df_mulf(u12, al[w][1])), df_mulf(i22, al[w][2])));
    }
    // M = Q^T diag(c) Q - R^-T Bt R^-1 (FP32, packed)
    float M[6];
    {
        const float Bf[3][3] = {{Bt[0], Bt[1], Bt[2]}, {Bt[1], Bt[3], Bt[4]}, {Bt[2], Bt[4], Bt[5]}};
        float T[3][3];   // Bt R^-1
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float t = 0.0f;
#pragma unroll
                for (int k = 0; k <= j; ++k) t = fmaf(Bf[i][k], Ri[k][j], t);
                T[i][j] = t;
            }
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const int a = ij[e][0], b = ij[e][1];
            float qcq = 0.0f, rbr = 0.0f;
#pragma unroll
            for (int w = 0; w < W; ++w) qcq = fmaf(__fmul_rn(cw[w], q[w][a]), q[w][b], qcq);
#pragma unroll
            for (int k = 0; k <= a; ++k) rbr = fmaf(Ri[k][a], T[k][b], rbr);
            M[e] = __fsub_rn(qcq, rbr);
        }
    }
    {
        // Sylvester's criterion on M; otherwise the negative part of H in FP64
        const float m2 = fmaf(M[0], M[3], -__fmul_rn(M[1], M[1]));
        const float det = fmaf(M[0], fmaf(M[3], M[5], -__fmul_rn(M[4], M[4])),
                               fmaf(-M[1], fmaf(M[1], M[5], -__fmul_rn(M[4], M[2])),
                                    __fmul_rn(M[2], fmaf(M[1], M[4], -__fmul_rn(M[3], M[2])))));
        if (!(M[0] > 0.0f && m2 > 0.0f && det > 0.0f)) {
            // H = sum_w c_w alpha_w alpha_w^T - Bt from exact products, in double-float
            double Hd[6];
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                dfl acc = {-Bt[e], 0.0f};
#pragma unroll
                for (int w = 0; w < W; ++w)
                    acc = df_add(acc, df_mulf(df_2prod(al[w][ij[e][0]], al[w][ij[e][1]]), cw[w]));
                Hd[e] = (double)acc.hi + (double)acc.lo;
            }
            double lam = 0.0, v[3] = {0.0, 0.0, 0.0};
            const int kind = clip_terms(Hd, lam, v);
            if (kind == 1 || kind == 2) {   // w = R^-T v; M - lam w w^T, or lam w w^T
                float wv[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float t = 0.0f;
#pragma unroll
                    for (int k = 0; k <= a; ++k) t = fmaf(Ri[k][a], (float)v[k], t);
                    wv[a] = t;
                }
                const float lf = (float)lam;
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    const float t = __fmul_rn(__fmul_rn(lf, wv[ij[e][0]]), wv[ij[e][1]]);
                    M[e] = kind == 1 ? __fsub_rn(M[e], t) : t;
                }
            } else if (kind == 3) {
#pragma unroll
                for (int e = 0; e < 6; ++e) M[e] = 0.0f;
            } else if (kind == 4) {   // H+ itself (diagonal H or the Jacobi fallback): M = R^-T H+ R^-1 in FP64
                const double Rd[3][3] = {{(double)i00.hi + i00.lo, (double)u01.hi + u01.lo, (double)u02.hi + u02.lo},
                                         {0.0, (double)i11.hi + i11.lo, (double)u12.hi + u12.lo},
                                         {0.0, 0.0, (double)i22.hi + i22.lo}};
                double Td[3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        double t = 0.0;
#pragma unroll
                        for (int k = 0; k <= j; ++k) t = fma(Hd[sidx[i][k]], Rd[k][j], t);
                        Td[i][j] = t;
                    }
#pragma unroll
                for (int e = 0; e < 6; ++e) {
                    double t = 0.0;
#pragma unroll
                    for (int k = 0; k <= ij[e][0]; ++k) t = fma(Rd[k][ij[e][0]], Td[k][ij[e][1]], t);
                    M[e] = (float)t;
                }
            }
        }
    }
    // S = Q^T Sigma^-1 Q, phi = Q^T Sigma^-1 (y - r)
    float S[6], phi[3] = {0.0f, 0.0f, 0.0f}, sd[W];
#pragma unroll
    for (int w = 0; w < W; ++w) sd[w] = __fmul_rn(sinv[w], df_f(df_sub(dfl{y[w], 0.0f}, r[w])));
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < W; ++w) t = fmaf(__fmul_rn(sinv[w], q[w][ij[e][0]]), q[w][ij[e][1]], t);
        S[e] = t;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int w = 0; w < W; ++w) phi[a] = fmaf(q[w][a], sd[w], phi[a]);
    // Mx = I + M S, rhs = M phi; z = Mx^-1 rhs by the adjugate (C[i][j] the cofactor of Mx[j][i])
    float Mx[3][3], rhs[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Mx[i][j] = fmaf(M[sidx[i][2]], S[sidx[2][j]],
                            fmaf(M[sidx[i][1]], S[sidx[1][j]], fmaf(M[sidx[i][0]], S[sidx[0][j]], i == j ? 1.0f : 0.0f)));
        rhs[i] = fmaf(M[sidx[i][2]], phi[2], fmaf(M[sidx[i][1]], phi[1], __fmul_rn(M[sidx[i][0]], phi[0])));
    }
    float C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
            C[i][j] = fmaf(Mx[r0][c0], Mx[r1][c1], -__fmul_rn(Mx[r0][c1], Mx[r1][c0]));
        }
    const float idet =
        __frcp_rn(fmaf(Mx[0][2], C[2][0], fmaf(Mx[0][1], C[1][0], __fmul_rn(Mx[0][0], C[0][0]))));
    float z[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        z[i] = __fmul_rn(idet, fmaf(C[i][2], rhs[2], fmaf(C[i][1], rhs[1], __fmul_rn(C[i][0], rhs[0]))));
    // y' = r + Q z
#pragma unroll
    for (int w = 0; w < W; ++w)
        yo[w] = df_f(df_add(r[w], dfl{fmaf(q[w][2], z[2], fmaf(q[w][1], z[1], __fmul_rn(q[w][0], z[0]))), 0.0f}));
    if (KEEP) {
        // column j of the prox map: Q Mx^-1 M q_j sinv_j
        for (int j = 0; j < W; ++j) {
            float mq[3], u[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                mq[i] = fmaf(M[sidx[i][2]], q[j][2], fmaf(M[sidx[i][1]], q[j][1], __fmul_rn(M[sidx[i][0]], q[j][0])));
#pragma unroll
            for (int i = 0; i < 3; ++i)
                u[i] = __fmul_rn(idet, fmaf(C[i][2], mq[2], fmaf(C[i][1], mq[1], __fmul_rn(C[i][0], mq[0]))));
#pragma unroll
            for (int w = 0; w < W; ++w)
                Bm[w][j] = __fmul_rn(sinv[j], fmaf(q[w][2], u[2], fmaf(q[w][1], u[1], __fmul_rn(q[w][0], u[0]))));
        }
    }
}

// ------------------------------------------------------------------ fused MOCCA kernels

// a1: line integrals of the three maps at the expansion point xbar.
__device__ __forceinline__ void proj_ray(const GeomC& C, const ExcTable& E, const RayRec* rec, const SolveD& D,
                                         int l) {
    const float4 r0 = rec[l].r0, r1 = rec[l].r1;
    LineSum acc;
    ray_pixels(C, E, r0, r1.x, r1.y, l, [&](int k, float w) { acc.add(w, __ldg(D.xbar + k)); });
    const float4 gs = acc.sum();
    D.g[l] = make_float4(gs.x, gs.y, gs.z, 0.f);
}

// Blocks run views fastest and bin groups centre-out: the long central rays are
// scheduled first and the short edge rays fill the tail of the grid.
__device__ __forceinline__ int centre_out(int i, int n) {
    const int c = (n - 1) / 2;
    return (i & 1) ? c + (i + 1) / 2 : c - i / 2;
}

__global__ void __launch_bounds__(kFwdThreads, 8) k_mocca_proj(GeomC C, ExcTable E, const RayRec* rec, SolveD D,
                                                                int v0, int v1) {
    const int l = ray_in_views(C, centre_out(blockIdx.y, gridDim.y), blockIdx.x, kFwdThreads / 32, v0, v1);
    if (l >= 0) proj_ray(C, E, rec, D, l);
}

// a2-a5 and the per-ray half of a8: spectral model, curvature, dual step.
// Returns the ray's D_TPL terms; sm holds the block's mu table (load_mu_smem).
template <bool KEEP, int W>
__device__ __forceinline__ double ray_step(const GeomC& C, RayRec* rec, const SpecD& S, const StepParams& P,
                                           const SolveD& D, const float* sm, int l) {
    static_assert(!KEEP || W == 4, "nested MOCCA keeps models of four windows");
    constexpr int F4 = win_f4<W>();
    double dsum = 0.0;
    {
        const float4 r1 = rec[l].r1;
        const float4 gg = D.g[l];
        const float g0 = gg.x, g1 = gg.y, g2 = gg.z;
        // a2/a3, one pass over energies: D_w, the alpha_w numerators and per window
        // U_w = sum_i softexp''(-p_i) s_wi mu_i mu_i^T, so that the curvature term
        // sum_i beta_i mu_i mu_i^T with beta_i = softexp''_i sum_w (r_w / D_w) s_wi
        // is sum_w (r_w / D_w) U_w once r and D are known.  D_w (positive terms) is
        // summed in two levels: plain FP32 over kDFold energies, the partials
        // compensated (Neumaier)
        const int b = l % C.n_bins, nb = C.n_bins, nE = S.n_energies;
        float Ds[W], Dc[W], An[W][3], U[W][6];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            Ds[w] = Dc[w] = 0.f;
            An[w][0] = An[w][1] = An[w][2] = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) U[w][k] = 0.f;
        }
        for (int i0 = 0; i0 < nE; i0 += kDFold) {
            float Pd[W];
#pragma unroll
            for (int w = 0; w < W; ++w) Pd[w] = 0.f;
            const int i1 = min(nE, i0 + kDFold);
#pragma unroll 2   // two energies in flight: the s-table loads overlap
            for (int i = i0; i < i1; ++i) {
                const float4 qa = *reinterpret_cast<const float4*>(sm + kSmemStride * i);
                const float4 qb = *reinterpret_cast<const float4*>(sm + kSmemStride * i + 4);
                const float4 qc = *reinterpret_cast<const float4*>(sm + kSmemStride * i + 8);
                const float p = fmaf(qa.z, g2, fmaf(qa.y, g1, qa.x * g0));
                float e0, e1, e2;
                sexp3(-p, S.exp_model != 0, e0, e1, e2);
                float sv[W];
                win_load<W, true>(S.s4 + F4 * ((size_t)i * nb + b), sv);
                const float mm[6] = {qa.w, qb.x, qb.y, qb.z, qb.w, qc.x};
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    Pd[w] = fmaf(sv[w], e0, Pd[w]);
                    const float a = sv[w] * e1, c2 = sv[w] * e2;
                    An[w][0] = fmaf(a, qa.x, An[w][0]);
                    An[w][1] = fmaf(a, qa.y, An[w][1]);
                    An[w][2] = fmaf(a, qa.z, An[w][2]);
#pragma unroll
                    for (int k = 0; k < 6; ++k) U[w][k] = fmaf(c2, mm[k], U[w][k]);
                }
            }
#pragma unroll
            for (int w = 0; w < W; ++w) neumaier(Ds[w], Dc[w], Pd[w]);
        }
        float Nv[W], cv[W], y[W];
        win_load<W, true>(S.N4 + F4 * b, Nv);
        win_load<W>(D.c + F4 * (size_t)l, cv);
        win_load<W>(D.y + F4 * (size_t)l, y);
        float al[W][3], qw[W], nw[W];
        dfl rw[W];   // r = c - N D exactly to double-float precision (N D is an exact product)
        float dt = 0.f;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float Dw = Ds[w] + Dc[w];
            const float invD = 1.0f / Dw;
#pragma unroll
            for (int m = 0; m < 3; ++m) al[w][m] = An[w][m] * invD;
            nw[w] = sqrtf(al[w][0] * al[w][0] + al[w][1] * al[w][1] + al[w][2] * al[w][2]);
            const dfl chat = df_2prod(Nv[w], Dw);
            rw[w] = df_sub(dfl{cv[w], 0.0f}, chat);
            qw[w] = df_f(rw[w]) * invD;
            dt += dtpl_term(chat.hi, cv[w]);
        }
        dsum = (double)dt;
        const float X1 = __ldg(D.chord + l);
        float yo[W];
        float Bm[W][W], sinv[W];   // the prox map and Sigma^-1, kept for nested MOCCA
        // a5: dual step matrix.  m-block SPC: (Sigma^-1)_w = lambda sum_k sqrt(sum_m K^2)
        // = lambda |alpha_w| (X 1)_l;  diagonal SPC: lambda sum_mk |K| = lambda (sum_m |alpha_wm|) (X 1)_l
        auto sigma_inv = [&]() {
#pragma unroll
            for (int w = 0; w < W; ++w)
                sinv[w] = P.lambda * X1 *
                          (P.spc == 0 ? nw[w] : fabsf(al[w][0]) + fabsf(al[w][1]) + fabsf(al[w][2]));
        };
        if (!(X1 > 0.f)) {   // the ray misses the image: Sigma^-1 = 0, the dual is kept
#pragma unroll
            for (int w = 0; w < W; ++w) yo[w] = y[w];
        } else if (P.model == 1) {   // W = 0: y' = y - Sigma Sigma^-1 (y - r) = r
#pragma unroll
            for (int w = 0; w < W; ++w) yo[w] = df_f(rw[w]);
            if (KEEP) {
                sigma_inv();
                for (int w = 0; w < W; ++w)
                    for (int j = 0; j < W; ++j) Bm[w][j] = 0.0f;
            }
        } else if (P.model == 3) {   // W = diag(c): y'_w = r_w + c_w sinv_w / (c_w sinv_w + 1) (y_w - r_w)
            sigma_inv();
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const float cs = cv[w] * sinv[w], f = cs / (cs + 1.0f);
                yo[w] = df_f(df_add(rw[w], df_mulf(df_sub(dfl{y[w], 0.0f}, rw[w]), f)));
                if (KEEP)
                    for (int j = 0; j < W; ++j) Bm[w][j] = j == w ? f : 0.0f;
            }
        } else {
            // model 0: sum_i beta_i mu_i mu_i^T = sum_w (r_w / D_w) U_w is subtracted from
            // sum_w c_w alpha_w alpha_w^T; model 2 (Gauss-Newton) keeps the first term alone
            float Bt[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                float t = qw[0] * U[0][k];
#pragma unroll
                for (int w = 1; w < W; ++w) t = fmaf(qw[w], U[w][k], t);
                Bt[k] = P.model == 2 ? 0.0f : t;
            }
            sigma_inv();
            ray_dual<KEEP, W>(al, sinv, cv, rw, Bt, y, yo, Bm);
        }
        if constexpr (KEEP) {
            float4* M = D.model + (size_t)kModelStride * l;
#pragma unroll
            for (int m = 0; m < 3; ++m) M[m] = make_float4(al[0][m], al[1][m], al[2][m], al[3][m]);
            M[3] = make_float4(g0, g1, g2, X1 > 0.f ? 1.0f : 0.0f);
            M[4] = make_float4(rw[0].hi, rw[1].hi, rw[2].hi, rw[3].hi);
            M[5] = make_float4(rw[0].lo, rw[1].lo, rw[2].lo, rw[3].lo);
            if (X1 > 0.f) {   // a ray outside the image (flag 0) keeps its dual: nothing more is read
                M[6] = make_float4(sinv[0], sinv[1], sinv[2], sinv[3]);
#pragma unroll
                for (int w = 0; w < 4; ++w) M[7 + w] = make_float4(Bm[w][0], Bm[w][1], Bm[w][2], Bm[w][3]);
            }
        }
        win_store<W>(D.y + F4 * (size_t)l, yo);
        const float (&yf)[W] = yo;
        // b = alpha^T y';  the ray's share of T^-1: m-block SPC S = sum_w alpha_w alpha_w^T / |alpha_w|,
        // diagonal SPC S = diag(sum_w |alpha_wm|)
        float bb[3] = {0.f, 0.f, 0.f}, Sm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int w = 0; w < W; ++w) {
#pragma unroll
            for (int m = 0; m < 3; ++m) bb[m] = fmaf(al[w][m], yf[w], bb[m]);
            if (P.spc == 0) {
                const float inw = nw[w] > 0.f ? 1.0f / nw[w] : 0.f;
                const float a0 = al[w][0] * inw, a1 = al[w][1] * inw, a2 = al[w][2] * inw;
                Sm[0] = fmaf(a0, al[w][0], Sm[0]); Sm[1] = fmaf(a0, al[w][1], Sm[1]);
                Sm[2] = fmaf(a0, al[w][2], Sm[2]); Sm[3] = fmaf(a1, al[w][1], Sm[3]);
                Sm[4] = fmaf(a1, al[w][2], Sm[4]); Sm[5] = fmaf(a2, al[w][2], Sm[5]);
            } else {
                Sm[0] += fabsf(al[w][0]);
                Sm[3] += fabsf(al[w][1]);
                Sm[5] += fabsf(al[w][2]);
            }
        }
        rec[l].r1 = make_float4(r1.x, r1.y, bb[0], bb[1]);
        RayStep* st = ray_steps(rec, C.n_views * C.n_bins) + l;
        st->s0 = make_float4(bb[2], Sm[0], Sm[1], Sm[2]);
        st->s1 = make_float4(Sm[3], Sm[4], Sm[5], 0.f);
    }
    return dsum;
}

// Resident blocks of 128 threads: five for four windows (96 registers, a few
// spills; 0.137 ms at 256x256 against 0.144 ms with four and 0.160 ms with six),
// four for five windows (128 registers; 0.136 ms against 0.152 ms with three).
template <bool KEEP, int W>
__global__ void __launch_bounds__(kFwdThreads, W == 4 ? 5 : 4) k_mocca_ray(GeomC C, RayRec* rec, SpecD S,
                                                                         StepParams P, SolveD D, int v0, int v1) {
    __shared__ float sm[kSmemStride * kMaxEnergies];
    load_mu_smem(S, sm);
    __syncthreads();
    const int l = ray_in_views(C, blockIdx.x, blockIdx.y, kFwdThreads / 32, v0, v1);
    const double dsum = l >= 0 ? ray_step<KEEP, W>(C, rec, S, P, D, sm, l) : 0.0;
    warp_partial(C, blockIdx.x, v0 + warp_view(blockIdx.y, kFwdThreads / 32), dsum, D.dtpl_part, v1);
}

// Inner iteration of nested MOCCA: the dual prox of the kept convex model at
// u = y + Sigma alpha (g - g0) (g = X xbar from k_mocca_proj), y' = r + B (u - r)
// in double-float, then b = alpha^T y'; the step matrix S stays the outer one.
__global__ void __launch_bounds__(kFwdThreads) k_mocca_ray_inner(GeomC C, RayRec* rec, SolveD D) {
    const int l = ray_of_thread(C);
    if (l < 0) return;
    const float4* M = D.model + (size_t)kModelStride * l;
    const float4 a0 = M[0], a1 = M[1], a2 = M[2], g0 = M[3];
    const float al[4][3] = {{a0.x, a1.x, a2.x}, {a0.y, a1.y, a2.y}, {a0.z, a1.z, a2.z}, {a0.w, a1.w, a2.w}};
    const float4 yy = D.y[l];
    const float y[4] = {yy.x, yy.y, yy.z, yy.w};
    float yo[4] = {y[0], y[1], y[2], y[3]};
    if (g0.w != 0.0f) {
        const float4 gg = D.g[l], rh = M[4], rl = M[5], si = M[6];
        const float dg[3] = {gg.x - g0.x, gg.y - g0.y, gg.z - g0.z};
        const float sv[4] = {si.x, si.y, si.z, si.w};
        const dfl r[4] = {{rh.x, rl.x}, {rh.y, rl.y}, {rh.z, rl.z}, {rh.w, rl.w}};
        dfl d[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float kz = fmaf(al[w][2], dg[2], fmaf(al[w][1], dg[1], al[w][0] * dg[0]));
            const float step = sv[w] > 0.0f ? kz / sv[w] : 0.0f;
            d[w] = df_sub(df_add(dfl{y[w], 0.0f}, dfl{step, 0.0f}), r[w]);   // u - r
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float4 B = M[7 + w];
            const dfl t = df_add(df_add(df_mulf(d[0], B.x), df_mulf(d[1], B.y)),
                                 df_add(df_mulf(d[2], B.z), df_mulf(d[3], B.w)));
            yo[w] = df_f(df_add(r[w], t));
        }
    }
    D.y[l] = make_float4(yo[0], yo[1], yo[2], yo[3]);
    float bb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int m = 0; m < 3; ++m) bb[m] = fmaf(al[w][m], yo[w], bb[m]);
    const float4 r1 = rec[l].r1;
    rec[l].r1 = make_float4(r1.x, r1.y, bb[0], bb[1]);
    ray_steps(rec, C.n_views * C.n_bins)[l].s0.x = bb[2];
}

// Box-constrained primal step: argmin over lo <= x <= hi of 1/2 (x - t)^T Q (x - t),
// by trying every active set and keeping the feasible candidate of least objective.
// Bounds may be infinite (nonnegativity: lo = 0, hi = +inf).
__device__ void box_prox3(const double Q[3][3], const double t[3], const float lo[3], const float hi[3],
                          double xo[3]) {
    double best = 1e308;
    xo[0] = fmin(fmax(t[0], (double)lo[0]), (double)hi[0]);
    xo[1] = fmin(fmax(t[1], (double)lo[1]), (double)hi[1]);
    xo[2] = fmin(fmax(t[2], (double)lo[2]), (double)hi[2]);
    for (int code = 0; code < 27; ++code) {
        const int st[3] = {code % 3, (code / 3) % 3, code / 9};
        double xc[3];
        int fr[3], nf = 0;
        bool unbounded = false;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            if (st[m] == 1) xc[m] = lo[m];
            else if (st[m] == 2) xc[m] = hi[m];
            else fr[nf++] = m;
            if (st[m] != 0 && isinf(xc[m])) unbounded = true;   // no point sits at an infinite bound
        }
        if (unbounded) continue;
        bool ok = true;
        if (nf > 0) {
            double Mf[3][3], rhs[3];
            for (int a = 0; a < nf; ++a) {
                double acc = 0.0;
                for (int m = 0; m < 3; ++m)
                    if (st[m] != 0) acc -= Q[fr[a]][m] * (xc[m] - t[m]);
                rhs[a] = acc;
                for (int c2 = 0; c2 < nf; ++c2) Mf[a][c2] = Q[fr[a]][fr[c2]];
            }
            // Gaussian elimination (nf <= 3, SPD sub-block)
            for (int c2 = 0; c2 < nf && ok; ++c2) {
                if (!(Mf[c2][c2] > 0.0)) { ok = false; break; }
                for (int r2 = c2 + 1; r2 < nf; ++r2) {
                    const double f = Mf[r2][c2] / Mf[c2][c2];
                    for (int k = c2; k < nf; ++k) Mf[r2][k] -= f * Mf[c2][k];
                    rhs[r2] -= f * rhs[c2];
                }
            }
            if (!ok) continue;
            double sol[3];
            for (int r2 = nf - 1; r2 >= 0; --r2) {
                double acc = rhs[r2];
                for (int k = r2 + 1; k < nf; ++k) acc -= Mf[r2][k] * sol[k];
                sol[r2] = acc / Mf[r2][r2];
            }
            for (int a = 0; a < nf; ++a) {
                const int m = fr[a];
                const double val = t[m] + sol[a];
                const double span = (double)hi[m] - (double)lo[m];
                const double tol = 1e-12 * (1.0 + (isfinite(span) ? fabs(span) : fabs(val)));
                if (val < lo[m] - tol || val > hi[m] + tol) ok = false;
                xc[m] = fmin(fmax(val, (double)lo[m]), (double)hi[m]);
            }
            if (!ok) continue;
        }
        double obj = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) obj += 0.5 * (xc[i] - t[i]) * Q[i][j] * (xc[j] - t[j]);
        if (obj < best) {
            best = obj;
            xo[0] = xc[0]; xo[1] = xc[1]; xo[2] = xc[2];
        }
    }
}

__device__ __forceinline__ void bp_finish(const GeomC& C, const StepParams& P, const SolveD& D, int ix, int iy,
                                          bool valid, int pix, int npix, int g, int G, float* red, float acc[9]);
__device__ __forceinline__ void pixel_step(const GeomC& C, const StepParams& P, const SolveD& D, int k,
                                           const float acc[9]);

// The nine channels of one footprint pair (weight w != 0): K^T y' (from b in
// r1.zw and s0.x) and the step matrix (s0.yzw, s1.xyz).
__device__ __forceinline__ void bp_accumulate(float acc[9], float w, const float4& r1, const float4& s0,
                                              const float4& s1) {
    acc[0] = fmaf(w, r1.z, acc[0]);
    acc[1] = fmaf(w, r1.w, acc[1]);
    acc[2] = fmaf(w, s0.x, acc[2]);
    acc[3] = fmaf(w, s0.y, acc[3]);
    acc[4] = fmaf(w, s0.z, acc[4]);
    acc[5] = fmaf(w, s0.w, acc[5]);
    acc[6] = fmaf(w, s1.x, acc[6]);
    acc[7] = fmaf(w, s1.y, acc[7]);
    acc[8] = fmaf(w, s1.z, acc[8]);
}

// Pixel-driven back-projection of pixel (ix, iy) over the views [v0, v1):
// for each view in order, the candidate bins of the pixel's corner shadow in
// ascending order, each weight from x_weight, the nine channels added for the
// nonzero ones.  Every form of the back-projection adds in this order.
__device__ __forceinline__ void bp_pixel_sum(const GeomC& C, const ExcTable& E, const RayRec* rec,
                                             const ViewF* views, int ix, int iy, int v0, int v1, float acc[9]) {
    const RayStep* steps = ray_steps(rec, C.n_views * C.n_bins);
    for (int v = v0; v < v1; ++v) {
        int blo, bhi;
        pixel_bin_range(C, views[v], ix, iy, blo, bhi);
        // two candidate rays per step: both records' first halves are loaded before either is used
        for (int b = blo; b <= bhi; b += 2) {
            const int l = v * C.n_bins + b;
            const bool two = b < bhi;
            const RecHalf A = ldg_half(&rec[l].r0);
            RecHalf B = A;
            if (two) B = ldg_half(&rec[l + 1].r0);
            const float wa = x_weight(A.a, A.b.x, A.b.y, C.grid, E, l, ix, iy);
            const float wb = two ? x_weight(B.a, B.b.x, B.b.y, C.grid, E, l + 1, ix, iy) : 0.0f;
            if (wa != 0.0f) {
                const RecHalf A2 = ldg_half(&steps[l].s0);
                bp_accumulate(acc, wa, A.b, A2.a, A2.b);
            }
            if (wb != 0.0f) {
                const RecHalf B2 = ldg_half(&steps[l + 1].s0);
                bp_accumulate(acc, wb, B.b, B2.a, B2.b);
            }
        }
    }
}

// The views of group g of G when [V0, V1) is split into contiguous ranges.
__device__ __forceinline__ void group_views(int V0, int V1, int g, int G, int& v0, int& v1) {
    const int per = (V1 - V0 + G - 1) / G;
    v0 = V0 + g * per;
    v1 = min(V1, v0 + per);
}

// Pixel-driven back-projection with the views split over blockDim.z thread
// groups per pixel (contiguous view ranges); the groups' partial sums are
// added in a fixed order in shared memory, so results are deterministic.
// red holds the tile's [G - 1][9][kBpPix] partials; every thread of the block
// must call this (it contains a block barrier).
__device__ __forceinline__ void bp_pixel(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                         const StepParams& P, const SolveD& D, int ix, int iy, int pix, int g, int G,
                                         float* red) {
    const bool valid = ix < C.grid.n && iy < C.grid.n;
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        int v0, v1;
        group_views(0, C.n_views, g, G, v0, v1);
        bp_pixel_sum(C, E, rec, views, ix, iy, v0, v1, acc);
    }
    bp_finish(C, P, D, ix, iy, valid, pix, kBpPix, g, G, red, acc);
}

// Group g > 0 stores its partial sums in red ([G - 1][9][npix]); group 0 adds
// them in group order and writes the nine summed channels of pixel k to
// chan ([9][P]) for a sum over view ranges.  Contains a block barrier.
__device__ __forceinline__ void bp_partial_out(int P_, int k, bool valid, int pix, int npix, int g, int G,
                                               float* red, float acc[9], float* chan) {
    if (g > 0) {
#pragma unroll
        for (int c = 0; c < 9; ++c) red[((g - 1) * 9 + c) * npix + pix] = acc[c];
    }
    __syncthreads();
    if (g != 0 || !valid) return;
    for (int gg = 1; gg < G; ++gg)
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] += red[((gg - 1) * 9 + c) * npix + pix];
#pragma unroll
    for (int c = 0; c < 9; ++c) chan[(size_t)c * P_ + k] = acc[c];
}

// The end of a pixel's back-projection: group g of G stores its nine partial
// sums in red ([G - 1][9][npix]); group 0 adds the others' in group order, then
// solves T_k v = K^T y' in FP64 and takes the primal step.  Every thread of the
// block must call this (it contains a block barrier).
__device__ __forceinline__ void bp_finish(const GeomC& C, const StepParams& P, const SolveD& D, int ix, int iy,
                                          bool valid, int pix, int npix, int g, int G, float* red, float acc[9]) {
    if (g > 0) {
#pragma unroll
        for (int c = 0; c < 9; ++c) red[((g - 1) * 9 + c) * npix + pix] = acc[c];
    }
    __syncthreads();
    if (g != 0 || !valid) return;
    for (int gg = 1; gg < G; ++gg)
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] += red[((gg - 1) * 9 + c) * npix + pix];
    pixel_step(C, P, D, iy * C.grid.n + ix, acc);
}

// a7 for pixel k from its nine back-projected channels: acc[0..2] = v_k = (K^T y')_k,
// acc[3..8] = P_k (packed 00 01 02 11 12 22), T^-1_k = P_k / lambda; the primal
// step x' = x - T_k v_k (optionally onto the box) and the extrapolation
// xbar' = 2 x' - x.  T_k = lambda (P_k + 1e-12 tr(P_k) I)^-1 (the regularisation
// that keeps T positive definite) is applied by the adjugate in double-float
// arithmetic on P_k scaled by an exact power of two near 1 / tr(P_k), so that the
// cubed entries stay inside the FP32 exponent range; T_k has a condition number
// near 6e6, and the ~48-bit double-float solve keeps the step to FP32 accuracy.
// Only a step that leaves the box goes to the FP64 active-set solve.
__device__ __forceinline__ void pixel_step(const GeomC& C, const StepParams& P, const SolveD& D, int k,
                                           const float acc[9]) {
    const float4 x = D.x[k];
    const int n = C.grid.n, kt = n * n + (k % n) * n + k / n;   // the column-major copy of xbar
    const double trd = (double)acc[3] + (double)acc[6] + (double)acc[8];
    if (!(trd > 0.0)) {
        D.xbar[k] = x;
        D.xbar[kt] = x;
        return;
    }
    int e;
    frexpf((float)trd, &e);
    const float sc = ldexpf(1.0f, -e);   // tr(P) sc in [0.5, 1)
    const float p1 = acc[4] * sc, p2 = acc[5] * sc, p4 = acc[7] * sc;
    const float reg = 1e-12f * ((acc[3] * sc + acc[6] * sc) + acc[8] * sc);
    const dfl p0 = df_2sum(acc[3] * sc, reg), p3 = df_2sum(acc[6] * sc, reg), p5 = df_2sum(acc[8] * sc, reg);
    const dfl P1 = {p1, 0.0f}, P2 = {p2, 0.0f};
    const dfl c00 = df_sub(df_mul(p3, p5), df_2prod(p4, p4));
    const dfl c01 = df_sub(df_2prod(p2, p4), df_mulf(p5, p1));
    const dfl c02 = df_sub(df_2prod(p1, p4), df_mulf(p3, p2));
    const dfl c11 = df_sub(df_mul(p0, p5), df_2prod(p2, p2));
    const dfl c12 = df_sub(df_2prod(p1, p2), df_mulf(p0, p4));
    const dfl c22 = df_sub(df_mul(p0, p3), df_2prod(p1, p1));
    const dfl det = df_add(df_add(df_mul(p0, c00), df_mul(P1, c01)), df_mul(P2, c02));
    dfl t[3] = {{x.x, 0.0f}, {x.y, 0.0f}, {x.z, 0.0f}};
    if (det.hi != 0.0f && isfinite(det.hi)) {
        const dfl f = df_mulf(df_rcp(det), P.lambda * sc);   // lambda sc / det
        const dfl u0 = df_add(df_add(df_mulf(c00, acc[0]), df_mulf(c01, acc[1])), df_mulf(c02, acc[2]));
        const dfl u1 = df_add(df_add(df_mulf(c01, acc[0]), df_mulf(c11, acc[1])), df_mulf(c12, acc[2]));
        const dfl u2 = df_add(df_add(df_mulf(c02, acc[0]), df_mulf(c12, acc[1])), df_mulf(c22, acc[2]));
        t[0] = df_sub(t[0], df_mul(u0, f));
        t[1] = df_sub(t[1], df_mul(u1, f));
        t[2] = df_sub(t[2], df_mul(u2, f));
    }
    float xo3[3] = {df_f(t[0]), df_f(t[1]), df_f(t[2])};
    if (P.use_box && (xo3[0] < P.lo[0] || xo3[0] > P.hi[0] || xo3[1] < P.lo[1] || xo3[1] > P.hi[1] ||
                      xo3[2] < P.lo[2] || xo3[2] > P.hi[2])) {
        const double il = 1.0 / (double)P.lambda;
        double T[6] = {acc[3] * il, acc[4] * il, acc[5] * il, acc[6] * il, acc[7] * il, acc[8] * il};
        const double tr = T[0] + T[3] + T[5];
        T[0] += 1e-12 * tr;
        T[3] += 1e-12 * tr;
        T[5] += 1e-12 * tr;
        const double Q[3][3] = {{T[0], T[1], T[2]}, {T[1], T[3], T[4]}, {T[2], T[4], T[5]}};
        const double td[3] = {(double)t[0].hi + (double)t[0].lo, (double)t[1].hi + (double)t[1].lo,
                              (double)t[2].hi + (double)t[2].lo};
        double xo[3];
        box_prox3(Q, td, P.lo, P.hi, xo);
        xo3[0] = (float)xo[0];
        xo3[1] = (float)xo[1];
        xo3[2] = (float)xo[2];
    }
    const float4 xn = make_float4(xo3[0], xo3[1], xo3[2], 0.f);
    D.x[k] = xn;
    const float4 xb = make_float4(2.f * xn.x - x.x, 2.f * xn.y - x.y, 2.f * xn.z - x.z, 0.f);
    D.xbar[k] = xb;
    D.xbar[kt] = xb;
}

// The back-projection and primal step of every pixel over the views [V0, V1);
// PARTIAL: the summed channels go to chan ([9][P]) instead of the primal step.
template <bool PARTIAL>
__global__ void __launch_bounds__(kBpMaxThreads) k_mocca_bp(GeomC C, ExcTable E, const RayRec* rec,
                                                           const ViewF* views, StepParams P, SolveD D, int V0,
                                                           int V1, float* chan) {
    extern __shared__ float red[];   // [blockDim.z - 1][9][kBpPix]
    const int ix = blockIdx.x * kBpPixX + threadIdx.x, iy = blockIdx.y * kBpPixY + threadIdx.y;
    const int pix = threadIdx.y * kBpPixX + threadIdx.x, g = threadIdx.z, G = blockDim.z;
    const bool valid = ix < C.grid.n && iy < C.grid.n;
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        int v0, v1;
        group_views(V0, V1, g, G, v0, v1);
        bp_pixel_sum(C, E, rec, views, ix, iy, v0, v1, acc);
    }
    if (PARTIAL)
        bp_partial_out(C.grid.n * C.grid.n, iy * C.grid.n + ix, valid, pix, kBpPix, g, G, red, acc, chan);
    else
        bp_finish(C, P, D, ix, iy, valid, pix, kBpPix, g, G, red, acc);
}

// a7 alone, from channels summed over view ranges (chan [9][P]).
__global__ void k_mocca_apply(GeomC C, StepParams P, SolveD D, const float* __restrict__ chan) {
    const int P_ = C.grid.n * C.grid.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P_) return;
    float acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = chan[(size_t)c * P_ + k];
    pixel_step(C, P, D, k, acc);
}

// ------------------------------------------------------------------ footprint tables
//
// X depends only on the geometry, so its pairs are written once per context in
// the order in which each projector visits them, and the per-iteration
// projections stream them instead of tracing rays and testing pixels again:
// about 8 bytes per pair read (forward) and about 10 bytes per pixel and view
// (back-projection) against roughly a hundred instructions of recomputation per
// pair.  The weights are x_weight's own values and the order of additions is
// the on-the-fly kernels' (k_mocca_proj, k_mocca_bp), so the results are bit
// for bit the same.  See FpTables for the layout.

// Forward table, pass 1: the footprint size of every ray, and per warp (view,
// 32-bin group) the largest one: its number of slot rows.
__global__ void __launch_bounds__(kFwdThreads) k_fp_fwd_count(GeomC C, ExcTable E, const RayRec* rec, int* cnt,
                                                              uint32_t* warp_rows) {
    const int l = ray_of_thread(C);
    int n = 0;
    if (l >= 0) {
        const float4 r0 = rec[l].r0, r1 = rec[l].r1;
        ray_pixels(C, E, r0, r1.x, r1.y, l, [&](int, float) { ++n; });
        cnt[l] = n;
    }
    n = __reduce_max_sync(0xffffffffu, n);
    const int v = warp_view(blockIdx.y, kFwdThreads / 32);
    if ((threadIdx.x & 31) == 0 && v < C.n_views) warp_rows[v * ((C.n_bins + 31) >> 5) + blockIdx.x] = (uint32_t)n;
}

// Forward table, pass 2: lane r of warp w writes its j-th pair (weight, pixel
// step) in visiting order, two per slot row from fwd_row[w] (see FpTables).
// Each ray's pixels index the xbar copy in which the warp's gathers at one
// table row are close.  The lanes advance from their first pixels at about the
// same pace along the slabs, so what matters is the image edge a ray enters
// by: lanes whose rays enter through a left or right edge start in one column
// and stay in neighbouring rows of a column (the column-major copy,
// P + ix n + iy); lanes whose rays enter through the bottom or top edge stay in
// neighbouring columns of a row (the row-major copy).  A lane chooses from its
// own first pixel: 7.8 distinct 128-byte lines per warp gather at 256x256,
// against 12.0 when the warp chose by the rays' direction.
__global__ void __launch_bounds__(kFwdThreads) k_fp_fwd_fill(GeomC C, ExcTable E, const RayRec* rec,
                                                             const uint32_t* __restrict__ fwd_row, float* fwd_w,
                                                             int16_t* fwd_d, int* fwd_k0, int* bad) {
    const int l = ray_of_thread(C);
    if (l < 0) return;
    const int v = warp_view(blockIdx.y, kFwdThreads / 32);
    const size_t row = fwd_row[v * ((C.n_bins + 31) >> 5) + blockIdx.x];
    const int lane = threadIdx.x & 31, n = C.grid.n;
    const float4 r0 = rec[l].r0, r1 = rec[l].r1;
    int j = 0, prev = -1;
    bool col = false;
    ray_pixels(C, E, r0, r1.x, r1.y, l, [&](int kr, float w) {
        if (j == 0) col = kr % n == 0 || kr % n == n - 1;   // entered through a left or right edge
        const int k = col ? n * n + (kr % n) * n + kr / n : kr;
        const size_t at = (row + (j & ~1)) * 32 + 2 * lane + (j & 1);
        if (j == 0) {
            fwd_k0[l] = k;
            prev = k;
        }
        const int d = k - prev;
        if (d < -32768 || d > 32767) *bad = 1;
        fwd_w[at] = w;
        fwd_d[at] = (int16_t)d;
        prev = k;
        ++j;
    });
    if (j == 0) fwd_k0[l] = 0;
}

// a1 from the forward table for ray l of warp wi = v nbg + bx: the same line sums
// as proj_ray, in the same order.  The table is read four entries (two loads of
// two) at a time, the next four loaded while the current four's gathers of xbar
// are added, so a table load is always in flight.
__device__ __forceinline__ void fp_proj_ray(const FpTables& T, const SolveD& D, int l, int wi) {
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)T.fwd_row[wi] * 32;
    const float2* pw = reinterpret_cast<const float2*>(T.fwd_w + base) + lane;
    const short2* pd = reinterpret_cast<const short2*>(T.fwd_d + base) + lane;
    const int n = __ldg(T.fwd_cnt + l);
    int k = __ldg(T.fwd_k0 + l);
    LineSum acc;
    int j = 0;
    if (n >= 4) {
        float2 w[2];
        short2 d[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            w[u] = __ldg(pw + 32 * u);
            d[u] = __ldg(pd + 32 * u);
        }
        for (; j + 3 < n; j += 4) {
            pw += 64;
            pd += 64;
            float2 wn[2];
            short2 dn[2];
            const bool more = j + 7 < n;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                wn[u] = more ? __ldg(pw + 32 * u) : make_float2(0.f, 0.f);
                dn[u] = more ? __ldg(pd + 32 * u) : make_short2(0, 0);
            }
            int kk[4];
            kk[0] = k + d[0].x;
            kk[1] = kk[0] + d[0].y;
            kk[2] = kk[1] + d[1].x;
            kk[3] = kk[2] + d[1].y;
            k = kk[3];
            float4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __ldg(D.xbar + kk[u]);
            acc.add(w[0].x, x[0]);
            acc.add(w[0].y, x[1]);
            acc.add(w[1].x, x[2]);
            acc.add(w[1].y, x[3]);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                w[u] = wn[u];
                d[u] = dn[u];
            }
        }
    }
    for (; j < n; j += 2, pw += 32, pd += 32) {
        const float2 w = __ldg(pw);
        const short2 d = __ldg(pd);
        k += d.x;
        acc.add(w.x, __ldg(D.xbar + k));
        if (j + 1 < n) {
            k += d.y;
            acc.add(w.y, __ldg(D.xbar + k));
        }
    }
    const float4 gs = acc.sum();
    D.g[l] = make_float4(gs.x, gs.y, gs.z, 0.f);
}

__global__ void __launch_bounds__(kFwdThreads, 8) k_fp_proj(GeomC C, FpTables T, SolveD D, int v0, int v1) {
    const int bx = centre_out(blockIdx.y, gridDim.y);
    const int l = ray_in_views(C, bx, blockIdx.x, kFwdThreads / 32, v0, v1);
    if (l >= 0) fp_proj_ray(T, D, l, (l / C.n_bins) * ((C.n_bins + 31) >> 5) + bx);
}

// The footprint pairs of pixel (ix, iy) in the views [v0, v1), in the order
// bp_pixel_sum adds them (views ascending, candidate bins ascending, nonzero
// weights only): visit(l, w).
template <class Visit>
__device__ __forceinline__ void pixel_pairs(const GeomC& C, const ExcTable& E, const RayRec* rec,
                                            const ViewF* views, int ix, int iy, int v0, int v1, Visit&& visit) {
    for (int v = v0; v < v1; ++v) {
        int blo, bhi;
        pixel_bin_range(C, views[v], ix, iy, blo, bhi);
        for (int b = blo; b <= bhi; ++b) {
            const int l = v * C.n_bins + b;
            const float4 r0 = rec[l].r0, r1 = rec[l].r1;
            const float w = x_weight(r0, r1.x, r1.y, C.grid, E, l, ix, iy);
            if (w != 0.0f) visit(l, w);
        }
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// ------------------------------------------------------------------ blocked back-projection table
//
// Block b = t G + g: pixel tile t (kBTX x kBTY pixels, one per thread) and view
// group g of G (the split of k_mocca_bp).  The group's views go in chunks of
// T.bp_chunk views; for chunk c the block stages, with asynchronous 16-byte
// copies, the records of the rays that can meet the tile (per view u the bins
// [tlo_u, tlo_u + span_u) of bp_span, view after view: stage slot
// off_u + b - tlo_u), and each pixel runs through its pairs (slot, weight) of
// the chunk, in the order of bp_pixel_sum.  A ray's record is read from L2 once
// per tile and view and then from shared memory by every pixel that meets it.

// The pixel of thread `tid` in tile t: warp w takes a 4 x 8 patch of the 16 x 16
// tile (four patches across, two down), lane l pixel (l mod 4, l / 4) of it.  A
// compact patch needs few neighbouring bins in any view, so the lanes' reads of
// the staged slots at one table row hit few banks (measured: 0.147 ms against
// 0.160 ms with a warp on two rows of 16, 0.156 ms with 8 x 4 patches).
__device__ __forceinline__ void bt_pixel(int n, int t, int tid, int& ix, int& iy) {
    static_assert(kBTX == 16 && kBTY == 16, "the warp patches tile 16 x 16");
    const int ntx = (n + kBTX - 1) / kBTX, w = tid >> 5, l = tid & 31;
    ix = (t % ntx) * kBTX + (w & 3) * 4 + (l & 3);
    iy = (t / ntx) * kBTY + (w >> 2) * 8 + (l >> 2);
}

// The views [u0, u1) of chunk c of group g (views [V0, V1) of the whole range
// split as group_views does, then in chunks of `chunk`).
__device__ __forceinline__ void chunk_views(int n_views, int g, int G, int chunk, int c, int& u0, int& u1) {
    int v0, v1;
    group_views(0, n_views, g, G, v0, v1);
    u0 = min(v1, v0 + c * chunk);
    u1 = min(v1, u0 + chunk);
}

// Table pass 0: per tile and view the union of its pixels' candidate bins,
// tlo | span << 16 (span 0: no pixel of the tile has a candidate there).
__global__ void __launch_bounds__(kBTThreads) k_fpb_span(GeomC C, const ViewF* views, uint32_t* span) {
    __shared__ int red_lo[kBTThreads / 32], red_hi[kBTThreads / 32];
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int ix, iy;
    bt_pixel(C.grid.n, t, tid, ix, iy);
    const bool valid = ix < C.grid.n && iy < C.grid.n;
    for (int v = 0; v < C.n_views; ++v) {
        int blo = 0x7fffffff, bhi = -1;
        if (valid) {
            int lo, hi;
            pixel_bin_range(C, views[v], ix, iy, lo, hi);
            if (lo <= hi) {
                blo = lo;
                bhi = hi;
            }
        }
        blo = __reduce_min_sync(0xffffffffu, blo);
        bhi = __reduce_max_sync(0xffffffffu, bhi);
        if (lane == 0) {
            red_lo[wid] = blo;
            red_hi[wid] = bhi;
        }
        __syncthreads();
        if (tid == 0) {
            int lo = red_lo[0], hi = red_hi[0];
            for (int w = 1; w < kBTThreads / 32; ++w) {
                lo = min(lo, red_lo[w]);
                hi = max(hi, red_hi[w]);
            }
            span[(size_t)t * C.n_views + v] = hi < lo ? 0u : (uint32_t)lo | ((uint32_t)(hi - lo + 1) << 16);
        }
        __syncthreads();
    }
}

// The stage slot offsets of chunk views [u0, u1) of tile t: off[i] for view u0 + i.
__device__ __forceinline__ int chunk_offsets(const uint32_t* span, int t, int n_views, int u0, int u1,
                                             int off[kBTMaxChunk], int tlo[kBTMaxChunk], int wid[kBTMaxChunk]) {
    int total = 0;
#pragma unroll
    for (int i = 0; i < kBTMaxChunk; ++i) {
        const int u = u0 + i;
        const uint32_t sp = u < u1 ? __ldg(span + (size_t)t * n_views + u) : 0u;
        off[i] = total;
        tlo[i] = (int)(sp & 0xffffu);
        wid[i] = (int)(sp >> 16);
        total += wid[i];
    }
    return total;
}

// The table rows of a warp are aligned per view: view u of a chunk takes K_u rows,
// the largest number of pairs any of the warp's pixels has in u, so that at every
// row the warp's lanes read stage slots of one view (neighbouring slots, few bank
// conflicts); a pixel with fewer pairs in u leaves the rest of them empty (slot
// kBTNoSlot).
constexpr uint16_t kBTNoSlot = 0xffff;

// Table pass 1: per (block, chunk) and warp the number of rows, the sum of K_u.
__global__ void __launch_bounds__(kBTThreads) k_fpb_count(GeomC C, ExcTable E, const RayRec* rec,
                                                          const ViewF* views, int G, int chunk, int nch,
                                                          uint32_t* warp_rows) {
    const int b = blockIdx.x, t = b / G, g = b % G, tid = threadIdx.x;
    int ix, iy;
    bt_pixel(C.grid.n, t, tid, ix, iy);
    const bool valid = ix < C.grid.n && iy < C.grid.n;
    for (int c = 0; c < nch; ++c) {
        int u0, u1;
        chunk_views(C.n_views, g, G, chunk, c, u0, u1);
        uint32_t rows = 0;
        for (int u = u0; u < u1; ++u) {
            int n = 0;
            if (valid) pixel_pairs(C, E, rec, views, ix, iy, u, u + 1, [&](int, float) { ++n; });
            rows += (uint32_t)__reduce_max_sync(0xffffffffu, n);
        }
        const size_t e = (size_t)b * nch + c;
        if ((tid & 31) == 0) warp_rows[e * (kBTThreads / 32) + (tid >> 5)] = rows;
    }
}

// Table pass 2: the pairs (stage slot, weight) at their rows: view u of the chunk
// from the warp's row offset of u, pair j of a lane at row bp_row[(e, warp)] + j
// (two rows side by side per lane).  The slots start as kBTNoSlot (memset).
__global__ void __launch_bounds__(kBTThreads) k_fpb_fill(GeomC C, ExcTable E, const RayRec* rec,
                                                         const ViewF* views, const uint32_t* __restrict__ span,
                                                         int G, int chunk, int nch,
                                                         const uint32_t* __restrict__ bp_row, float* bp_w,
                                                         uint16_t* bp_slot) {
    const int b = blockIdx.x, t = b / G, g = b % G, tid = threadIdx.x, lane = tid & 31;
    int ix, iy;
    bt_pixel(C.grid.n, t, tid, ix, iy);
    const bool valid = ix < C.grid.n && iy < C.grid.n;
    for (int c = 0; c < nch; ++c) {
        int u0, u1;
        chunk_views(C.n_views, g, G, chunk, c, u0, u1);
        int off[kBTMaxChunk], tlo[kBTMaxChunk], wid[kBTMaxChunk];
        chunk_offsets(span, t, C.n_views, u0, u1, off, tlo, wid);
        const size_t e = (size_t)b * nch + c;
        const size_t row = bp_row[e * (kBTThreads / 32) + (tid >> 5)];
        int j0 = 0;   // the warp's first row of view u
        for (int u = u0; u < u1; ++u) {
            int n = 0;
            if (valid) pixel_pairs(C, E, rec, views, ix, iy, u, u + 1, [&](int, float) { ++n; });
            const int K = __reduce_max_sync(0xffffffffu, n);
            int j = j0;
            if (valid)
                pixel_pairs(C, E, rec, views, ix, iy, u, u + 1, [&](int l, float w) {
                    const int i = u - u0;
                    const int slot = off[i] + (l - u * C.n_bins) - tlo[i];
                    const size_t at = (row + (j & ~1)) * 32 + 2 * lane + (j & 1);   // rows j, j + 1 side by side
                    bp_w[at] = w;
                    bp_slot[at] = (uint16_t)slot;
                    ++j;
                });
            j0 += K;
        }
    }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}

// One stage buffer of S slots: the step halves (b2 and S in s0.x..s1.z), b0 and
// b1 (the .zw of the weight half), and the ray index of each slot.
struct StageBuf {
    float4* s0;
    float4* s1;
    float2* b01;
    int* ray;
    __device__ StageBuf(float4* base, int S)
        : s0(base), s1(base + S), b01(reinterpret_cast<float2*>(base + 2 * S)),
          ray(reinterpret_cast<int*>(reinterpret_cast<float2*>(base + 2 * S) + S)) {}
};
// float4 units per stage buffer of S slots (S a multiple of 4: 44 S bytes).
__host__ __device__ __forceinline__ int stage_f4(int S) { return (44 * S) / 16; }

// Stage entry e's rays (bp_rays[bp_roff[e] ..]) into the buffer, asynchronously.
__device__ __forceinline__ void stage_entry(const FpTables& T, const RayRec* rec, const RayStep* steps, size_t e,
                                            StageBuf B) {
    const uint32_t r0 = __ldg(T.bp_roff + e), nr = __ldg(T.bp_roff + e + 1) - r0;
    for (uint32_t r = threadIdx.x; r < nr; r += kBTThreads) {
        const int l = __ldg(T.bp_rays + r0 + r);
        cp_async16(B.s0 + r, &steps[l].s0);
        cp_async16(B.s1 + r, &steps[l].s1);
        cp_async8(B.b01 + r, &rec[l].r1.z);
        B.ray[r] = l;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The nine channels of one pair from a stage slot.
__device__ __forceinline__ void bp_accumulate_slot(float acc[9], float w, const StageBuf& B, int s) {
    const float2 b = B.b01[s];
    const float4 s0 = B.s0[s], s1 = B.s1[s];
    acc[0] = fmaf(w, b.x, acc[0]);
    acc[1] = fmaf(w, b.y, acc[1]);
    acc[2] = fmaf(w, s0.x, acc[2]);
    acc[3] = fmaf(w, s0.y, acc[3]);
    acc[4] = fmaf(w, s0.z, acc[4]);
    acc[5] = fmaf(w, s0.w, acc[5]);
    acc[6] = fmaf(w, s1.x, acc[6]);
    acc[7] = fmaf(w, s1.y, acc[7]);
    acc[8] = fmaf(w, s1.z, acc[8]);
}

// a6 from the blocked table for block b = t G + g: each pixel's nine channels
// over its group's views, written to part ([G][9][P]); the group sums and the
// step follow in a second pass.  The chunks go through two stage buffers (smem):
// chunk c + 1 is copied while chunk c is summed.  PARTIAL: only the rays of the
// views [V0, V1) (one GPU's share of a split solve).  Every thread of the block
// must call this (it contains block barriers).
template <bool PARTIAL>
__device__ __forceinline__ void fpb_block(const GeomC& C, const FpTables& T, const RayRec* rec, int V0, int V1,
                                          float* part, int b, float4* smem) {
    const int G = T.bp_groups, t = b / G, g = b % G, tid = threadIdx.x, lane = tid & 31;
    const int S = T.bp_slots, nch = T.bp_nch, nb = C.n_bins;
    int ix, iy;
    bt_pixel(C.grid.n, t, tid, ix, iy);
    const bool valid = ix < C.grid.n && iy < C.grid.n;
    const RayStep* steps = ray_steps(rec, C.n_views * nb);
    const int l_lo = V0 * nb, l_hi = V1 * nb;
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const size_t e0 = (size_t)b * nch;
    // PARTIAL: only the chunks whose views meet [V0, V1), a contiguous run of the
    // group's chunks (the same for every thread of the block), so a rank streams
    // the table of its own views only; the per-slot test below keeps the rays of
    // a chunk that straddles V0 or V1 apart
    int c_lo = 0, c_hi = nch;
    if (PARTIAL) {
        c_lo = nch;
        c_hi = 0;
        for (int c = 0; c < nch; ++c) {
            int u0, u1;
            chunk_views(C.n_views, g, G, T.bp_chunk, c, u0, u1);
            if (u0 < u1 && u0 < V1 && u1 > V0) {
                c_lo = min(c_lo, c);
                c_hi = c + 1;
            }
        }
    }
    const StageBuf B0(smem, S), B1(smem + stage_f4(S), S);
    if (c_lo < c_hi) stage_entry(T, rec, steps, e0 + c_lo, (c_lo & 1) ? B1 : B0);
    for (int c = c_lo; c < c_hi; ++c) {
        const StageBuf& B = (c & 1) ? B1 : B0;
        if (c + 1 < c_hi) {   // the next chunk into the other buffer (free since the barrier ending chunk c - 1)
            stage_entry(T, rec, steps, e0 + c + 1, (c & 1) ? B0 : B1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();   // chunk c staged by every thread
        const size_t e = e0 + c;
        const uint32_t* rp = T.bp_row + e * (kBTThreads / 32) + (tid >> 5);
        const size_t row = __ldg(rp);                  // even
        const int n = (int)(__ldg(rp + 1) - row);      // the warp's rows (even): the same for every lane
        const float2* wp = reinterpret_cast<const float2*>(T.bp_w + row * 32) + lane;
        const ushort2* sp = reinterpret_cast<const ushort2*>(T.bp_slot + row * 32) + lane;
        auto take = [&](float w, unsigned s) {
            if (s != kBTNoSlot && (!PARTIAL || (B.ray[s] >= l_lo && B.ray[s] < l_hi))) bp_accumulate_slot(acc, w, B, s);
        };
        int j = 0;
        for (; j + 7 < n; j += 8) {   // eight table entries (four loads of two) in flight
            float2 w[4];
            ushort2 sl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                w[q] = ld_stream(wp + 32 * q);
                sl[q] = ld_stream(sp + 32 * q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                take(w[q].x, sl[q].x);
                take(w[q].y, sl[q].y);
            }
            wp += 128;
            sp += 128;
        }
        for (; j < n; j += 2, wp += 32, sp += 32) {
            const float2 w = ld_stream(wp);
            const ushort2 sl = ld_stream(sp);
            take(w.x, sl.x);
            take(w.y, sl.y);
        }
        __syncthreads();   // this buffer is read by everyone before chunk c + 2 overwrites it
    }
    if (valid) {
        const size_t P_ = (size_t)C.grid.n * C.grid.n, k = (size_t)iy * C.grid.n + ix;
#pragma unroll
        for (int ch = 0; ch < 9; ++ch) part[((size_t)g * 9 + ch) * P_ + k] = acc[ch];
    }
}

template <bool PARTIAL>
__global__ void __launch_bounds__(kBTThreads) k_fpb_bp(GeomC C, FpTables T, const RayRec* rec, int V0, int V1,
                                                       float* part) {
    extern __shared__ float4 bt_smem[];   // two stage buffers
    fpb_block<PARTIAL>(C, T, rec, V0, V1, part, blockIdx.x, bt_smem);
}

// The view groups of pixel k added in group order (as bp_finish does).
__device__ __forceinline__ void fpb_sum(const float* __restrict__ part, int G, size_t P_, size_t k, float acc[9]) {
#pragma unroll
    for (int ch = 0; ch < 9; ++ch) acc[ch] = part[(size_t)ch * P_ + k];
    for (int gg = 1; gg < G; ++gg)
#pragma unroll
        for (int ch = 0; ch < 9; ++ch) acc[ch] += part[((size_t)gg * 9 + ch) * P_ + k];
}

// The view groups' channels added in group order (as bp_finish does), then a7
// for every pixel; PARTIAL: the sum goes to chan ([9][P]) instead.
template <bool PARTIAL>
__global__ void k_fpb_finish(GeomC C, StepParams P, SolveD D, const float* __restrict__ part, int G, float* chan) {
    const int P_ = C.grid.n * C.grid.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P_) return;
    float acc[9];
    fpb_sum(part, G, P_, k, acc);
    if (PARTIAL) {
#pragma unroll
        for (int ch = 0; ch < 9; ++ch) chan[(size_t)ch * P_ + k] = acc[ch];
    } else {
        pixel_step(C, P, D, k, acc);
    }
}

constexpr int kReduceThreads = 1024;

// Fixed-order sum of the partials: four independent strided accumulators per
// thread, then a block tree (deterministic for a given n).
__device__ __forceinline__ void dtpl_reduce_body(const double* part, int n, double* out) {
    __shared__ double red[kReduceThreads / 32];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * kReduceThreads < n; i += 4 * kReduceThreads) {
        s0 += part[i];
        s1 += part[i + kReduceThreads];
        s2 += part[i + 2 * kReduceThreads];
        s3 += part[i + 3 * kReduceThreads];
    }
    for (; i < n; i += kReduceThreads) s0 += part[i];
    const double t = block_sum((s0 + s1) + (s2 + s3), red);
    if (threadIdx.x == 0) *out = t;
}

__global__ void __launch_bounds__(kReduceThreads) k_dtpl_reduce(const double* part, int n, double* out) {
    dtpl_reduce_body(part, n, out);
}

// ------------------------------------------------------------------ batched (multi-solve) kernels
//
// Many independent solves of different sizes in one launch per step.  Each
// launch walks a work list of (solve, tile) items: CTA i takes items i,
// i + gridDim.x, ...  With one CTA per item this is a flat grid scheduled by the
// hardware; with fewer CTAs it is a persistent grid.  Every ray and pixel runs
// the same arithmetic as in the per-solve kernels, so each solve's iterates
// are bit-identical to its own plain path whatever the batch around it.

__global__ void __launch_bounds__(kBatchProjMaxThreads) k_batch_proj(const SolveDesc* __restrict__ sd,
                                                                     const int2* __restrict__ items, int n_items) {
    const int vb = blockDim.x >> 5;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = __ldg(items + it);
        const SolveDesc& d = sd[w.x];
        const GeomC C = d.C;
        const int nbx = (C.n_bins + 31) >> 5, nby = (C.n_views + vb - 1) / vb;
        // views fastest, bin groups centre-out (long central rays first), as in k_mocca_proj
        const int bx = centre_out(w.y / nby, nbx);
        const int l = ray_at(C, bx, w.y % nby, vb);
        if (l >= 0) {
            if (d.T.fwd_w) fp_proj_ray(d.T, d.D, l, (l / C.n_bins) * nbx + bx);   // the solve's table
            else proj_ray(C, d.E, d.rec, d.D, l);
        }
    }
}

// Batched back-projection from the solves' blocked tables: item (solve, block b)
// runs fpb_block; the dynamic shared memory holds the largest solve's stages.
__global__ void __launch_bounds__(kBTThreads) k_batch_fpb_bp(const SolveDesc* __restrict__ sd,
                                                             const int2* __restrict__ items, int n_items) {
    extern __shared__ float4 bt_smem[];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = __ldg(items + it);
        const SolveDesc& d = sd[w.x];
        fpb_block<false>(d.C, d.T, d.rec, 0, d.C.n_views, d.T.bp_part, w.y, bt_smem);
    }
}

// The view groups added and a7, item (solve, block of 256 pixels).
__global__ void __launch_bounds__(256) k_batch_fpb_finish(const SolveDesc* __restrict__ sd,
                                                          const int2* __restrict__ items, int n_items) {
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = __ldg(items + it);
        const SolveDesc& d = sd[w.x];
        const size_t P_ = (size_t)d.C.grid.n * d.C.grid.n, k = (size_t)w.y * 256 + threadIdx.x;
        if (k < P_) {
            float acc[9];
            fpb_sum(d.T.bp_part, d.T.bp_groups, P_, k, acc);
            pixel_step(d.C, d.P, d.D, (int)k, acc);
        }
    }
}

__global__ void __launch_bounds__(kFwdThreads, 5) k_batch_ray(const SolveDesc* __restrict__ sd,
                                                              const int2* __restrict__ items, int n_items) {
    __shared__ float sm[kSmemStride * kMaxEnergies];
    int cur = -1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = __ldg(items + it);
        const SolveDesc& d = sd[w.x];
        if (w.x != cur) {   // the same for every thread of the block
            __syncthreads();
            load_mu_smem(d.S, sm);
            __syncthreads();
            cur = w.x;
        }
        const GeomC C = d.C;
        const int nbx = (C.n_bins + 31) >> 5, bx = w.y % nbx, by = w.y / nbx;
        const int l = ray_at(C, bx, by, kFwdThreads / 32);
        const double dsum = l >= 0 ? ray_step<false, 4>(C, d.rec, d.S, d.P, d.D, sm, l) : 0.0;
        warp_partial(C, bx, warp_view(by, kFwdThreads / 32), dsum, d.D.dtpl_part);
    }
}

// 512 threads = kBpPix pixels x 8 thread groups.  A solve with G view groups
// (G divides 8) takes 8 / G pixel tiles per item, so the block stays full.
__global__ void __launch_bounds__(kBpMaxThreads) k_batch_bp(const SolveDesc* __restrict__ sd,
                                                           const int2* __restrict__ items, int n_items, int tx) {
    __shared__ float red[7 * 9 * kBpPix];
    const int pix = threadIdx.x % kBpPix, z = threadIdx.x / kBpPix, ty = kBpPix / tx;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = __ldg(items + it);
        const SolveDesc& d = sd[w.x];
        const GeomC C = d.C;
        const int G = d.bp_groups, sub = z / G, g = z % G;
        const int ntx = (C.grid.n + tx - 1) / tx, nty = (C.grid.n + ty - 1) / ty;
        const int tile = w.y * (8 / G) + sub;
        int ix = C.grid.n, iy = C.grid.n;   // outside the image: no work, but the barrier is reached
        if (tile < ntx * nty) {
            ix = (tile % ntx) * tx + pix % tx;
            iy = (tile / ntx) * ty + pix / tx;
        }
        bp_pixel(C, d.E, d.rec, d.views, d.P, d.D, ix, iy, pix, g, G, red + sub * (G - 1) * 9 * kBpPix);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kReduceThreads) k_batch_dtpl(const SolveDesc* __restrict__ sd) {
    const SolveDesc& d = sd[blockIdx.x];
    dtpl_reduce_body(d.D.dtpl_part, d.n_part, d.dtpl_out);
}

inline int blocks(int n, int t) { return (n + t - 1) / t; }

// The column-major copy of xbar (P + ix n + iy) from the row-major maps.
__global__ void k_xbar_columns(int n, float4* xbar) {
    const int P = n * n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x)
        xbar[P + (k % n) * n + k / n] = xbar[k];
}

}  // namespace

cudaError_t launch_forward4(const GeomC& C, const ExcTable& E, const RayRec* rec, const float4* x, float4* g,
                            cudaStream_t st) {
    k_forward4<<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, E, rec, x, g);
    return cudaGetLastError();
}

cudaError_t launch_backproject4(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                const float4* rf, float4* img, cudaStream_t st) {
    dim3 grid(blocks(C.grid.n, kBpTileX), blocks(C.grid.n, kBpTileY)), blk(kBpTileX, kBpTileY);
    k_backproject4<<<grid, blk, 0, st>>>(C, E, rec, views, rf, img);
    return cudaGetLastError();
}

cudaError_t launch_counts(const GeomC& C, const ExcTable& E, const RayRec* rec, const SpecD& S, const float4* f,
                          float4* chat, const float4* c, double* dtpl_part, cudaStream_t st) {
    if (S.n_windows == 5)
        k_counts<5><<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, E, rec, S, f, chat, c, dtpl_part);
    else
        k_counts<4><<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, E, rec, S, f, chat, c, dtpl_part);
    return cudaGetLastError();
}

cudaError_t launch_mocca_proj(const GeomC& C, const ExcTable& E, const RayRec* rec, const SolveD& D,
                              cudaStream_t st, int v0, int v1, const FpTables* T) {
    if (v1 < 0) v1 = C.n_views;
    const dim3 fg = fwd_grid(C.n_bins, v1 - v0);
    if (T) k_fp_proj<<<dim3(fg.y, fg.x), kFwdThreads, 0, st>>>(C, *T, D, v0, v1);
    else k_mocca_proj<<<dim3(fg.y, fg.x), kFwdThreads, 0, st>>>(C, E, rec, D, v0, v1);
    return cudaGetLastError();
}

cudaError_t launch_mocca_ray(const GeomC& C, RayRec* rec, const SpecD& S, const StepParams& P, const SolveD& D,
                             cudaStream_t st, int v0, int v1) {
    if (v1 < 0) v1 = C.n_views;
    if (S.n_windows == 5)
        k_mocca_ray<false, 5><<<fwd_grid(C.n_bins, v1 - v0), kFwdThreads, 0, st>>>(C, rec, S, P, D, v0, v1);
    else
        k_mocca_ray<false, 4><<<fwd_grid(C.n_bins, v1 - v0), kFwdThreads, 0, st>>>(C, rec, S, P, D, v0, v1);
    return cudaGetLastError();
}

cudaError_t launch_mocca_ray_keep(const GeomC& C, RayRec* rec, const SpecD& S, const StepParams& P,
                                  const SolveD& D, cudaStream_t st) {
    if (S.n_windows != 4) return cudaErrorInvalidValue;   // nested MOCCA keeps four-window models
    k_mocca_ray<true, 4><<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, rec, S, P, D, 0, C.n_views);
    return cudaGetLastError();
}

cudaError_t launch_mocca_ray_inner(const GeomC& C, RayRec* rec, const SolveD& D, cudaStream_t st) {
    k_mocca_ray_inner<<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, rec, D);
    return cudaGetLastError();
}

// The table-driven back-projection: the blocked pass into T.bp_part, then the
// group sums with a7 (or into chan).
template <bool PARTIAL>
cudaError_t launch_fpb(const GeomC& C, const FpTables& T, const RayRec* rec, const StepParams& P, const SolveD& D,
                       int v0, int v1, float* chan, cudaStream_t st) {
    const size_t smem = sizeof(float4) * 2 * (size_t)stage_f4(T.bp_slots);
    k_fpb_bp<PARTIAL><<<bt_tiles(C.grid.n) * T.bp_groups, kBTThreads, smem, st>>>(C, T, rec, v0, v1, T.bp_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fpb_finish<PARTIAL><<<blocks(C.grid.n * C.grid.n, 256), 256, 0, st>>>(C, P, D, T.bp_part, T.bp_groups, chan);
    return cudaGetLastError();
}

cudaError_t launch_mocca_bp(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                            const StepParams& P, const SolveD& D, cudaStream_t st, const FpTables* T) {
    if (T && T->bp_w) return launch_fpb<false>(C, *T, rec, P, D, 0, C.n_views, nullptr, st);
    const int G = bp_view_groups(C.grid.n * C.grid.n, C.n_views);
    dim3 grid(blocks(C.grid.n, kBpPixX), blocks(C.grid.n, kBpPixY)), blk(kBpPixX, kBpPixY, G);
    const size_t smem = sizeof(float) * (size_t)(G - 1) * 9 * kBpPix;
    k_mocca_bp<false><<<grid, blk, smem, st>>>(C, E, rec, views, P, D, 0, C.n_views, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_mocca_bp_partial(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                    const StepParams& P, const SolveD& D, int v0, int v1, float* chan,
                                    cudaStream_t st, const FpTables* T) {
    if (T && T->bp_w) return launch_fpb<true>(C, *T, rec, P, D, v0, v1, chan, st);
    const int G = bp_view_groups(C.grid.n * C.grid.n, v1 - v0);
    dim3 grid(blocks(C.grid.n, kBpPixX), blocks(C.grid.n, kBpPixY)), blk(kBpPixX, kBpPixY, G);
    const size_t smem = sizeof(float) * (size_t)(G - 1) * 9 * kBpPix;
    k_mocca_bp<true><<<grid, blk, smem, st>>>(C, E, rec, views, P, D, v0, v1, chan);
    return cudaGetLastError();
}

cudaError_t launch_xbar_columns(int n, float4* xbar, cudaStream_t st) {
    const int P = n * n, blocks = (P + 255) / 256 < 4096 ? (P + 255) / 256 : 4096;
    k_xbar_columns<<<blocks, 256, 0, st>>>(n, xbar);
    return cudaGetLastError();
}

cudaError_t launch_fp_fwd_count(const GeomC& C, const ExcTable& E, const RayRec* rec, int* cnt,
                                uint32_t* warp_rows, cudaStream_t st) {
    k_fp_fwd_count<<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, E, rec, cnt, warp_rows);
    return cudaGetLastError();
}

cudaError_t launch_fp_fwd_fill(const GeomC& C, const ExcTable& E, const RayRec* rec, const uint32_t* fwd_row,
                               float* fwd_w, int16_t* fwd_d, int* fwd_k0, int* bad, cudaStream_t st) {
    k_fp_fwd_fill<<<fwd_grid(C.n_bins, C.n_views), kFwdThreads, 0, st>>>(C, E, rec, fwd_row, fwd_w, fwd_d, fwd_k0,
                                                                         bad);
    return cudaGetLastError();
}
cudaError_t launch_fpb_span(const GeomC& C, const ViewF* views, uint32_t* span, cudaStream_t st) {
    k_fpb_span<<<bt_tiles(C.grid.n), kBTThreads, 0, st>>>(C, views, span);
    return cudaGetLastError();
}

cudaError_t launch_fpb_count(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views, int G,
                             int chunk, int nch, uint32_t* warp_rows, cudaStream_t st) {
    k_fpb_count<<<bt_tiles(C.grid.n) * G, kBTThreads, 0, st>>>(C, E, rec, views, G, chunk, nch, warp_rows);
    return cudaGetLastError();
}

cudaError_t launch_fpb_fill(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                            const uint32_t* span, int G, int chunk, int nch, const uint32_t* bp_row, float* bp_w,
                            uint16_t* bp_slot, cudaStream_t st) {
    k_fpb_fill<<<bt_tiles(C.grid.n) * G, kBTThreads, 0, st>>>(C, E, rec, views, span, G, chunk, nch, bp_row, bp_w,
                                                               bp_slot);
    return cudaGetLastError();
}

int fpb_stage_bytes(int slots) { return 2 * 16 * stage_f4(slots); }

cudaError_t launch_mocca_apply(const GeomC& C, const StepParams& P, const SolveD& D, const float* chan,
                               cudaStream_t st) {
    k_mocca_apply<<<blocks(C.grid.n * C.grid.n, 128), 128, 0, st>>>(C, P, D, chan);
    return cudaGetLastError();
}

cudaError_t launch_dtpl_reduce(const double* part, int n, double* out, cudaStream_t st) {
    k_dtpl_reduce<<<1, kReduceThreads, 0, st>>>(part, n, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_proj(const SolveDesc* sd, const int2* items, int n_items, int vb, int grid,
                              cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    k_batch_proj<<<grid > 0 ? grid : n_items, 32 * vb, 0, st>>>(sd, items, n_items);
    return cudaGetLastError();
}

cudaError_t launch_batch_ray(const SolveDesc* sd, const int2* items, int n_items, int grid, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    k_batch_ray<<<grid > 0 ? grid : n_items, kFwdThreads, 0, st>>>(sd, items, n_items);
    return cudaGetLastError();
}

cudaError_t launch_batch_bp(const SolveDesc* sd, const int2* items, int n_items, int tx, int grid,
                            cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    k_batch_bp<<<grid > 0 ? grid : n_items, kBpMaxThreads, 0, st>>>(sd, items, n_items, tx);
    return cudaGetLastError();
}

cudaError_t launch_batch_dtpl(const SolveDesc* sd, int n_solves, cudaStream_t st) {
    if (n_solves <= 0) return cudaSuccess;
    k_batch_dtpl<<<n_solves, kReduceThreads, 0, st>>>(sd);
    return cudaGetLastError();
}

cudaError_t launch_batch_fpb(const SolveDesc* sd, const int2* items, int n_items, const int2* fin_items,
                             int n_fin, int grid, size_t smem, cudaStream_t st) {
    if (n_items > 0) {
        k_batch_fpb_bp<<<grid > 0 ? grid : n_items, kBTThreads, smem, st>>>(sd, items, n_items);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_fin <= 0) return cudaSuccess;
    k_batch_fpb_finish<<<n_fin, 256, 0, st>>>(sd, fin_items, n_fin);
    return cudaGetLastError();
}

cudaError_t batch_resident_ctas(int kernel, int threads, int* per_sm, size_t smem) {
    switch (kernel) {
        case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_proj, threads, 0);
        case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_ray, threads, 0);
        case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_fpb_bp, threads, smem);
        default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_bp, threads, 0);
    }
}

}  // namespace osscir
