// Internal device-side definitions shared by the library's kernels.
//
// Projector X (Eq. fullModel's X_{l,k}): X_{l,k} is the length of ray l inside
// pixel k.  Both the ray-driven forward projection and the pixel-driven
// back-projection evaluate the SAME function x_weight(ray, ix, iy) on the SAME
// per-ray FP32 record, so the two kernels use bit-identical weights and are
// exact adjoints up to summation order.  Membership of (l, k) in the footprint
// is decided in FP32 when the FP32 chord is farther than a rigorous per-ray
// error bound from zero, and otherwise read from a per-geometry exception
// table that a setup kernel fills in FP64 (chord > 1e-9 pixel), so the
// footprint equals the FP64 definition exactly.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace osscir {

constexpr int NM = 3;  // basis materials

// Window vectors.  A per-ray quantity over the W energy windows (counts, duals,
// spectral weights) is stored in whole float4s: one for W = 4, two for W = 5
// (components W..7 zero), so every load is an aligned 16-byte load.
template <int W>
constexpr int win_f4() { return (W + 3) / 4; }

template <int W, bool LDG = false>
__device__ __forceinline__ void win_load(const float4* p, float (&v)[W]) {
    static_assert(W >= 4 && W <= 8, "4 to 8 windows");
    const float4 a = LDG ? __ldg(p) : p[0];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    if constexpr (W > 4) {
        const float4 b = LDG ? __ldg(p + 1) : p[1];
        const float t[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int w = 4; w < W; ++w) v[w] = t[w - 4];
    }
}

template <int W>
__device__ __forceinline__ void win_store(float4* p, const float (&v)[W]) {
    p[0] = make_float4(v[0], v[1], v[2], v[3]);
    if constexpr (W > 4) {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int w = 4; w < W; ++w) t[w - 4] = v[w];
        p[1] = make_float4(t[0], t[1], t[2], t[3]);
    }
}

// Pixel grid: n x n pixels of side h, planes at x0 + i h (i = 0..n), x0 = -n h / 2.
struct GridF {
    int n;
    float h, x0;
};

__device__ __forceinline__ float grid_plane(const GridF& G, int i) {
    return __fmaf_rn(static_cast<float>(i), G.h, G.x0);
}

// Per-ray record, 64 bytes per ray l = v * n_bins + b, stored as two arrays of
// 32-byte halves in one allocation of 2 L RayRec: the weight half rec[l] and the
// step half ray_steps(rec, L)[l].  Consecutive rays' halves are contiguous, so a
// warp gathering the weight halves of neighbouring rays touches half as many
// cache lines as with whole records.
//   rec[l].r0 = (bx, by, idx, idy)    foot point of the ray line nearest the origin and
//                                     the reciprocal unit-direction components (inf if 0)
//   rec[l].r1 = (ex, ey, b0, b1)      FP32 error bounds on t for x- and y-planes; b = alpha^T y'
//   step.s0   = (b2, S00, S01, S02)   b and the block step matrix S = sum_w alpha_w alpha_w^T / |alpha_w|
//   step.s1   = (S11, S12, S22, -)
// r0 and r1.xy are written once per geometry; the rest once per MOCCA iteration.
struct __align__(32) RayRec {
    float4 r0, r1;
};
struct __align__(32) RayStep {
    float4 s0, s1;
};
__host__ __device__ __forceinline__ RayStep* ray_steps(RayRec* rec, int L) {
    return reinterpret_cast<RayStep*>(rec + L);
}
__host__ __device__ __forceinline__ const RayStep* ray_steps(const RayRec* rec, int L) {
    return reinterpret_cast<const RayStep*>(rec + L);
}

// t(X) for the x-plane X along the unit direction from the foot point (mm).
__device__ __forceinline__ float t_plane(float X, float b, float inv_d) {
    return __fmul_rn(__fsub_rn(X, b), inv_d);
}

// The error bound of a chord: that of the plane deciding each end (both on a tie).
__device__ __forceinline__ float chord_bound(float txl, float txh, float tyl, float tyh, float ex, float ey) {
    const float elo = txl > tyl ? ex : (tyl > txl ? ey : fmaxf(ex, ey));
    const float ehi = txh < tyh ? ex : (tyh < txh ? ey : fmaxf(ex, ey));
    return __fadd_rn(elo, ehi);
}

// The chord of a pixel from the ray parameters of its four planes: the ray is
// inside the pixel for max(entry planes) < t < min(exit planes).  The planes of
// each axis are ordered by the sign of the reciprocal direction (t is monotone
// in the plane position), which equals fminf/fmaxf on these values.
__device__ __forceinline__ void chord_from_planes(float tx0, float tx1, float ty0, float ty1, float idx, float idy,
                                                  float ex, float ey, float& w, float& eb) {
    const float txl = idx >= 0.0f ? tx0 : tx1, txh = idx >= 0.0f ? tx1 : tx0;
    const float tyl = idy >= 0.0f ? ty0 : ty1, tyh = idy >= 0.0f ? ty1 : ty0;
    w = __fsub_rn(fminf(txh, tyh), fmaxf(txl, tyl));
    eb = chord_bound(txl, txh, tyl, tyh, ex, ey);
}

// FP32 chord of pixel (ix, iy) on the ray and the error bound that applies to it.
__device__ __forceinline__ void chord32(const float4& r0, float ex, float ey, const GridF& G, int ix,
                                        int iy, float& w, float& eb) {
    chord_from_planes(t_plane(grid_plane(G, ix), r0.x, r0.z), t_plane(grid_plane(G, ix + 1), r0.x, r0.z),
                      t_plane(grid_plane(G, iy), r0.y, r0.w), t_plane(grid_plane(G, iy + 1), r0.y, r0.w), r0.z,
                      r0.w, ex, ey, w, eb);
}

// Footprint exception table (CSR over rays): entries (key, weight bits) of the
// ray's pixels whose FP32 chord is within its error bound of zero.  key =
// major * n + minor, with major the pixel's index along the ray's dominant axis
// (iy when |d_y| >= |d_x|, else ix) and minor the other; each ray's entries
// are in increasing key order (the order in which the setup pass enumerates
// them).  A ray running exactly along a grid line has about 2n entries.
struct ExcTable {
    const int* off;    // [L + 1]
    const int2* ent;   // [off[L]]
};

__device__ __forceinline__ bool ray_rows(const float4& r0) { return fabsf(r0.w) <= fabsf(r0.z); }

__device__ __forceinline__ int exc_key(bool rows, int n, int ix, int iy) { return rows ? iy * n + ix : ix * n + iy; }

// Binary search of the ray's entries for key.
__device__ __forceinline__ float exc_lookup(const ExcTable& E, int l, int key) {
    int lo = __ldg(E.off + l), hi = __ldg(E.off + l + 1);
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&E.ent[mid].x) < key) lo = mid + 1;
        else hi = mid;
    }
    if (lo < end) {
        const int2 e = __ldg(E.ent + lo);
        if (e.x == key) return __int_as_float(e.y);
    }
    return 0.0f;
}

// Membership decision shared by both projectors: chord w > bound -> member with
// weight w; w < -bound -> not a member; otherwise the FP64 table decides.  The
// bound of a chord never exceeds 2 max(ex, ey), so that test settles most pairs
// before the exact bound is formed; the outcome is the same either way.
__device__ __forceinline__ float member_weight(float w, float txl, float txh, float tyl, float tyh, float ex,
                                               float ey, const ExcTable& E, int l, int key) {
    const float ebmax = 2.0f * fmaxf(ex, ey);
    if (w > ebmax) return w;
    if (w < -ebmax) return 0.0f;
    const float eb = chord_bound(txl, txh, tyl, tyh, ex, ey);
    if (w > eb) return w;
    if (w < -eb) return 0.0f;
    return exc_lookup(E, l, key);   // also reached by NaN (axis-parallel rays)
}

// X_{l,k}: the weight both projectors use.  The entry and exit parameters of
// each axis are the min and max of its two plane parameters: t is monotone in
// the plane position for a finite reciprocal direction, so this is the
// direction-sign choice of chord_from_planes; only an axis-parallel ray
// (reciprocal infinite, possibly a NaN parameter) can differ, and such a ray
// has infinite error bounds, so its weight comes from the FP64 table either way.
__device__ __forceinline__ float x_weight(const float4& r0, float ex, float ey, const GridF& G,
                                          const ExcTable& E, int l, int ix, int iy) {
    const float tx0 = t_plane(grid_plane(G, ix), r0.x, r0.z), tx1 = t_plane(grid_plane(G, ix + 1), r0.x, r0.z);
    const float ty0 = t_plane(grid_plane(G, iy), r0.y, r0.w), ty1 = t_plane(grid_plane(G, iy + 1), r0.y, r0.w);
    const float txl = fminf(tx0, tx1), txh = fmaxf(tx0, tx1);
    const float tyl = fminf(ty0, ty1), tyh = fmaxf(ty0, ty1);
    const float w = __fsub_rn(fminf(txh, tyh), fmaxf(txl, tyl));
    return member_weight(w, txl, txh, tyl, tyh, ex, ey, E, l, exc_key(ray_rows(r0), G.n, ix, iy));
}

// float -> int with saturation (huge or infinite coordinates stay in range).
__device__ __forceinline__ int sat_floor(float v) {
    return static_cast<int>(floorf(fminf(fmaxf(v, -1.0e9f), 1.0e9f)));
}

// Candidate enumeration of a ray's pixels with their chords: slabs along the
// dominant axis (ROWS: y), within each slab the minor-axis cells the ray can
// touch (with a margin that exceeds the FP32 error of the crossing points).
// Every plane parameter is computed once and shared by the neighbouring
// cells; the chord and bound equal chord32's bit for bit.  Calls
// visit(ix, iy, w, eb) for a superset of the footprint.
template <bool ROWS, class Visit>
__device__ __forceinline__ void ray_chords_dir(const float4& r0, float ex, float ey, const GridF& G, float margin,
                                               Visit&& visit) {
    const float bM = ROWS ? r0.y : r0.x, bm = ROWS ? r0.x : r0.y;
    const float iM = ROWS ? r0.w : r0.z, im = ROWS ? r0.z : r0.w;
    const float slope = iM / im;   // d_minor / d_major, |slope| <= 1 (0 for axis-parallel rays)
    const float xlo = G.x0, xhi = grid_plane(G, G.n);
    int jlo = 0, jhi = G.n - 1;
    if (slope != 0.0f) {
        const float ya = bM + (xlo - margin - bm) / slope;
        const float yb = bM + (xhi + margin - bm) / slope;
        jlo = max(jlo, sat_floor((fminf(ya, yb) - G.x0) / G.h) - 1);
        jhi = min(jhi, sat_floor((fmaxf(ya, yb) - G.x0) / G.h) + 1);
    } else if (bm < xlo - margin || bm > xhi + margin) {
        return;
    }
    const float inv_h = 1.0f / G.h;
    float pM0 = grid_plane(G, jlo);
    float tM0 = t_plane(pM0, bM, iM);
    for (int j = jlo; j <= jhi; ++j) {
        const float pM1 = grid_plane(G, j + 1);
        const float tM1 = t_plane(pM1, bM, iM);
        const float ma = fmaf(slope, pM0 - bM, bm), mb = fmaf(slope, pM1 - bM, bm);
        const int ilo = max(sat_floor((fminf(ma, mb) - margin - G.x0) * inv_h), 0);
        const int ihi = min(sat_floor((fmaxf(ma, mb) + margin - G.x0) * inv_h), G.n - 1);
        if (ilo <= ihi) {
            float tm0 = t_plane(grid_plane(G, ilo), bm, im);
            for (int i = ilo; i <= ihi; ++i) {
                const float tm1 = t_plane(grid_plane(G, i + 1), bm, im);
                float w, eb;
                if (ROWS) {
                    chord_from_planes(tm0, tm1, tM0, tM1, r0.z, r0.w, ex, ey, w, eb);
                    visit(i, j, w, eb);
                } else {
                    chord_from_planes(tM0, tM1, tm0, tm1, r0.z, r0.w, ex, ey, w, eb);
                    visit(j, i, w, eb);
                }
                tm0 = tm1;
            }
        }
        pM0 = pM1;
        tM0 = tM1;
    }
}

template <class Visit>
__device__ __forceinline__ void ray_chords(const float4& r0, float ex, float ey, const GridF& G, float margin,
                                           Visit&& visit) {
    // r0.zw = (1/dx, 1/dy): the ray is row-major (|dy| >= |dx|) iff |1/dy| <= |1/dx|
    if (ray_rows(r0)) ray_chords_dir<true>(r0, ex, ey, G, margin, visit);
    else ray_chords_dir<false>(r0, ex, ey, G, margin, visit);
}

// X_{l,k} for every pixel of ray l with a nonzero weight: visit(k, w).  The
// same slab enumeration as ray_chords, written once in (major, minor)
// coordinates: the membership test is symmetric under exchanging the x and y
// roles (fminf, fmaxf and chord_bound commute with the exchange), so one code
// path serves both orientations and both direction signs, and every weight
// equals x_weight's bit for bit.  A single copy matters: eight specialised
// copies (axis x signs) made instruction fetch the projection's main stall.
// The <= 3 cells a slab can contribute (|slope| <= 1, margin < h/2) are unrolled.
template <class Visit>
__device__ __forceinline__ void ray_weights(const float4& r0, float ex, float ey, const GridF& G, float margin,
                                            const ExcTable& E, int l, Visit&& visit) {
    const bool rows = ray_rows(r0);
    const float bM = rows ? r0.y : r0.x, bm = rows ? r0.x : r0.y;   // foot point, major / minor axis
    const float iM = rows ? r0.w : r0.z, im = rows ? r0.z : r0.w;   // reciprocal direction
    const float eM = rows ? ey : ex, em = rows ? ex : ey;           // plane-parameter error bounds
    const int sM = rows ? G.n : 1, sm = rows ? 1 : G.n;             // pixel-index strides
    const bool PM = iM >= 0.0f, Pm = im >= 0.0f;
    const float slope = iM / im;   // d_minor / d_major, |slope| <= 1 (0 for axis-parallel rays)
    const float xlo = G.x0, xhi = grid_plane(G, G.n);
    int jlo = 0, jhi = G.n - 1;
    if (slope != 0.0f) {
        const float ya = bM + (xlo - margin - bm) / slope;
        const float yb = bM + (xhi + margin - bm) / slope;
        jlo = max(jlo, sat_floor((fminf(ya, yb) - G.x0) / G.h) - 1);
        jhi = min(jhi, sat_floor((fmaxf(ya, yb) - G.x0) / G.h) + 1);
    } else if (bm < xlo - margin || bm > xhi + margin) {
        return;
    }
    const float inv_h = 1.0f / G.h;
    const float c_lo = (-margin - G.x0) * inv_h, c_hi = (margin - G.x0) * inv_h;
    float pM0 = grid_plane(G, jlo);
    float tM0 = t_plane(pM0, bM, iM);
    float m0 = fmaf(slope, pM0 - bM, bm);
#pragma unroll 2   // two slabs per trip: more independent loads in flight
    for (int j = jlo; j <= jhi; ++j) {
        const float pM1 = grid_plane(G, j + 1);
        const float tM1 = t_plane(pM1, bM, iM);
        const float m1 = fmaf(slope, pM1 - bM, bm);
        const int ilo = max(__float2int_rd(fmaf(fminf(m0, m1), inv_h, c_lo)), 0);
        const int ihi = min(__float2int_rd(fmaf(fmaxf(m0, m1), inv_h, c_hi)), G.n - 1);
        const float tMl = PM ? tM0 : tM1, tMh = PM ? tM1 : tM0;
        if (ilo <= ihi) {
            float tm[4];
            tm[0] = t_plane(grid_plane(G, ilo), bm, im);
            tm[1] = t_plane(grid_plane(G, ilo + 1), bm, im);
            tm[2] = t_plane(grid_plane(G, ilo + 2), bm, im);
            tm[3] = t_plane(grid_plane(G, ilo + 3), bm, im);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int i = ilo + c;
                if (i > ihi) break;
                const float tml = Pm ? tm[c] : tm[c + 1], tmh = Pm ? tm[c + 1] : tm[c];
                const float w = __fsub_rn(fminf(tmh, tMh), fmaxf(tml, tMl));
                const float x = member_weight(w, tml, tmh, tMl, tMh, em, eM, E, l, j * G.n + i);
                if (x != 0.0f) visit(j * sM + i * sm, x);
            }
        }
        tM0 = tM1;
        m0 = m1;
    }
}

// Per-view constants for the pixel-driven back-projection: the detector bin
// coordinate of a point q is beta(q) = scale * (q . e_u) / (sid - q . e) + mid
// with e = (cos th, sin th), e_u = (-sin th, cos th).
struct ViewF {
    float c, s;   // cos th, sin th
};

// Library geometry constants shared by all kernels of one context.
struct GeomC {
    GridF grid;
    int n_views, n_bins;
    float sid, scale, mid;   // scale = sdd / bin_mm, mid = (n_bins - 1) / 2
    float margin_mm;         // candidate margin for the ray-driven enumeration
    float margin_bins;       // candidate margin for the pixel-driven enumeration
};

// Candidate bin range of pixel (ix, iy) in a view: bins whose centre ray can
// cross the pixel square (FP32 shadow of the four corners, with a margin).
__device__ __forceinline__ void pixel_bin_range(const GeomC& C, const ViewF& V, int ix, int iy, int& blo,
                                                int& bhi) {
    const float X0 = grid_plane(C.grid, ix), X1 = grid_plane(C.grid, ix + 1);
    const float Y0 = grid_plane(C.grid, iy), Y1 = grid_plane(C.grid, iy + 1);
    float bmin = 3.0e38f, bmax = -3.0e38f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float X = (q & 1) ? X1 : X0, Y = (q & 2) ? Y1 : Y0;
        const float num = -V.s * X + V.c * Y;
        const float den = C.sid - (V.c * X + V.s * Y);
        const float beta = C.scale * __fdividef(num, den) + C.mid;   // 2-ulp division; the margin covers it
        bmin = fminf(bmin, beta);
        bmax = fmaxf(bmax, beta);
    }
    blo = max(0, -sat_floor(-(bmin - C.margin_bins)));
    bhi = min(C.n_bins - 1, sat_floor(bmax + C.margin_bins));
}

}  // namespace osscir
