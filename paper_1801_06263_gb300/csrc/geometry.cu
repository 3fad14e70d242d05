// Per-geometry setup kernels (run once per context): FP64 ray parameters, the
// FP32 per-ray records both projectors read, the FP64-decided footprint
// exception table, the per-ray chord sums (X 1)_l, and debug footprint dumps.
#include "osscir_internal.cuh"
#include "osscir_launch.h"

namespace osscir {

namespace {

constexpr double kPi = 3.14159265358979323846;

// FP64 ray of view v, bin b: foot point B (nearest the origin) and unit direction.
// Source S = sid (cos th, sin th); bin centre D = (sid - sdd)(cos th, sin th) + u_b (-sin th, cos th).
__device__ Ray64 ray64(const GeomD& G, int v, int b) {
    const double th = __ddiv_rn(__dmul_rn(__dadd_rn(G.start_deg, __ddiv_rn(__dmul_rn((double)v, G.arc_deg),
                                                                           (double)G.n_views)),
                                          kPi),
                                180.0);
    const double c = cos(th), s = sin(th);
    const double u = __dmul_rn(__dsub_rn((double)b, __dmul_rn(0.5, (double)(G.n_bins - 1))), G.bin_mm);
    const double back = __dsub_rn(G.sid, G.sdd);
    const double Sx = __dmul_rn(G.sid, c), Sy = __dmul_rn(G.sid, s);
    const double Dx = __dsub_rn(__dmul_rn(back, c), __dmul_rn(u, s));
    const double Dy = __dadd_rn(__dmul_rn(back, s), __dmul_rn(u, c));
    const double ddx = __dsub_rn(Dx, Sx), ddy = __dsub_rn(Dy, Sy);
    const double len = sqrt(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)));
    const double dx = __ddiv_rn(ddx, len), dy = __ddiv_rn(ddy, len);
    const double sd = __dadd_rn(__dmul_rn(Sx, dx), __dmul_rn(Sy, dy));
    return Ray64{__dsub_rn(Sx, __dmul_rn(sd, dx)), __dsub_rn(Sy, __dmul_rn(sd, dy)), dx, dy};
}

// FP64 chord of pixel (ix, iy): the ray is inside the x-slab for t between the
// plane crossings, or for all t when parallel to it and lo <= coordinate < hi.
__device__ double chord64(const Ray64& R, const GeomD& G, int ix, int iy) {
    double lo = -1.0e300, hi = 1.0e300;
    const double b[2] = {R.x, R.y}, d[2] = {R.z, R.w};
    const int idx[2] = {ix, iy};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const double p0 = __dadd_rn(G.x0, __dmul_rn((double)idx[a], G.h));
        const double p1 = __dadd_rn(G.x0, __dmul_rn((double)(idx[a] + 1), G.h));
        if (d[a] == 0.0) {
            if (!(p0 <= b[a] && b[a] < p1)) return 0.0;
        } else {
            const double t0 = __ddiv_rn(__dsub_rn(p0, b[a]), d[a]);
            const double t1 = __ddiv_rn(__dsub_rn(p1, b[a]), d[a]);
            lo = fmax(lo, fmin(t0, t1));
            hi = fmin(hi, fmax(t0, t1));
        }
    }
    return hi > lo ? hi - lo : 0.0;
}

__global__ void k_ray_setup(GeomD G, double r_img, RayRec* rec, Ray64* r64, int L) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const Ray64 R = ray64(G, l / G.n_bins, l % G.n_bins);
    r64[l] = R;
    const double rb = r_img + sqrt(R.x * R.x + R.y * R.y);
    const double u = 1.0 / 8388608.0;   // 2^-23
    const bool aligned = (R.z == 0.0) || (R.w == 0.0);
    const float idx = R.z != 0.0 ? (float)(1.0 / R.z) : INFINITY;
    const float idy = R.w != 0.0 ? (float)(1.0 / R.w) : INFINITY;
    const float ex = aligned ? INFINITY : (float)(u * rb * (5.83 * fabs(1.0 / R.z) + 4.0));
    const float ey = aligned ? INFINITY : (float)(u * rb * (5.83 * fabs(1.0 / R.w) + 4.0));
    RayRec q;
    q.r0 = make_float4((float)R.x, (float)R.y, idx, idy);
    q.r1 = make_float4(ex, ey, 0.f, 0.f);
    rec[l] = q;
    RayStep z;
    z.s0 = z.s1 = make_float4(0.f, 0.f, 0.f, 0.f);
    ray_steps(rec, L)[l] = z;
}

__global__ void k_view_setup(GeomD G, ViewF* views) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.n_views) return;
    const double th = __ddiv_rn(__dmul_rn(__dadd_rn(G.start_deg, __ddiv_rn(__dmul_rn((double)v, G.arc_deg),
                                                                           (double)G.n_views)),
                                          kPi),
                                180.0);
    views[v] = ViewF{(float)cos(th), (float)sin(th)};
}

// Ambiguous candidates (FP32 chord within its error bound of zero) decided in
// FP64; count == nullptr selects the fill pass.
__global__ void k_exc_pass(GeomC C, GeomD G, const RayRec* rec, const Ray64* r64, int* count,
                           const int* off, int2* ent, int L) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const float4 r0 = rec[l].r0;
    const float ex = rec[l].r1.x, ey = rec[l].r1.y;
    const Ray64 R = r64[l];
    int cnt = 0;
    const int base = count ? 0 : off[l];
    const bool rows = ray_rows(r0);
    // ray_chords enumerates (major, minor) in increasing order, so the keys come out sorted
    ray_chords(r0, ex, ey, C.grid, C.margin_mm, [&](int ix, int iy, float w, float eb) {
        if (w > eb || w < -eb) return;
        const double c64 = chord64(R, G, ix, iy);
        if (c64 > G.thr) {
            if (!count) ent[base + cnt] = make_int2(exc_key(rows, C.grid.n, ix, iy), __float_as_int((float)c64));
            ++cnt;
        }
    });
    if (count) count[l] = cnt;
}

// (X 1)_l = sum_k X_{l,k}: the chord of each ray through the image.
__global__ void k_chord(GeomC C, ExcTable E, const RayRec* rec, float* chord, int L) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const float4 r0 = rec[l].r0;
    const float ex = rec[l].r1.x, ey = rec[l].r1.y;
    float acc = 0.f;
    ray_weights(r0, ex, ey, C.grid, C.margin_mm, E, l, [&](int, float w) { acc += w; });
    chord[l] = acc;
}

// Footprint of rays [l0, l0 + n) as the forward projection sees it.
__global__ void k_footprint_rays(GeomC C, ExcTable E, const RayRec* rec, int l0, int n, int cap, int* cnt,
                                 int* pix, float* wt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int l = l0 + j;
    const float4 r0 = rec[l].r0;
    const float ex = rec[l].r1.x, ey = rec[l].r1.y;
    int c = 0;
    ray_weights(r0, ex, ey, C.grid, C.margin_mm, E, l, [&](int k, float w) {
        if (c < cap) {
            pix[(size_t)j * cap + c] = k;
            wt[(size_t)j * cap + c] = w;
        }
        ++c;
    });
    cnt[j] = c;
}

// Footprint of pixels [k0, k0 + n) as the back-projection sees it.
__global__ void k_footprint_pixels(GeomC C, ExcTable E, const RayRec* rec, const ViewF* views, int k0, int n,
                                   int cap, int* cnt, int* ray, float* wt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int k = k0 + j, ix = k % C.grid.n, iy = k / C.grid.n;
    int c = 0;
    for (int v = 0; v < C.n_views; ++v) {
        int blo, bhi;
        pixel_bin_range(C, views[v], ix, iy, blo, bhi);
        for (int b = blo; b <= bhi; ++b) {
            const int l = v * C.n_bins + b;
            const float4 r0 = rec[l].r0;
            const float w = x_weight(r0, rec[l].r1.x, rec[l].r1.y, C.grid, E, l, ix, iy);
            if (w != 0.f) {
                if (c < cap) {
                    ray[(size_t)j * cap + c] = l;
                    wt[(size_t)j * cap + c] = w;
                }
                ++c;
            }
        }
    }
    cnt[j] = c;
}

inline int blocks(int n, int t) { return (n + t - 1) / t; }

}  // namespace

cudaError_t launch_ray_setup(const GeomD& G, double r_img, RayRec* rec, Ray64* r64, ViewF* views,
                             cudaStream_t st) {
    const int L = G.n_views * G.n_bins;
    k_ray_setup<<<blocks(L, 128), 128, 0, st>>>(G, r_img, rec, r64, L);
    k_view_setup<<<blocks(G.n_views, 128), 128, 0, st>>>(G, views);
    return cudaGetLastError();
}

cudaError_t launch_exc_pass(const GeomC& C, const GeomD& G, const RayRec* rec, const Ray64* r64, int* count,
                            const int* off, int2* ent, cudaStream_t st) {
    const int L = G.n_views * G.n_bins;
    k_exc_pass<<<blocks(L, 128), 128, 0, st>>>(C, G, rec, r64, count, off, ent, L);
    return cudaGetLastError();
}

cudaError_t launch_chord(const GeomC& C, const ExcTable& E, const RayRec* rec, float* chord, cudaStream_t st) {
    const int L = C.n_views * C.n_bins;
    k_chord<<<blocks(L, 128), 128, 0, st>>>(C, E, rec, chord, L);
    return cudaGetLastError();
}

cudaError_t launch_footprint_rays(const GeomC& C, const ExcTable& E, const RayRec* rec, int l0, int n, int cap,
                                  int* cnt, int* pix, float* wt, cudaStream_t st) {
    k_footprint_rays<<<blocks(n, 64), 64, 0, st>>>(C, E, rec, l0, n, cap, cnt, pix, wt);
    return cudaGetLastError();
}

cudaError_t launch_footprint_pixels(const GeomC& C, const ExcTable& E, const RayRec* rec, const ViewF* views,
                                    int k0, int n, int cap, int* cnt, int* ray, float* wt, cudaStream_t st) {
    k_footprint_pixels<<<blocks(n, 64), 64, 0, st>>>(C, E, rec, views, k0, n, cap, cnt, ray, wt);
    return cudaGetLastError();
}

}  // namespace osscir
