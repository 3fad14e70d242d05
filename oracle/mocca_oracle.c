/*
 * FP64 CPU oracle: one-step three-material spectral CT reconstruction by MOCCA
 * with m-block-diagonal step-preconditioning (Sidky, Barber, Gilat-Schmidt,
 * Pan, "Three material decomposition for spectral computed tomography enabled
 * by block-diagonal step-preconditioning", arXiv:1801.06263).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library never
 * calls it and shares no code with it.
 *
 * Everything is double precision, written in the paper's notation:
 *   f_{k,m}  material maps (pixel k, material m = PMMA, Al, Gd)
 *   X_{l,k}  intersection length of ray l with pixel k        (Eq. fullModel)
 *   g_{l,m} = sum_k X_{l,k} f_{k,m}   material line integrals
 *   p_{l,i} = sum_m mu_{m,i} g_{l,m}  (Zf)_{l,i}
 *   c^_{w,l} = N_{w,l} sum_i s_{w,l,i} softexp(-p_{l,i})       (Eq. finalModel)
 *   D_TPL = sum_{w,l} c^ - c - c log(c^/c)                     (Eq. DTPL)
 *   A, B of Eq. (aeq); K = A Z;  Sigma, T of the m-block SPC (Sec. 2).
 *
 * Where the paper is silent the following readings are used (each is listed
 * with its reason in the design notes of the repository):
 *   - X: exact (Siddon) intersection lengths; pixels closed on the low side;
 *     a pair (l,k) belongs to the footprint iff its length > 1e-9 pixel_mm.
 *   - MOCCA step (the pseudo-code lives in Barber et al. 2016, not in the
 *     paper): expansion point f0 = xbar = 2 x_n - x_{n-1};  per-ray local
 *     quadratic Q(z) = r^T (z - z0) + 1/2 (z - z0)^T W (z - z0) on z = K f with
 *     W = G^T H+ G, G = (alpha^T alpha)^-1 alpha^T, H+ = the per-ray Hessian of
 *     Sec. 2 with its negative eigenvalues set to zero ("removing directions of
 *     negative curvature", Sec. 1);  dual step = exact preconditioned prox of
 *     Q*:  y' = y - Sigma (W + Sigma)^-1 (y - r);  primal step
 *     x' = argmin_{x in C} 1/2 ||x - (x - T K^T y')||^2_{T^-1} with C = R^3
 *     (default) or a box;  xbar' = 2 x' - x.
 *   - Rays that miss the image keep their dual; pixels seen by no ray keep x.
 *   - 0 log 0 = 0 in D_TPL.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NWMAX 8 /* energy windows: n_windows of the spectra, at most NWMAX */
#define NM 3 /* basis materials */

typedef struct {
    int n;
    double pixel_mm;
    int n_views;
    double arc_deg, start_deg;
    int n_bins;
    double bin_mm, sid_mm, sdd_mm;
} orc_geometry;

typedef struct {
    int n_energies;
    const double *s;  /* [n_bins][nE][W]  normalised spectral response s_{w,l,i} */
    const double *N;  /* [n_bins][W]      incident photons N_{w,l}              */
    const double *mu; /* [3][nE]          mu_{m,i} in 1/mm                       */
    int exp_model;    /* 0: softexp (Eq. finalModel); 1: exp (the standard model, Eq. fullModel) */
    int n_windows;    /* W, the energy windows (1 .. NWMAX); every per-ray window array is [W] */
} orc_spectra;

typedef struct {
    double lambda; /* step-size ratio of the SPC (Sec. 2 leaves it to tuning) */
    int use_box;   /* 0: C = R^3, 1: box lo <= x <= hi                     */
    double lo[3], hi[3];
    int spc;   /* 0: m-block-diagonal SPC (Sec. 2); 1: diagonal SPC (Pock-Chambolle) */
    int model; /* curvature of the local quadratic: 0 the eigen-clipped per-ray Hessian; 1 W = 0
                  (preconditioned gradient step); 2 the Hessian's first term alone, sum_w c_w alpha_w
                  alpha_w^T (Gauss-Newton, always PSD); 3 W = diag(c) on the window line integrals
                  (separable; equal to 2 on the range of K) */
    int inner; /* iterations per local model: 1 single-loop MOCCA; k > 1 nested (see orc_mocca) */
} orc_params;

static const double PI = 3.14159265358979323846;

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ geometry */

/* Source point S and detector-bin centre D of ray (v, b): fan beam, flat
 * detector, source at radius sid on angle start + v * arc / n_views (CCW),
 * detector centre at (sid - sdd) on the same angle, bin centres at
 * u_b = (b - (n_bins-1)/2) * bin_mm along the detector axis (-sin, cos). */
void orc_ray_endpoints(const orc_geometry *G, int v, int b, double S[2], double D[2]) {
    double th = (G->start_deg + (double)v * G->arc_deg / (double)G->n_views) * PI / 180.0;
    double c = cos(th), s = sin(th);
    double u = ((double)b - 0.5 * (double)(G->n_bins - 1)) * G->bin_mm;
    double back = G->sid_mm - G->sdd_mm;
    S[0] = G->sid_mm * c;
    S[1] = G->sid_mm * s;
    D[0] = back * c - u * s;
    D[1] = back * s + u * c;
}

/* Siddon's parametric method (Siddon 1985): the ray S + a (D - S), a in [0, 1],
 * is split at every crossing with a pixel plane, a = (plane - S) / (D - S);
 * each piece lies in one pixel and has length (a_{j+1} - a_j) |D - S|.  The
 * pixel indices are tracked incrementally: the entry column/row is the number
 * of planes already passed at the entry parameter, and every crossing moves
 * the index by one in the direction of travel (a ray parallel to an axis sits
 * in the slab lo <= coordinate < hi).  Returns the number of pieces longer
 * than 1e-9 pixel_mm written to pix/len (cap must be >= 2n + 2). */
int orc_siddon(const orc_geometry *G, int v, int b, int *pix, double *len, int cap) {
    double S[2], D[2];
    orc_ray_endpoints(G, v, b, S, D);
    const int n = G->n;
    const double h = G->pixel_mm;
    const double x0 = -0.5 * n * h, y0 = -0.5 * n * h;
    const double d[2] = {D[0] - S[0], D[1] - S[1]};
    const double o[2] = {x0, y0};
    const double raylen = sqrt(d[0] * d[0] + d[1] * d[1]);
    const double thr = 1e-9 * h;

    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 2; ++a) {
        if (d[a] != 0.0) {
            double a0 = (o[a] - S[a]) / d[a], a1 = (o[a] + n * h - S[a]) / d[a];
            amin = fmax(amin, fmin(a0, a1));
            amax = fmin(amax, fmax(a0, a1));
        } else if (!(S[a] >= o[a] && S[a] < o[a] + n * h)) {
            return 0;
        }
    }
    if (!(amax > amin)) return 0;

    /* plane parameters in increasing order, the entry index, and the crossings */
    double cr[2][n + 1];
    int ncr[2] = {0, 0}, idx[2], step[2];
    for (int a = 0; a < 2; ++a) {
        if (d[a] == 0.0) {
            idx[a] = (int)floor((S[a] - o[a]) / h);
            step[a] = 0;
            continue;
        }
        step[a] = d[a] > 0.0 ? 1 : -1;
        int passed = 0;
        for (int t = 0; t <= n; ++t) {
            int i = d[a] > 0.0 ? t : n - t;
            double al = (o[a] + i * h - S[a]) / d[a];
            if (al <= amin) ++passed;
            if (al > amin && al < amax) cr[a][ncr[a]++] = al;
        }
        idx[a] = d[a] > 0.0 ? passed - 1 : n - passed;
    }
    int cnt = 0, next[2] = {0, 0};
    double a_prev = amin;
    while (1) {
        double a_next;
        int which;
        if (next[0] < ncr[0] && (next[1] >= ncr[1] || cr[0][next[0]] <= cr[1][next[1]])) {
            which = 0;
            a_next = cr[0][next[0]];
        } else if (next[1] < ncr[1]) {
            which = 1;
            a_next = cr[1][next[1]];
        } else {
            which = -1;
            a_next = amax;
        }
        double l = (a_next - a_prev) * raylen;
        if (l > thr && idx[0] >= 0 && idx[0] < n && idx[1] >= 0 && idx[1] < n && cnt < cap) {
            pix[cnt] = idx[1] * n + idx[0];
            len[cnt] = l;
            ++cnt;
        }
        a_prev = a_next;
        if (which < 0) break;
        idx[which] += step[which];
        ++next[which];
    }
    return cnt;
}

/* g[l][c] = sum_k X_{l,k} f[k][c]  (ray-driven, Eq. fullModel's X) */
void orc_forward(const orc_geometry *G, const double *f, int C, double *g) {
    const int L = G->n_views * G->n_bins;
    const int cap = 2 * G->n + 4;
#pragma omp parallel
    {
        int *pix = (int *)malloc(sizeof(int) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(static)
        for (int l = 0; l < L; ++l) {
            int cnt = orc_siddon(G, l / G->n_bins, l % G->n_bins, pix, len, cap);
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int j = 0; j < cnt; ++j) acc += len[j] * f[(size_t)pix[j] * C + c];
                g[(size_t)l * C + c] = acc;
            }
        }
        free(pix);
        free(len);
    }
}

/* img[k][c] = sum_l X_{l,k} rf[l][c]  (the adjoint X^T, as a serial scatter) */
void orc_backproject(const orc_geometry *G, const double *rf, int C, double *img) {
    const int L = G->n_views * G->n_bins;
    const int cap = 2 * G->n + 4;
    int *pix = (int *)malloc(sizeof(int) * cap);
    double *len = (double *)malloc(sizeof(double) * cap);
    memset(img, 0, sizeof(double) * (size_t)G->n * G->n * C);
    for (int l = 0; l < L; ++l) {
        int cnt = orc_siddon(G, l / G->n_bins, l % G->n_bins, pix, len, cap);
        for (int j = 0; j < cnt; ++j)
            for (int c = 0; c < C; ++c) img[(size_t)pix[j] * C + c] += len[j] * rf[(size_t)l * C + c];
    }
    free(pix);
    free(len);
}

/* ------------------------------------------------------------------ counts model */

/* softexp and its first two derivatives (Sec. 2): exp for x <= 0, x + 1 above.
 * With expm = 1 the standard model's exp (Eq. fullModel) everywhere. */
static double sexp0(double x, int expm) { return (x <= 0.0 || expm) ? exp(x) : x + 1.0; }
static double sexp1(double x, int expm) { return (x <= 0.0 || expm) ? exp(x) : 1.0; }
static double sexp2(double x, int expm) { return (x <= 0.0 || expm) ? exp(x) : 0.0; }

/* Per-ray quantities of Sec. 2 at line integrals g (one ray, detector bin b):
 *   chat_w = N_w sum_i s_wi softexp(-p_i)                        (Eq. finalModel)
 *   r_w    = c_w - chat_w
 *   A_wi   = s_wi softexp'(-p_i) / sum_i' s_wi' softexp(-p_i')    (Eq. aeq)
 *   B_wi   = s_wi softexp''(-p_i) / sum_i' s_wi' softexp(-p_i')
 *   alpha_wm = sum_i A_wi mu_mi       (K_{wl,mk} = alpha_wm X_lk)
 *   grad_m   = sum_w r_w alpha_wm     (the ray's share of Z^T A^T r)
 *   H_mn = sum_w (chat_w + r_w) alpha_wm alpha_wn - sum_i (B^T r)_i mu_mi mu_ni
 *          (the ray's block of the Hessian of Sec. 2, in g)
 * Any output pointer may be NULL. */
void orc_ray_terms(const orc_spectra *sp, int b, const double g[3], const double cw[] /* [W] */,
                   double chat[] /* [W] */, double r[] /* [W] */, double alpha[] /* [W][3] */, double grad[3],
                   double H[9], double A_out[] /* [W][nE] or NULL */, double B_out[] /* [W][nE] or NULL */) {
    const int nE = sp->n_energies, NW = sp->n_windows;
    const double *s = sp->s + (size_t)b * nE * NW;
    double *e0 = (double *)malloc(sizeof(double) * nE);
    double *e1 = (double *)malloc(sizeof(double) * nE);
    double *e2 = (double *)malloc(sizeof(double) * nE);
    for (int i = 0; i < nE; ++i) {
        double p = 0.0;
        for (int m = 0; m < NM; ++m) p += sp->mu[m * nE + i] * g[m];
        e0[i] = sexp0(-p, sp->exp_model);
        e1[i] = sexp1(-p, sp->exp_model);
        e2[i] = sexp2(-p, sp->exp_model);
    }
    double D[NWMAX], ch[NWMAX], rr[NWMAX], al[NWMAX][NM];
    for (int w = 0; w < NW; ++w) {
        D[w] = 0.0;
        for (int i = 0; i < nE; ++i) D[w] += s[i * NW + w] * e0[i];
        ch[w] = sp->N[(size_t)b * NW + w] * D[w];
        rr[w] = (cw ? cw[w] : 0.0) - ch[w];
    }
    for (int w = 0; w < NW; ++w)
        for (int m = 0; m < NM; ++m) {
            double a = 0.0;
            for (int i = 0; i < nE; ++i) a += (s[i * NW + w] * e1[i] / D[w]) * sp->mu[m * nE + i];
            al[w][m] = a;
        }
    if (A_out)
        for (int w = 0; w < NW; ++w)
            for (int i = 0; i < nE; ++i) A_out[w * nE + i] = s[i * NW + w] * e1[i] / D[w];
    if (B_out)
        for (int w = 0; w < NW; ++w)
            for (int i = 0; i < nE; ++i) B_out[w * nE + i] = s[i * NW + w] * e2[i] / D[w];
    if (chat) memcpy(chat, ch, sizeof(double) * NW);
    if (r) memcpy(r, rr, sizeof(double) * NW);
    if (alpha)
        for (int w = 0; w < NW; ++w)
            for (int m = 0; m < NM; ++m) alpha[w * NM + m] = al[w][m];
    if (grad)
        for (int m = 0; m < NM; ++m) {
            double a = 0.0;
            for (int w = 0; w < NW; ++w) a += rr[w] * al[w][m];
            grad[m] = a;
        }
    if (H) {
        for (int m = 0; m < NM; ++m)
            for (int q = 0; q < NM; ++q) {
                double t1 = 0.0, t2 = 0.0;
                for (int w = 0; w < NW; ++w) t1 += (ch[w] + rr[w]) * al[w][m] * al[w][q];
                for (int i = 0; i < nE; ++i) {
                    double btr = 0.0;
                    for (int w = 0; w < NW; ++w) btr += (s[i * NW + w] * e2[i] / D[w]) * rr[w];
                    t2 += btr * sp->mu[m * nE + i] * sp->mu[q * nE + i];
                }
                H[m * NM + q] = t1 - t2;
            }
    }
    free(e0);
    free(e1);
    free(e2);
}

/* Expected counts c^_{w,l}(f) of Eq. (finalModel) for a whole image. */
void orc_counts(const orc_geometry *G, const orc_spectra *sp, const double *f, double *chat) {
    const int L = G->n_views * G->n_bins;
    double *g = (double *)malloc(sizeof(double) * (size_t)L * NM);
    orc_forward(G, f, NM, g);
#pragma omp parallel for schedule(static)
    for (int l = 0; l < L; ++l)
        orc_ray_terms(sp, l % G->n_bins, g + (size_t)l * NM, NULL, chat + (size_t)l * sp->n_windows, NULL, NULL,
                      NULL, NULL, NULL, NULL);
    free(g);
}

/* One term of Eq. (DTPL); c log(c^/c) is taken as 0 when c = 0. */
static double dtpl_term(double chat, double c) {
    return c > 0.0 ? chat - c - c * log(chat / c) : chat;
}

double orc_dtpl(int n, const double *c, const double *chat) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += dtpl_term(chat[j], c[j]);
    return acc;
}

/* D_TPL(c, c^(f)) and its gradient Z^T A^T r per pixel (grad may be NULL). */
double orc_objective(const orc_geometry *G, const orc_spectra *sp, const double *c, const double *f,
                     double *grad /* [P][3] */) {
    const int L = G->n_views * G->n_bins, NW = sp->n_windows;
    double *g = (double *)malloc(sizeof(double) * (size_t)L * NM);
    double *chat = (double *)malloc(sizeof(double) * (size_t)L * NW);
    double *gr = (double *)malloc(sizeof(double) * (size_t)L * NM);
    orc_forward(G, f, NM, g);
#pragma omp parallel for schedule(static)
    for (int l = 0; l < L; ++l)
        orc_ray_terms(sp, l % G->n_bins, g + (size_t)l * NM, c + (size_t)l * NW, chat + (size_t)l * NW,
                      NULL, NULL, gr + (size_t)l * NM, NULL, NULL, NULL);
    double d = orc_dtpl(L * NW, c, chat);
    if (grad) orc_backproject(G, gr, NM, grad);
    free(g);
    free(chat);
    free(gr);
    return d;
}

/* ------------------------------------------------------------------ small dense algebra */

/* Solve the n x n system M x = rhs by Gaussian elimination with partial
 * pivoting (M and rhs are copied).  Returns 0 on success, -1 if singular. */
int orc_solve(int n, const double *M, const double *rhs, double *x) {
    double a[NWMAX * NWMAX], bb[NWMAX];
    if (n > NWMAX) return -1;
    memcpy(a, M, sizeof(double) * n * n);
    memcpy(bb, rhs, sizeof(double) * n);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r2 = col + 1; r2 < n; ++r2)
            if (fabs(a[r2 * n + col]) > fabs(a[piv * n + col])) piv = r2;
        if (a[piv * n + col] == 0.0) return -1;
        if (piv != col) {
            for (int k = 0; k < n; ++k) {
                double t = a[col * n + k];
                a[col * n + k] = a[piv * n + k];
                a[piv * n + k] = t;
            }
            double t = bb[col];
            bb[col] = bb[piv];
            bb[piv] = t;
        }
        for (int r2 = col + 1; r2 < n; ++r2) {
            double f = a[r2 * n + col] / a[col * n + col];
            for (int k = col; k < n; ++k) a[r2 * n + k] -= f * a[col * n + k];
            bb[r2] -= f * bb[col];
        }
    }
    for (int r2 = n - 1; r2 >= 0; --r2) {
        double acc = bb[r2];
        for (int k = r2 + 1; k < n; ++k) acc -= a[r2 * n + k] * x[k];
        x[r2] = acc / a[r2 * n + r2];
    }
    return 0;
}

/* Inverse of a 3 x 3 matrix, column by column through orc_solve. */
static int inv3(const double *M, double *Mi) {
    for (int j = 0; j < 3; ++j) {
        double e[3] = {0, 0, 0}, col[3];
        e[j] = 1.0;
        if (orc_solve(3, M, e, col)) return -1;
        for (int i = 0; i < 3; ++i) Mi[i * 3 + j] = col[i];
    }
    return 0;
}

/* Cyclic Jacobi eigenvalue method for a symmetric 3 x 3 matrix
 * (Golub & Van Loan, Sec. 8.5): each rotation in the (p, q) plane zeroes
 * entry (p, q).  On return H = V diag(lam) V^T, V column-orthonormal. */
int orc_eig_sym3(const double *Hin, double lam[3], double V[9]) {
    double a[9];
    memcpy(a, Hin, sizeof a);
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
        double nrm = 0.0;
        for (int i = 0; i < 9; ++i) nrm += a[i] * a[i];
        if (off == 0.0 || off <= 1e-34 * nrm) break;
        static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
        for (int t = 0; t < 3; ++t) {
            int p = P[t], q = Q[t];
            double apq = a[p * 3 + q];
            if (apq == 0.0) continue;
            double tau = (a[q * 3 + q] - a[p * 3 + p]) / (2.0 * apq);
            double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
            /* J = identity with J_pp = c, J_pq = s, J_qp = -s, J_qq = c;  a <- J^T a J, V <- V J */
            double J[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            J[p * 3 + p] = c;
            J[p * 3 + q] = s;
            J[q * 3 + p] = -s;
            J[q * 3 + q] = c;
            double t1[9], t2[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += a[i * 3 + k] * J[k * 3 + j];
                    t1[i * 3 + j] = acc;
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += J[k * 3 + i] * t1[k * 3 + j];
                    t2[i * 3 + j] = acc;
                }
            memcpy(a, t2, sizeof a);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += V[i * 3 + k] * J[k * 3 + j];
                    t1[i * 3 + j] = acc;
                }
            memcpy(V, t1, sizeof t1);
        }
    }
    for (int i = 0; i < 3; ++i) lam[i] = a[i * 3 + i];
    return 0;
}

/* Negative-curvature removal: H+ = V max(Lambda, 0) V^T. */
void orc_clip_psd3(const double *H, double *Hp) {
    double lam[3], V[9];
    orc_eig_sym3(H, lam, V);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += V[i * 3 + k] * fmax(lam[k], 0.0) * V[j * 3 + k];
            Hp[i * 3 + j] = acc;
        }
}

/* ------------------------------------------------------------------ MOCCA step pieces */

/* Dual step of one ray.  sigma_inv[w] is (Sigma^-1)_{wl}; Hp the curvature in
 * the ray's line integrals g (models 0 and 2); c the measured counts (model 3).
 * With Sigma = diag(1/sigma_inv),
 *   models 0, 2:  G = (alpha^T alpha)^-1 alpha^T,  W = G^T Hp G;
 *   model 1:      W = 0;
 *   model 3:      W = diag(c);
 *   y' = y - Sigma (W + Sigma)^-1 (y - r).
 * A ray with a zero entry of sigma_inv misses the image and keeps y. */
int orc_dual_update(int NW, const double alpha[] /* [W][3] */, const double Hp[9], const double r[],
                    const double sigma_inv[], int model, const double c[], const double y[], double y_out[]) {
    for (int w = 0; w < NW; ++w)
        if (!(sigma_inv[w] > 0.0)) {
            memcpy(y_out, y, sizeof(double) * NW);
            return 0;
        }
    double sig[NWMAX];
    for (int w = 0; w < NW; ++w) sig[w] = 1.0 / sigma_inv[w];
    double W[NWMAX * NWMAX] = {0};
    if (model == 3)
        for (int w = 0; w < NW; ++w) W[w * NW + w] = c[w];
    if (model == 0 || model == 2) {
        double AtA[9], AtAi[9], Gm[NM * NWMAX];
        for (int m = 0; m < NM; ++m)
            for (int q = 0; q < NM; ++q) {
                double acc = 0.0;
                for (int w = 0; w < NW; ++w) acc += alpha[w * NM + m] * alpha[w * NM + q];
                AtA[m * NM + q] = acc;
            }
        if (inv3(AtA, AtAi)) return -1;
        for (int m = 0; m < NM; ++m) /* G[m][w] = sum_q AtAi[m][q] alpha[w][q] */
            for (int w = 0; w < NW; ++w) {
                double acc = 0.0;
                for (int q = 0; q < NM; ++q) acc += AtAi[m * NM + q] * alpha[w * NM + q];
                Gm[m * NW + w] = acc;
            }
        for (int w1 = 0; w1 < NW; ++w1)
            for (int w2 = 0; w2 < NW; ++w2) {
                double acc = 0.0;
                for (int m = 0; m < NM; ++m)
                    for (int q = 0; q < NM; ++q) acc += Gm[m * NW + w1] * Hp[m * NM + q] * Gm[q * NW + w2];
                W[w1 * NW + w2] = acc;
            }
    }
    double M4[NWMAX * NWMAX], d[NWMAX], u[NWMAX];
    for (int i = 0; i < NW * NW; ++i) M4[i] = W[i];
    for (int w = 0; w < NW; ++w) {
        M4[w * NW + w] += sig[w];
        d[w] = y[w] - r[w];
    }
    if (orc_solve(NW, M4, d, u)) return -1;
    for (int w = 0; w < NW; ++w) y_out[w] = y[w] - sig[w] * u[w];
    return 0;
}

/* Primal step of one pixel: x' = argmin_{x in C} 1/2 ||x - t||^2_{Tinv}, with
 * t = x - T v (T = Tinv^-1).  C is R^3 or the box [lo, hi]; the box problem is
 * solved by trying every active set (free / at lo / at hi per material) and
 * keeping the feasible candidate of least objective.  Bounds may be infinite
 * (nonnegativity is lo = 0, hi = +inf); no active set sits at an infinite one.  A pixel with Tinv = 0 is
 * seen by no ray and keeps x.  A tiny multiple of the trace is added to Tinv,
 * which keeps the step condition M >= 0 (Sec. 2). */
int orc_primal_update(const double Tinv_in[9], const double v[3], const double x[3], int use_box,
                      const double lo[3], const double hi[3], double x_out[3]) {
    double tr = Tinv_in[0] + Tinv_in[4] + Tinv_in[8];
    if (!(tr > 0.0)) {
        memcpy(x_out, x, sizeof(double) * 3);
        return 0;
    }
    double Tinv[9];
    memcpy(Tinv, Tinv_in, sizeof Tinv);
    for (int m = 0; m < 3; ++m) Tinv[m * 4] += 1e-12 * tr;
    double delta[3], t[3];
    if (orc_solve(3, Tinv, v, delta)) return -1;
    for (int m = 0; m < 3; ++m) t[m] = x[m] - delta[m];
    if (!use_box) {
        memcpy(x_out, t, sizeof t);
        return 0;
    }
    double best = INFINITY, bestx[3] = {0, 0, 0};
    for (int code = 0; code < 27; ++code) {
        int st[3] = {code % 3, (code / 3) % 3, code / 9}; /* 0 free, 1 lo, 2 hi */
        double xc[3];
        int fr[3], nf = 0, unbounded = 0;
        for (int m = 0; m < 3; ++m) {
            if (st[m] == 1) xc[m] = lo[m];
            else if (st[m] == 2) xc[m] = hi[m];
            else fr[nf++] = m;
            if (st[m] != 0 && isinf(xc[m])) unbounded = 1; /* no point sits at an infinite bound */
        }
        if (unbounded) continue;
        if (nf > 0) {
            /* Tinv_FF (x_F - t_F) = -Tinv_FB (x_B - t_B) */
            double Mf[9], rhs[3], sol[3];
            for (int a = 0; a < nf; ++a) {
                double acc = 0.0;
                for (int m = 0; m < 3; ++m)
                    if (st[m] != 0) acc -= Tinv[fr[a] * 3 + m] * (xc[m] - t[m]);
                rhs[a] = acc;
                for (int c2 = 0; c2 < nf; ++c2) Mf[a * nf + c2] = Tinv[fr[a] * 3 + fr[c2]];
            }
            if (orc_solve(nf, Mf, rhs, sol)) continue;
            int ok = 1;
            for (int a = 0; a < nf; ++a) {
                int m = fr[a];
                double val = t[m] + sol[a];
                double span = hi[m] - lo[m];
                double tol = 1e-12 * (1.0 + (isfinite(span) ? fabs(span) : fabs(val)));
                if (val < lo[m] - tol || val > hi[m] + tol) ok = 0;
                xc[m] = fmin(fmax(val, lo[m]), hi[m]);
            }
            if (!ok) continue;
        }
        double obj = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) obj += 0.5 * (xc[i] - t[i]) * Tinv[i * 3 + j] * (xc[j] - t[j]);
        if (obj < best) {
            best = obj;
            memcpy(bestx, xc, sizeof xc);
        }
    }
    memcpy(x_out, bestx, sizeof bestx);
    return 0;
}

/* ------------------------------------------------------------------ per-iteration quantities */

/* The data-space step matrix of one ray and the per-ray clipped Hessian at the
 * expansion point, with K_{wl,mk} = alpha_wm X_lk (Sec. 2):
 *   block SPC:    (Sigma^-1)_{wl} = lambda sum_k sqrt(sum_m K_{wl,mk}^2)
 *   diagonal SPC: (Sigma^-1)_{wl} = lambda sum_{m,k} |K_{wl,mk}|
 * both written out over the ray's footprint. */
static void ray_sigma_inv(const orc_params *P, int NW, const double alpha[], int cnt, const double *len,
                          double sigma_inv[]) {
    for (int w = 0; w < NW; ++w) {
        double acc = 0.0;
        for (int j = 0; j < cnt; ++j) {
            if (P->spc == 0) {
                double ss = 0.0;
                for (int m = 0; m < NM; ++m) {
                    double K = alpha[w * NM + m] * len[j];
                    ss += K * K;
                }
                acc += sqrt(ss);
            } else {
                for (int m = 0; m < NM; ++m) acc += fabs(alpha[w * NM + m] * len[j]);
            }
        }
        sigma_inv[w] = P->lambda * acc;
    }
}

/* Scatter of one ray into the per-pixel primal quantities of the pixels k in
 * [k_lo, k_hi) (the whole image, or one thread's band of rows):
 *   v_k    += sum_w K_{wl,mk} y'_{wl}                       (K^T y')
 *   block SPC:    Tinv_k[m][m'] += (1/lambda) sum_w K_m K_m' / sqrt(sum_m'' K_m''^2)
 *   diagonal SPC: Tinv_k[m][m]  += (1/lambda) sum_w |K_m|                       */
static void ray_scatter(const orc_params *P, int NW, const double alpha[], const double yp[], int cnt,
                        const int *pix, const double *len, int k_lo, int k_hi, double *v, double *Tinv) {
    for (int j = 0; j < cnt; ++j) {
        if (pix[j] < k_lo || pix[j] >= k_hi) continue;   /* another thread's pixels */
        double *vk = v + (size_t)pix[j] * 3;
        double *Tk = Tinv + (size_t)pix[j] * 9;
        for (int w = 0; w < NW; ++w) {
            double K[3], ss = 0.0;
            for (int m = 0; m < NM; ++m) {
                K[m] = alpha[w * NM + m] * len[j];
                ss += K[m] * K[m];
                vk[m] += K[m] * yp[w];
            }
            if (P->spc == 0) {
                double nk = sqrt(ss);
                if (nk > 0.0)
                    for (int m = 0; m < NM; ++m)
                        for (int q = 0; q < NM; ++q) Tk[m * 3 + q] += K[m] * K[q] / nk / P->lambda;
            } else {
                for (int m = 0; m < NM; ++m) Tk[m * 3 + m] += fabs(K[m]) / P->lambda;
            }
        }
    }
}

/* The scatter of every ray l = 0, 1, ..., L-1 (ray_scatter) into v and Tinv,
 * which it zeroes first.  The rays go in chunks of kScatterChunk: the threads
 * trace a chunk's footprints (Siddon) side by side into fp_cnt / fp_pix /
 * fp_len, then each thread scatters the whole chunk, in ray order, into the
 * pixels of its own band of image rows only.  Every pixel therefore receives
 * the same additions in the same order as a serial scatter over l, whatever
 * the number of threads, and the result is bit-identical to it. */
enum { kScatterChunk = 2048 };

static void scatter_rays(const orc_geometry *G, const orc_params *P, int NW, const double *al, const double *y,
                         double *v, double *Tinv, int *fp_cnt, int *fp_pix, double *fp_len) {
    const int L = G->n_views * G->n_bins, Pn = G->n * G->n, cap = 2 * G->n + 4;
    memset(v, 0, sizeof(double) * (size_t)Pn * 3);
    memset(Tinv, 0, sizeof(double) * (size_t)Pn * 9);
#pragma omp parallel
    {
        int t = 0, nt = 1;
#ifdef _OPENMP
        t = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        const int k_lo = (int)((long long)G->n * t / nt) * G->n;
        const int k_hi = (int)((long long)G->n * (t + 1) / nt) * G->n;
        for (int l0 = 0; l0 < L; l0 += kScatterChunk) {
            const int l1 = l0 + kScatterChunk < L ? l0 + kScatterChunk : L;
#pragma omp for schedule(static)
            for (int l = l0; l < l1; ++l)
                fp_cnt[l - l0] = orc_siddon(G, l / G->n_bins, l % G->n_bins, fp_pix + (size_t)(l - l0) * cap,
                                            fp_len + (size_t)(l - l0) * cap, cap);
            /* (the implicit barrier: the chunk's footprints are complete) */
            for (int l = l0; l < l1; ++l)
                ray_scatter(P, NW, al + (size_t)l * NM * NW, y + (size_t)l * NW, fp_cnt[l - l0],
                            fp_pix + (size_t)(l - l0) * cap, fp_len + (size_t)(l - l0) * cap, k_lo, k_hi, v,
                            Tinv);
#pragma omp barrier
        }
    }
}

/* Step matrices at the expansion point xbar without updating anything:
 * sigma_inv [L][W], Tinv [P][9], alpha [L][W][3] (any may be NULL). */
void orc_step_matrices(const orc_geometry *G, const orc_spectra *sp, const orc_params *P,
                       const double *xbar, double *sigma_inv, double *Tinv, double *alpha_out) {
    const int L = G->n_views * G->n_bins, Pn = G->n * G->n, cap = 2 * G->n + 4, NW = sp->n_windows;
    double *g = (double *)malloc(sizeof(double) * (size_t)L * NM);
    double *al = (double *)malloc(sizeof(double) * (size_t)L * NM * NW);
    double *zeros = (double *)calloc((size_t)L * NW, sizeof(double));
    orc_forward(G, xbar, NM, g);
    int *pix = (int *)malloc(sizeof(int) * cap);
    double *len = (double *)malloc(sizeof(double) * cap);
    double *v = (double *)calloc((size_t)Pn * 3, sizeof(double));
    if (Tinv) memset(Tinv, 0, sizeof(double) * (size_t)Pn * 9);
    for (int l = 0; l < L; ++l) {
        orc_ray_terms(sp, l % G->n_bins, g + (size_t)l * NM, NULL, NULL, NULL, al + (size_t)l * NM * NW,
                      NULL, NULL, NULL, NULL);
        int cnt = orc_siddon(G, l / G->n_bins, l % G->n_bins, pix, len, cap);
        if (sigma_inv) ray_sigma_inv(P, NW, al + (size_t)l * NM * NW, cnt, len, sigma_inv + (size_t)l * NW);
        if (Tinv) ray_scatter(P, NW, al + (size_t)l * NM * NW, zeros, cnt, pix, len, 0, Pn, v, Tinv);
    }
    if (alpha_out) memcpy(alpha_out, al, sizeof(double) * (size_t)L * NM * NW);
    free(g);
    free(al);
    free(zeros);
    free(pix);
    free(len);
    free(v);
}

/* n_iters MOCCA iterations.  State: x = x_n, xbar = 2 x_n - x_{n-1}, y = y_n
 * (all updated in place; start from zeros).  dtpl_hist[it] (if not NULL)
 * receives D_TPL(c, c^(xbar_n)) at the expansion point of iteration it.
 *
 * With P->inner = k > 1 the loop is nested (the inner/outer form the paper
 * mentions and sets aside, Sec. 3): iterations 0, k, 2k, ... of the call are
 * outer ones, exactly the single-loop iteration above, and they keep each
 * ray's local model (alpha, the clipped Hessian, r, Sigma^-1 and g0 = X xbar);
 * the k - 1 iterations after each take one primal-dual step on that fixed
 * convex model: with g = X xbar, the dual prox acts on
 *   u = y + Sigma alpha (g - g0)
 * (the prox argument y + Sigma K xbar, measured from the expansion point
 * K f0 = alpha g0), y' = u - Sigma (W + Sigma)^-1 (u - r), and K = alpha X keeps
 * the stored alpha in the back-projection and the step matrix T.  An outer
 * iteration has g = g0, so u = y and k = 1 is the single-loop method.
 * Returns 0, or -1 if a small system was singular. */
int orc_mocca(const orc_geometry *G, const orc_spectra *sp, const orc_params *P, const double *c,
              double *x, double *xbar, double *y, int n_iters, double *dtpl_hist) {
    const int L = G->n_views * G->n_bins, Pn = G->n * G->n, cap = 2 * G->n + 4, NW = sp->n_windows;
    double *g = (double *)malloc(sizeof(double) * (size_t)L * NM);
    double *al = (double *)malloc(sizeof(double) * (size_t)L * NM * NW);
    double *dt = (double *)malloc(sizeof(double) * (size_t)L);
    double *v = (double *)malloc(sizeof(double) * (size_t)Pn * 3);
    double *Tinv = (double *)malloc(sizeof(double) * (size_t)Pn * 9);
    int *fp_cnt = (int *)malloc(sizeof(int) * kScatterChunk);
    int *fp_pix = (int *)malloc(sizeof(int) * (size_t)kScatterChunk * cap);
    double *fp_len = (double *)malloc(sizeof(double) * (size_t)kScatterChunk * cap);
    const int inner = P->inner > 1 ? P->inner : 1;
    double *mHp = NULL, *mr = NULL, *msinv = NULL, *mg0 = NULL;   /* the stored local models */
    if (inner > 1) {
        mHp = (double *)malloc(sizeof(double) * (size_t)L * 9);
        mr = (double *)malloc(sizeof(double) * (size_t)L * NW);
        msinv = (double *)malloc(sizeof(double) * (size_t)L * NW);
        mg0 = (double *)malloc(sizeof(double) * (size_t)L * NM);
    }
    int status = 0;
    for (int it = 0; it < n_iters && status == 0; ++it) {
        const int outer = it % inner == 0;
        /* forward projection at the expansion point f0 = xbar */
        orc_forward(G, xbar, NM, g);
        /* per-ray model, local quadratic and dual step */
#pragma omp parallel
        {
            int *pp = (int *)malloc(sizeof(int) * cap);
            double *ll = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(static)
            for (int l = 0; l < L; ++l) {
                const int b = l % G->n_bins;
                double chat[NWMAX], r[NWMAX], H[9], Hp[9], sinv[NWMAX], yn[NWMAX], u[NWMAX];
                const double *cl = c + (size_t)l * NW;
                double *all = al + (size_t)l * NM * NW;
                if (outer) {
                    orc_ray_terms(sp, b, g + (size_t)l * NM, cl, chat, r, all, NULL, H, NULL, NULL);
                    if (P->model == 0) {
                        orc_clip_psd3(H, Hp);
                    } else if (P->model == 2) {   /* sum_w c_w alpha_w alpha_w^T */
                        for (int m = 0; m < NM; ++m)
                            for (int q = 0; q < NM; ++q) {
                                double acc = 0.0;
                                for (int w = 0; w < NW; ++w) acc += cl[w] * all[w * NM + m] * all[w * NM + q];
                                Hp[m * NM + q] = acc;
                            }
                    } else {
                        memset(Hp, 0, sizeof Hp);
                    }
                    int cnt = orc_siddon(G, l / G->n_bins, b, pp, ll, cap);
                    ray_sigma_inv(P, NW, all, cnt, ll, sinv);
                    memcpy(u, y + (size_t)l * NW, sizeof(double) * NW);
                    if (inner > 1) {
                        memcpy(mHp + (size_t)l * 9, Hp, sizeof Hp);
                        memcpy(mr + (size_t)l * NW, r, sizeof(double) * NW);
                        memcpy(msinv + (size_t)l * NW, sinv, sizeof(double) * NW);
                        memcpy(mg0 + (size_t)l * NM, g + (size_t)l * NM, sizeof(double) * NM);
                    }
                } else {
                    double dummy[NM * NWMAX];   /* D_TPL at xbar as a diagnostic; the model stays fixed */
                    orc_ray_terms(sp, b, g + (size_t)l * NM, cl, chat, NULL, dummy, NULL, NULL, NULL, NULL);
                    memcpy(Hp, mHp + (size_t)l * 9, sizeof Hp);
                    memcpy(r, mr + (size_t)l * NW, sizeof(double) * NW);
                    memcpy(sinv, msinv + (size_t)l * NW, sizeof(double) * NW);
                    const double *gl = g + (size_t)l * NM, *g0 = mg0 + (size_t)l * NM;
                    for (int w = 0; w < NW; ++w) {
                        double kz = 0.0;   /* (K (xbar - f0))_w = alpha_w . (g - g0) */
                        for (int m = 0; m < NM; ++m) kz += all[w * NM + m] * (gl[m] - g0[m]);
                        u[w] = y[(size_t)l * NW + w] + (sinv[w] > 0.0 ? kz / sinv[w] : 0.0);
                    }
                }
                double d = 0.0;
                for (int w = 0; w < NW; ++w) d += dtpl_term(chat[w], cl[w]);
                dt[l] = d;
                if (orc_dual_update(NW, all, Hp, r, sinv, P->model, cl, u, yn)) {
#pragma omp atomic write
                    status = -1;
                }
                memcpy(y + (size_t)l * NW, yn, sizeof(double) * NW);
            }
            free(pp);
            free(ll);
        }
        if (dtpl_hist) {
            double acc = 0.0;
            for (int l = 0; l < L; ++l) acc += dt[l];
            dtpl_hist[it] = acc;
        }
        /* back-projection of K^T y' and of the block step matrix */
        scatter_rays(G, P, NW, al, y, v, Tinv, fp_cnt, fp_pix, fp_len);
        /* per-pixel primal step and extrapolation */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < Pn; ++k) {
            double xn[3];
            if (orc_primal_update(Tinv + (size_t)k * 9, v + (size_t)k * 3, x + (size_t)k * 3, P->use_box,
                                  P->lo, P->hi, xn)) {
#pragma omp atomic write
                status = -1;
            }
            for (int m = 0; m < 3; ++m) {
                xbar[(size_t)k * 3 + m] = 2.0 * xn[m] - x[(size_t)k * 3 + m];
                x[(size_t)k * 3 + m] = xn[m];
            }
        }
    }
    free(g);
    free(al);
    free(dt);
    free(v);
    free(Tinv);
    free(fp_cnt);
    free(fp_pix);
    free(fp_len);
    free(mHp);
    free(mr);
    free(msinv);
    free(mg0);
    return status;
}
