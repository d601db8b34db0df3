/*
 * FP64 CPU oracle: the discretised objective of Sec. II-D of arXiv 1807.00467,
 * its exact gradient, the Gauss-Newton matrix, a fixed GN-PCG schedule with
 * Armijo backtracking, and the multilevel (pyramid) driver.
 *
 * TEST INFRASTRUCTURE ONLY (see ngf_oracle.h).  Written for a reader who
 * checks it against the paper: every loop runs over voxels, grid nodes, grid
 * cells or keypoints exactly as the sums in the equations do, with no tiling,
 * fusion or reordering.  OpenMP only splits independent loop iterations.
 *
 * Discretisation readings (the paper is silent on these):
 *   - D, Eq. (1): central differences of R and of the warped template
 *     Tw(x) = T(y(x)) on the fixed grid; D = hbar * sum over interior voxels
 *     (1 .. n-2 on every axis) of 1 - r^2, with
 *     r = <f,g>_eta / (|f|_eta |g|_eta), <f,g>_eta = eta^2 + f.g.
 *   - T(y) is trilinear in voxel-index coordinates s = y/h - 1/2.  Along an
 *     axis where s lies outside [0, n-1] the sample is clamped to the border
 *     and its derivative along that axis is 0.  At s = n-1 exactly the cell
 *     n-2 with fraction 1 is used.
 *   - The trilinear derivative jumps at integer s.  Which cell a voxel uses
 *     is an integer decision taken from floating point, so it is taken in the
 *     GPU kernel's precision (FP32, with the fixed operation order of
 *     decide_cells() below); the interpolation itself is FP64.
 *   - The NGF Gauss-Newton matrix is 2 hbar J^T J with J = dr/du.
 *   - R, Eq. (5), with y_hat = identity: nodal 3-point second differences
 *     along each axis at nodes interior to that axis (zero at that axis'
 *     boundary nodes), L = sum of the three; R = ghat/2 sum_nodes |L u|^2,
 *     ghat = g1 g2 g3 the cell volume.
 *   - V-hat, Eq. (9): per grid cell, e1_a (a = 4 x-edges), e2_b, e3_c are the
 *     edge difference quotients of y; d_abc = det(e1_a, e2_b, e3_c) are the
 *     64 values of Eq. (8) (multilinearity of det); C = ghat; no 1/64.
 *   - K, Eq. (10): trilinear evaluation of y at the keypoint positions.
 */
#include "ngf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(n, i1, i2, i3) ((((long)(i3)) * (n)[1] + (i2)) * (long)(n)[0] + (i1))

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static long nvox(const orc_problem *p) { return (long)p->n[0] * p->n[1] * p->n[2]; }
static long nnod(const orc_problem *p) { return (long)p->m[0] * p->m[1] * p->m[2]; }
static int ratio(const orc_problem *p, int a) { return p->n[a] / (p->m[a] - 1); }
static double gsp(const orc_problem *p, int a) { return p->n[a] * p->h[a] / (p->m[a] - 1); }
static double hbar(const orc_problem *p) { return p->h[0] * p->h[1] * p->h[2]; }
static double ghat(const orc_problem *p) { return gsp(p, 0) * gsp(p, 1) * gsp(p, 2); }

int orc_check(const orc_problem *p) {
    for (int a = 0; a < 3; ++a) {
        if (p->n[a] < 4 || p->m[a] < 2 || p->h[a] <= 0) return -1;
        if (p->n[a] % (p->m[a] - 1) != 0) return -1;
        int r = ratio(p, a);
        if (r & (r - 1)) return -1;          /* power of two */
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Trilinear prolongation P (first-order B-spline on the node grid).   */
/* Voxel i on an axis with ratio rho lies at grid coordinate          */
/* t = (i + 1/2)/rho; it uses nodes c = floor(t), c + 1 with weights   */
/* 1 - f, f where f = t - c.                                           */
/* ------------------------------------------------------------------ */
static void axis_weight(int i, int rho, int *c, double *f) {
    double t = (i + 0.5) / rho;
    int ci = (int)floor(t);
    *c = ci;
    *f = t - ci;
}

static void prolong_voxel(const orc_problem *p, const double *u, int i1, int i2, int i3, double d[3]) {
    int c[3];
    double f[3];
    int ii[3] = {i1, i2, i3};
    for (int a = 0; a < 3; ++a) axis_weight(ii[a], ratio(p, a), &c[a], &f[a]);
    long M = nnod(p);
    for (int comp = 0; comp < 3; ++comp) {
        double s = 0.0;
        for (int o3 = 0; o3 < 2; ++o3)
            for (int o2 = 0; o2 < 2; ++o2)
                for (int o1 = 0; o1 < 2; ++o1) {
                    double w = (o1 ? f[0] : 1 - f[0]) * (o2 ? f[1] : 1 - f[1]) * (o3 ? f[2] : 1 - f[2]);
                    s += w * u[comp * M + IDX(p->m, c[0] + o1, c[1] + o2, c[2] + o3)];
                }
        d[comp] = s;
    }
}

void orc_prolong(const orc_problem *p, const double *u, double *disp) {
    long N = nvox(p);
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < p->n[2]; ++i3)
        for (int i2 = 0; i2 < p->n[1]; ++i2)
            for (int i1 = 0; i1 < p->n[0]; ++i1) {
                double d[3];
                prolong_voxel(p, u, i1, i2, i3, d);
                long v = IDX(p->n, i1, i2, i3);
                disp[v] = d[0];
                disp[N + v] = d[1];
                disp[2 * N + v] = d[2];
            }
}

/* The integer cell decision in FP32, fixed order: interpolate along x, then
 * y, then z, each step fmaf(w1, b, w0 * a) with one rounding per operation;
 * q = Pu * (float)(1/h); the sample cell is i + floor(q). */
static float lerp32(float a, float b, float w0, float w1) {
    float t = w0 * a;
    return fmaf(w1, b, t);
}

static void decide_cells(const orc_problem *p, const double *u, int i1, int i2, int i3,
                         int k[3], float fr[3]) {
    int c[3];
    double f[3];
    int ii[3] = {i1, i2, i3};
    for (int a = 0; a < 3; ++a) axis_weight(ii[a], ratio(p, a), &c[a], &f[a]);
    long M = nnod(p);
    float w1[3], w0[3];
    for (int a = 0; a < 3; ++a) { w1[a] = (float)f[a]; w0[a] = (float)(1.0 - f[a]); }
    for (int comp = 0; comp < 3; ++comp) {
        float ux[2][2];
        for (int o3 = 0; o3 < 2; ++o3)
            for (int o2 = 0; o2 < 2; ++o2) {
                float a0 = (float)u[comp * M + IDX(p->m, c[0], c[1] + o2, c[2] + o3)];
                float a1 = (float)u[comp * M + IDX(p->m, c[0] + 1, c[1] + o2, c[2] + o3)];
                ux[o3][o2] = lerp32(a0, a1, w0[0], w1[0]);
            }
        float uxy0 = lerp32(ux[0][0], ux[0][1], w0[1], w1[1]);
        float uxy1 = lerp32(ux[1][0], ux[1][1], w0[1], w1[1]);
        float pu = lerp32(uxy0, uxy1, w0[2], w1[2]);
        float invh = (float)(1.0 / p->h[comp]);
        float q = pu * invh;
        float fl = floorf(q);
        k[comp] = ii[comp] + (int)fl;
        fr[comp] = q - fl;
    }
}

void orc_cells(const orc_problem *p, const double *u, int *k) {
    long N = nvox(p);
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < p->n[2]; ++i3)
        for (int i2 = 0; i2 < p->n[1]; ++i2)
            for (int i1 = 0; i1 < p->n[0]; ++i1) {
                int kk[3];
                float fr[3];
                decide_cells(p, u, i1, i2, i3, kk, fr);
                long v = IDX(p->n, i1, i2, i3);
                for (int a = 0; a < 3; ++a) k[a * N + v] = kk[a];
            }
}

/* Per-axis sample placement: cell index, FP64 fraction, inside flag. */
static void place_axis(int n, int k, float fr32, double s, int *cell, double *frac, int *inside) {
    if (k < 0) {                         /* below the domain: clamp to 0 */
        *cell = 0; *frac = 0.0; *inside = 0;
    } else if (k > n - 1 || (k == n - 1 && fr32 > 0.0f)) {   /* above: clamp */
        *cell = n - 2; *frac = 1.0; *inside = 0;
    } else if (k == n - 1) {             /* exactly on the last voxel */
        *cell = n - 2; *frac = s - (n - 2); *inside = 1;
    } else {
        *cell = k; *frac = s - k; *inside = 1;
    }
}

void orc_warp(const orc_problem *p, const double *u, double *Tw, double *dT) {
    long N = nvox(p);
    const int *n = p->n;
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < n[2]; ++i3)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i1 = 0; i1 < n[0]; ++i1) {
                int ii[3] = {i1, i2, i3};
                double d[3];
                prolong_voxel(p, u, i1, i2, i3, d);
                int k[3];
                float fr[3];
                decide_cells(p, u, i1, i2, i3, k, fr);
                int cell[3], in[3];
                double w[3];
                for (int a = 0; a < 3; ++a) {
                    double s = ii[a] + d[a] / p->h[a];   /* y/h - 1/2 with y = (i+1/2)h + d */
                    place_axis(n[a], k[a], fr[a], s, &cell[a], &w[a], &in[a]);
                }
                double val = 0.0, der[3] = {0.0, 0.0, 0.0};
                for (int o3 = 0; o3 < 2; ++o3)
                    for (int o2 = 0; o2 < 2; ++o2)
                        for (int o1 = 0; o1 < 2; ++o1) {
                            double t = p->T[IDX(n, cell[0] + o1, cell[1] + o2, cell[2] + o3)];
                            double wx = o1 ? w[0] : 1 - w[0];
                            double wy = o2 ? w[1] : 1 - w[1];
                            double wz = o3 ? w[2] : 1 - w[2];
                            val += wx * wy * wz * t;
                            der[0] += (o1 ? 1.0 : -1.0) * wy * wz * t;
                            der[1] += wx * (o2 ? 1.0 : -1.0) * wz * t;
                            der[2] += wx * wy * (o3 ? 1.0 : -1.0) * t;
                        }
                long v = IDX(n, i1, i2, i3);
                Tw[v] = val;
                for (int a = 0; a < 3; ++a) dT[a * N + v] = in[a] ? der[a] / p->h[a] : 0.0;
            }
}

/* ------------------------------------------------------------------ */
/* NGF distance, Eq. (1).                                              */
/* ------------------------------------------------------------------ */
static int interior(const int *n, int i1, int i2, int i3) {
    return i1 >= 1 && i1 <= n[0] - 2 && i2 >= 1 && i2 <= n[1] - 2 && i3 >= 1 && i3 <= n[2] - 2;
}

double orc_ngf_distance(const orc_problem *p, const double *Tw, double *r, double *a) {
    long N = nvox(p);
    const int *n = p->n;
    double eta2 = p->eta * p->eta, hb = hbar(p);
    /* the sum over voxels in a fixed order: each x row in order, then the rows */
    double *row = calloc((size_t)n[1] * n[2], sizeof(double));
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < n[2]; ++i3)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i1 = 0; i1 < n[0]; ++i1) {
                double *D = &row[(long)i3 * n[1] + i2];
                long v = IDX(n, i1, i2, i3);
                if (!interior(n, i1, i2, i3)) {
                    if (r) r[v] = 0.0;
                    if (a) a[v] = a[N + v] = a[2 * N + v] = 0.0;
                    continue;
                }
                long st[3] = {1, n[0], (long)n[0] * n[1]};
                double f[3], g[3];
                for (int k = 0; k < 3; ++k) {
                    f[k] = ((double)p->R[v + st[k]] - (double)p->R[v - st[k]]) / (2.0 * p->h[k]);
                    g[k] = (Tw[v + st[k]] - Tw[v - st[k]]) / (2.0 * p->h[k]);
                }
                double fg = eta2 + f[0] * g[0] + f[1] * g[1] + f[2] * g[2];
                double ff = eta2 + f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
                double gg = eta2 + g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
                /* Eq. (1) as printed: 1 - <f,g>^2 / (|f|^2 |g|^2) */
                *D += hb * (1.0 - (fg * fg) / (ff * gg));
                double nf = sqrt(ff), ng = sqrt(gg);
                double rv = fg / (nf * ng);
                if (r) r[v] = rv;
                if (a)   /* dr/dg = f/(|f| |g|) - r g/|g|^2 */
                    for (int k = 0; k < 3; ++k) a[k * N + v] = f[k] / (nf * ng) - rv * g[k] / gg;
            }
    double D = 0.0;
    for (long i = 0; i < (long)n[1] * n[2]; ++i) D += row[i];
    free(row);
    return D;
}

/* Adjoint of the central difference followed by the chain rule through the
 * warp: given per-voxel c (3 comps, zero off the interior), returns
 * z_w = dT_w * sum_a (c_{w-e_a,a} - c_{w+e_a,a}) / (2 h_a). */
static void adjoint_to_voxels(const orc_problem *p, const double *c, const double *dT, double *z) {
    long N = nvox(p);
    const int *n = p->n;
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < n[2]; ++i3)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i1 = 0; i1 < n[0]; ++i1) {
                long v = IDX(n, i1, i2, i3);
                int ii[3] = {i1, i2, i3};
                long st[3] = {1, n[0], (long)n[0] * n[1]};
                double b = 0.0;
                for (int k = 0; k < 3; ++k) {
                    if (ii[k] - 1 >= 0) b += c[k * N + v - st[k]] / (2.0 * p->h[k]);
                    if (ii[k] + 1 <= n[k] - 1) b -= c[k * N + v + st[k]] / (2.0 * p->h[k]);
                }
                for (int k = 0; k < 3; ++k) z[k * N + v] = b * dT[k * N + v];
            }
}

/* P^T: out(node) = sum over voxels in the node's support of weight * z. */
static void prolong_transpose(const orc_problem *p, const double *z, double *out) {
    long N = nvox(p), M = nnod(p);
    const int *n = p->n, *m = p->m;
#pragma omp parallel for collapse(2)
    for (int k3 = 0; k3 < m[2]; ++k3)
        for (int k2 = 0; k2 < m[1]; ++k2)
            for (int k1 = 0; k1 < m[0]; ++k1) {
                int kk[3] = {k1, k2, k3};
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    int rho = ratio(p, a);
                    lo[a] = (kk[a] - 1) * rho; if (lo[a] < 0) lo[a] = 0;
                    hi[a] = (kk[a] + 1) * rho - 1; if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
                }
                double acc[3] = {0, 0, 0};
                for (int i3 = lo[2]; i3 <= hi[2]; ++i3)
                    for (int i2 = lo[1]; i2 <= hi[1]; ++i2)
                        for (int i1 = lo[0]; i1 <= hi[0]; ++i1) {
                            int ii[3] = {i1, i2, i3};
                            double w = 1.0;
                            for (int a = 0; a < 3; ++a) {
                                int c; double f;
                                axis_weight(ii[a], ratio(p, a), &c, &f);
                                if (c == kk[a]) w *= 1.0 - f;
                                else if (c == kk[a] - 1) w *= f;
                                else w = 0.0;
                            }
                            if (w == 0.0) continue;
                            long v = IDX(n, i1, i2, i3);
                            for (int comp = 0; comp < 3; ++comp) acc[comp] += w * z[comp * N + v];
                        }
                long node = IDX(m, k1, k2, k3);
                for (int comp = 0; comp < 3; ++comp) out[comp * M + node] = acc[comp];
            }
}

int orc_ngf_gradient(const orc_problem *p, const double *u, double *Dout, double *grad) {
    long N = nvox(p);
    double *Tw = malloc(sizeof(double) * N), *dT = malloc(sizeof(double) * 3 * N);
    double *r = malloc(sizeof(double) * N), *a = malloc(sizeof(double) * 3 * N);
    if (!Tw || !dT || !r || !a) { free(Tw); free(dT); free(r); free(a); return -3; }
    orc_warp(p, u, Tw, dT);
    double D = orc_ngf_distance(p, Tw, r, a);
    if (Dout) *Dout = D;
    if (grad) {
        /* dD/dg_v = hbar * d(1 - r^2)/dg = -2 hbar r a  (interior voxels) */
        double hb = hbar(p);
        double *c = a;   /* reuse storage */
        for (long v = 0; v < N; ++v)
            for (int k = 0; k < 3; ++k) c[k * N + v] = -2.0 * hb * r[v] * a[k * N + v];
        double *z = malloc(sizeof(double) * 3 * N);
        if (!z) { free(Tw); free(dT); free(r); free(a); return -3; }
        adjoint_to_voxels(p, c, dT, z);
        prolong_transpose(p, z, grad);
        free(z);
    }
    free(Tw); free(dT); free(r); free(a);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Curvature regulariser, Eq. (5), y_hat = identity.                   */
/* ------------------------------------------------------------------ */
static int node_interior_axis(const int *m, const int kk[3], int a) {
    return kk[a] >= 1 && kk[a] <= m[a] - 2;
}

static void apply_L(const orc_problem *p, const double *u, double *Lu) {
    long M = nnod(p);
    const int *m = p->m;
    double g2[3];
    for (int a = 0; a < 3; ++a) g2[a] = gsp(p, a) * gsp(p, a);
    long st[3] = {1, m[0], (long)m[0] * m[1]};
#pragma omp parallel for collapse(2)
    for (int k3 = 0; k3 < m[2]; ++k3)
        for (int k2 = 0; k2 < m[1]; ++k2)
            for (int k1 = 0; k1 < m[0]; ++k1) {
                int kk[3] = {k1, k2, k3};
                long node = IDX(m, k1, k2, k3);
                for (int comp = 0; comp < 3; ++comp) {
                    const double *uc = u + comp * M;
                    double s = 0.0;
                    for (int a = 0; a < 3; ++a)
                        if (node_interior_axis(m, kk, a))
                            s += (uc[node + st[a]] - 2.0 * uc[node] + uc[node - st[a]]) / g2[a];
                    Lu[comp * M + node] = s;
                }
            }
}

static void apply_LT(const orc_problem *p, const double *w, double *out) {
    long M = nnod(p);
    const int *m = p->m;
    double g2[3];
    for (int a = 0; a < 3; ++a) g2[a] = gsp(p, a) * gsp(p, a);
    long st[3] = {1, m[0], (long)m[0] * m[1]};
#pragma omp parallel for collapse(2)
    for (int k3 = 0; k3 < m[2]; ++k3)
        for (int k2 = 0; k2 < m[1]; ++k2)
            for (int k1 = 0; k1 < m[0]; ++k1) {
                int kk[3] = {k1, k2, k3};
                long node = IDX(m, k1, k2, k3);
                for (int comp = 0; comp < 3; ++comp) {
                    const double *wc = w + comp * M;
                    double s = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        /* rows j of L that reference node k along axis a */
                        if (node_interior_axis(m, kk, a)) s += -2.0 * wc[node] / g2[a];
                        int km[3] = {kk[0], kk[1], kk[2]}, kp[3] = {kk[0], kk[1], kk[2]};
                        km[a] -= 1; kp[a] += 1;
                        if (km[a] >= 0 && node_interior_axis(m, km, a)) s += wc[node - st[a]] / g2[a];
                        if (kp[a] <= m[a] - 1 && node_interior_axis(m, kp, a)) s += wc[node + st[a]] / g2[a];
                    }
                    out[comp * M + node] = s;
                }
            }
}

void orc_curvature(const orc_problem *p, const double *u, const double *v, double *energy, double *out) {
    long M = nnod(p);
    double G = ghat(p);
    double *Lu = malloc(sizeof(double) * 3 * M);
    apply_L(p, u, Lu);
    if (energy) {
        double e = 0.0;
        for (long i = 0; i < 3 * M; ++i) e += Lu[i] * Lu[i];
        *energy = 0.5 * G * e;
    }
    if (out) {
        if (v) apply_L(p, v, Lu);
        apply_LT(p, Lu, out);
        for (long i = 0; i < 3 * M; ++i) out[i] *= G;
    }
    free(Lu);
}

/* ------------------------------------------------------------------ */
/* Volume change control, Eqs. (7)-(9).                                */
/* ------------------------------------------------------------------ */
static double psi(double t) { return (t - 1.0) * (t - 1.0) / t; }
static double dpsi(double t) { return 1.0 - 1.0 / (t * t); }
static double d2psi(double t) { return 2.0 / (t * t * t); }

static void cross(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Node offset of the two ends of edge number e (0..3) along axis a. */
static void edge_ends(int a, int e, int o0[3], int o1[3]) {
    int p = e & 1, q = (e >> 1) & 1;       /* offsets along the two other axes */
    int b = (a + 1) % 3, c = (a + 2) % 3;
    int lo = b < c ? b : c, hi = b < c ? c : b;
    o0[a] = 0; o1[a] = 1;
    o0[lo] = o1[lo] = p;
    o0[hi] = o1[hi] = q;
}

/* Edge vectors e_a[e] = unit_a + (u(end) - u(start)) / g_a of one cell. */
static void cell_edges(const orc_problem *p, const double *u, int c1, int c2, int c3, double E[3][4][3]) {
    long M = nnod(p);
    for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 4; ++e) {
            int o0[3], o1[3];
            edge_ends(a, e, o0, o1);
            long n0 = IDX(p->m, c1 + o0[0], c2 + o0[1], c3 + o0[2]);
            long n1 = IDX(p->m, c1 + o1[0], c2 + o1[1], c3 + o1[2]);
            for (int comp = 0; comp < 3; ++comp)
                E[a][e][comp] = (comp == a ? 1.0 : 0.0) + (u[comp * M + n1] - u[comp * M + n0]) / gsp(p, a);
        }
}

/* The 64 values d_abc of one cell, index a + 4 b + 16 c (Eq. (8)). */
void orc_vcc_cell_dets(const orc_problem *p, const double *u, const int *cell, double *d64) {
    double E[3][4][3];
    cell_edges(p, u, cell[0], cell[1], cell[2], E);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) {
                double x23[3];
                cross(E[1][b], E[2][c], x23);
                d64[a + 4 * b + 16 * c] = dot3(E[0][a], x23);
            }
}

/* Per-cell contributions to the 8 corner nodes, scattered through a
 * per-cell buffer and then gathered per node. */
int orc_vcc(const orc_problem *p, const double *u, const double *v, double *energy, double *out,
            double *dminmax) {
    const int *m = p->m;
    long M = nnod(p);
    int nc[3] = {m[0] - 1, m[1] - 1, m[2] - 1};
    long NC = (long)nc[0] * nc[1] * nc[2];
    double G = ghat(p);
    double *cellout = out ? calloc((size_t)NC * 24, sizeof(double)) : NULL;
    double dmin = INFINITY, dmax = -INFINITY;
    int fold = 0;
    /* the energy summed in a fixed order: each x row of cells in order, then the rows */
    double *erow = calloc((size_t)nc[1] * nc[2], sizeof(double));
#pragma omp parallel for collapse(2) reduction(+ : fold) reduction(min : dmin) reduction(max : dmax)
    for (int c3 = 0; c3 < nc[2]; ++c3)
        for (int c2 = 0; c2 < nc[1]; ++c2)
            for (int c1 = 0; c1 < nc[0]; ++c1) {
                double *e = &erow[(long)c3 * nc[1] + c2];
                double E[3][4][3], V[3][4][3];
                cell_edges(p, u, c1, c2, c3, E);
                if (v) {   /* edge differences of v (no unit term) */
                    cell_edges(p, v, c1, c2, c3, V);
                    for (int a = 0; a < 3; ++a)
                        for (int k = 0; k < 4; ++k) V[a][k][a] -= 1.0;
                }
                double GE[3][4][3];
                memset(GE, 0, sizeof GE);
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b)
                        for (int c = 0; c < 4; ++c) {
                            double x23[3], x31[3], x12[3];
                            cross(E[1][b], E[2][c], x23);   /* d d / d e1 */
                            cross(E[2][c], E[0][a], x31);   /* d d / d e2 */
                            cross(E[0][a], E[1][b], x12);   /* d d / d e3 */
                            double d = dot3(E[0][a], x23);
                            if (d < dmin) dmin = d;
                            if (d > dmax) dmax = d;
                            if (d <= 0.0) { fold += 1; continue; }
                            *e += G * psi(d);
                            double wgt;
                            if (!v) wgt = G * dpsi(d);
                            else wgt = G * d2psi(d) * (dot3(x23, V[0][a]) + dot3(x31, V[1][b]) + dot3(x12, V[2][c]));
                            for (int k = 0; k < 3; ++k) {
                                GE[0][a][k] += wgt * x23[k];
                                GE[1][b][k] += wgt * x31[k];
                                GE[2][c][k] += wgt * x12[k];
                            }
                        }
                if (cellout) {
                    double *co = cellout + 24 * (long)IDX(nc, c1, c2, c3);
                    for (int a = 0; a < 3; ++a)
                        for (int k = 0; k < 4; ++k) {
                            int o0[3], o1[3];
                            edge_ends(a, k, o0, o1);
                            int s0 = o0[0] + 2 * o0[1] + 4 * o0[2], s1 = o1[0] + 2 * o1[1] + 4 * o1[2];
                            for (int comp = 0; comp < 3; ++comp) {
                                co[3 * s1 + comp] += GE[a][k][comp] / gsp(p, a);
                                co[3 * s0 + comp] -= GE[a][k][comp] / gsp(p, a);
                            }
                        }
                }
            }
    double e = 0.0;
    for (long i = 0; i < (long)nc[1] * nc[2]; ++i) e += erow[i];
    free(erow);
    if (dminmax) { dminmax[0] = dmin; dminmax[1] = dmax; }
    if (energy) *energy = fold ? INFINITY : e;
    if (out) {
#pragma omp parallel for collapse(2)
        for (int k3 = 0; k3 < m[2]; ++k3)
            for (int k2 = 0; k2 < m[1]; ++k2)
                for (int k1 = 0; k1 < m[0]; ++k1) {
                    double acc[3] = {0, 0, 0};
                    for (int o3 = 0; o3 < 2; ++o3)
                        for (int o2 = 0; o2 < 2; ++o2)
                            for (int o1 = 0; o1 < 2; ++o1) {
                                int c1 = k1 - o1, c2 = k2 - o2, c3 = k3 - o3;
                                if (c1 < 0 || c2 < 0 || c3 < 0 || c1 >= nc[0] || c2 >= nc[1] || c3 >= nc[2]) continue;
                                const double *co = cellout + 24 * (long)IDX(nc, c1, c2, c3);
                                int s = o1 + 2 * o2 + 4 * o3;
                                for (int comp = 0; comp < 3; ++comp) acc[comp] += co[3 * s + comp];
                            }
                    long node = IDX(m, k1, k2, k3);
                    for (int comp = 0; comp < 3; ++comp) out[comp * M + node] = acc[comp];
                }
        free(cellout);
    }
    return fold ? 1 : 0;
}

/* Diagonal of the VCC Gauss-Newton matrix: ghat sum_cells sum_abc
 * psi''(d) (d d_abc / d u_{k,c})^2, gathered per node. */
void orc_vcc_diag(const orc_problem *p, const double *u, double *out) {
    const int *m = p->m;
    long M = nnod(p);
    int nc[3] = {m[0] - 1, m[1] - 1, m[2] - 1};
    long NC = (long)nc[0] * nc[1] * nc[2];
    double G = ghat(p);
    double *cellout = calloc((size_t)NC * 24, sizeof(double));
#pragma omp parallel for collapse(2)
    for (int c3 = 0; c3 < nc[2]; ++c3)
        for (int c2 = 0; c2 < nc[1]; ++c2)
            for (int c1 = 0; c1 < nc[0]; ++c1) {
                double E[3][4][3];
                cell_edges(p, u, c1, c2, c3, E);
                double *co = cellout + 24 * (long)IDX(nc, c1, c2, c3);
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b)
                        for (int c = 0; c < 4; ++c) {
                            double x23[3], x31[3], x12[3];
                            cross(E[1][b], E[2][c], x23);
                            cross(E[2][c], E[0][a], x31);
                            cross(E[0][a], E[1][b], x12);
                            double d = dot3(E[0][a], x23);
                            if (d <= 0.0) continue;
                            double gd[8][3];
                            memset(gd, 0, sizeof gd);
                            int idx[3] = {a, b, c};
                            const double *X[3] = {x23, x31, x12};
                            for (int ax = 0; ax < 3; ++ax) {
                                int o0[3], o1[3];
                                edge_ends(ax, idx[ax], o0, o1);
                                int s0 = o0[0] + 2 * o0[1] + 4 * o0[2], s1 = o1[0] + 2 * o1[1] + 4 * o1[2];
                                for (int k = 0; k < 3; ++k) {
                                    gd[s1][k] += X[ax][k] / gsp(p, ax);
                                    gd[s0][k] -= X[ax][k] / gsp(p, ax);
                                }
                            }
                            for (int o = 0; o < 8; ++o)
                                for (int k = 0; k < 3; ++k) co[3 * o + k] += G * d2psi(d) * gd[o][k] * gd[o][k];
                        }
            }
#pragma omp parallel for collapse(2)
    for (int k3 = 0; k3 < m[2]; ++k3)
        for (int k2 = 0; k2 < m[1]; ++k2)
            for (int k1 = 0; k1 < m[0]; ++k1) {
                double acc[3] = {0, 0, 0};
                for (int o3 = 0; o3 < 2; ++o3)
                    for (int o2 = 0; o2 < 2; ++o2)
                        for (int o1 = 0; o1 < 2; ++o1) {
                            int c1 = k1 - o1, c2 = k2 - o2, c3 = k3 - o3;
                            if (c1 < 0 || c2 < 0 || c3 < 0 || c1 >= nc[0] || c2 >= nc[1] || c3 >= nc[2]) continue;
                            const double *co = cellout + 24 * (long)IDX(nc, c1, c2, c3);
                            int sidx = o1 + 2 * o2 + 4 * o3;
                            for (int comp = 0; comp < 3; ++comp) acc[comp] += co[3 * sidx + comp];
                        }
                long node = IDX(m, k1, k2, k3);
                for (int comp = 0; comp < 3; ++comp) out[comp * M + node] = acc[comp];
            }
    free(cellout);
}

/* ------------------------------------------------------------------ */
/* Keypoint penalty, Eq. (10).                                         */
/* ------------------------------------------------------------------ */
static void kp_weights(const orc_problem *p, const double *x, int c[3], double f[3]) {
    for (int a = 0; a < 3; ++a) {
        double t = x[a] / gsp(p, a);
        int ci = (int)floor(t);
        if (ci < 0) ci = 0;
        if (ci > p->m[a] - 2) ci = p->m[a] - 2;
        c[a] = ci;
        f[a] = t - ci;
    }
}

void orc_keypoints(const orc_problem *p, const double *u, const double *v, double *energy, double *out) {
    long M = nnod(p);
    if (out) memset(out, 0, sizeof(double) * 3 * M);
    double e = 0.0;
    for (int i = 0; i < p->nk; ++i) {
        int c[3];
        double f[3];
        kp_weights(p, p->kx + 3 * i, c, f);
        double yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
        for (int o3 = 0; o3 < 2; ++o3)
            for (int o2 = 0; o2 < 2; ++o2)
                for (int o1 = 0; o1 < 2; ++o1) {
                    double w = (o1 ? f[0] : 1 - f[0]) * (o2 ? f[1] : 1 - f[1]) * (o3 ? f[2] : 1 - f[2]);
                    long node = IDX(p->m, c[0] + o1, c[1] + o2, c[2] + o3);
                    for (int comp = 0; comp < 3; ++comp) {
                        yu[comp] += w * u[comp * M + node];
                        if (v) yv[comp] += w * v[comp * M + node];
                    }
                }
        double res[3];
        for (int comp = 0; comp < 3; ++comp) {
            res[comp] = p->kx[3 * i + comp] + yu[comp] - p->ky[3 * i + comp];
            e += res[comp] * res[comp];
        }
        if (out) {
            const double *src = v ? yv : res;      /* H_K v = 2 P^T P v;  grad = 2 P^T res */
            for (int o3 = 0; o3 < 2; ++o3)
                for (int o2 = 0; o2 < 2; ++o2)
                    for (int o1 = 0; o1 < 2; ++o1) {
                        double w = (o1 ? f[0] : 1 - f[0]) * (o2 ? f[1] : 1 - f[1]) * (o3 ? f[2] : 1 - f[2]);
                        long node = IDX(p->m, c[0] + o1, c[1] + o2, c[2] + o3);
                        for (int comp = 0; comp < 3; ++comp) out[comp * M + node] += 2.0 * w * src[comp];
                    }
        }
    }
    if (energy) *energy = e;
}

/* ------------------------------------------------------------------ */
/* Full objective, Eq. (11) (beta = 0: the mask term B is not used).   */
/* ------------------------------------------------------------------ */
int orc_gradient(const orc_problem *p, const double *u, double *terms, double *grad) {
    long M = nnod(p);
    double D = 0, Rc = 0, V = 0, K = 0;
    double *tmp = grad ? malloc(sizeof(double) * 3 * M) : NULL;
    int st = orc_ngf_gradient(p, u, &D, grad);
    if (st < 0) { free(tmp); return st; }
    orc_curvature(p, u, NULL, &Rc, tmp);
    if (grad) for (long i = 0; i < 3 * M; ++i) grad[i] += p->alpha * tmp[i];
    int fold = 0;
    if (p->gamma != 0.0) {
        fold = orc_vcc(p, u, NULL, &V, tmp, NULL);
        if (grad) for (long i = 0; i < 3 * M; ++i) grad[i] += p->gamma * tmp[i];
    }
    if (p->nk > 0) {
        orc_keypoints(p, u, NULL, &K, tmp);
        if (grad) for (long i = 0; i < 3 * M; ++i) grad[i] += p->delta * tmp[i];
    }
    free(tmp);
    double J = D + p->alpha * Rc + (p->gamma != 0.0 ? p->gamma * V : 0.0) + p->delta * K;
    if (fold) J = INFINITY;
    if (terms) { terms[0] = D; terms[1] = Rc; terms[2] = V; terms[3] = K; terms[4] = J; }
    return fold ? 1 : 0;
}

int orc_objective(const orc_problem *p, const double *u, double *terms) {
    return orc_gradient(p, u, terms, NULL);
}

/* ------------------------------------------------------------------ */
/* Gauss-Newton matrix.                                                */
/* ------------------------------------------------------------------ */
struct orc_lin {
    double *u;     /* linearisation point [3M] */
    double *dT;    /* dT/dy at voxels [3N] */
    double *a;     /* dr/dg at interior voxels [3N] */
};

orc_lin *orc_linearize(const orc_problem *p, const double *u) {
    long N = nvox(p), M = nnod(p);
    orc_lin *L = calloc(1, sizeof(orc_lin));
    L->u = malloc(sizeof(double) * 3 * M);
    L->dT = malloc(sizeof(double) * 3 * N);
    L->a = malloc(sizeof(double) * 3 * N);
    double *Tw = malloc(sizeof(double) * N);
    memcpy(L->u, u, sizeof(double) * 3 * M);
    orc_warp(p, u, Tw, L->dT);
    orc_ngf_distance(p, Tw, NULL, L->a);
    free(Tw);
    return L;
}

void orc_lin_free(orc_lin *L) {
    if (!L) return;
    free(L->u); free(L->dT); free(L->a); free(L);
}

/* H_D v = 2 hbar J^T (J v), J v at voxel = a . G(dT . P v). */
void orc_ngf_gn_matvec(const orc_problem *p, const orc_lin *L, const double *v, double *Hv) {
    long N = nvox(p);
    const int *n = p->n;
    double *Pv = malloc(sizeof(double) * 3 * N);
    double *dTw = malloc(sizeof(double) * N);
    double *c = malloc(sizeof(double) * 3 * N);
    orc_prolong(p, v, Pv);
    for (long w = 0; w < N; ++w) dTw[w] = L->dT[w] * Pv[w] + L->dT[N + w] * Pv[N + w] + L->dT[2 * N + w] * Pv[2 * N + w];
    double hb = hbar(p);
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < n[2]; ++i3)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i1 = 0; i1 < n[0]; ++i1) {
                long vx = IDX(n, i1, i2, i3);
                if (!interior(n, i1, i2, i3)) { c[vx] = c[N + vx] = c[2 * N + vx] = 0.0; continue; }
                long st[3] = {1, n[0], (long)n[0] * n[1]};
                double dr = 0.0;
                for (int k = 0; k < 3; ++k) dr += L->a[k * N + vx] * (dTw[vx + st[k]] - dTw[vx - st[k]]) / (2.0 * p->h[k]);
                for (int k = 0; k < 3; ++k) c[k * N + vx] = 2.0 * hb * dr * L->a[k * N + vx];
            }
    adjoint_to_voxels(p, c, L->dT, Pv);
    prolong_transpose(p, Pv, Hv);
    free(Pv); free(dTw); free(c);
}

void orc_gn_matvec(const orc_problem *p, const orc_lin *L, const double *v, double *Hv) {
    long M = nnod(p);
    double *tmp = malloc(sizeof(double) * 3 * M);
    orc_ngf_gn_matvec(p, L, v, Hv);
    orc_curvature(p, L->u, v, NULL, tmp);
    for (long i = 0; i < 3 * M; ++i) Hv[i] += p->alpha * tmp[i];
    if (p->gamma != 0.0) {
        orc_vcc(p, L->u, v, NULL, tmp, NULL);
        for (long i = 0; i < 3 * M; ++i) Hv[i] += p->gamma * tmp[i];
    }
    if (p->nk > 0) {
        orc_keypoints(p, L->u, v, NULL, tmp);
        for (long i = 0; i < 3 * M; ++i) Hv[i] += p->delta * tmp[i];
    }
    free(tmp);
}

/* Jacobi preconditioner: diagonal of the Gauss-Newton matrix H, with the
 * NGF part taken without the cross terms of the central-difference adjoint:
 *   M = 2 hbar sum_x w_k(x)^2 dT_c(x)^2 beta_x                 (NGF, approximate)
 *     + alpha diag(H_R) + gamma diag(H_V) + delta diag(H_K)     (exact)
 *     + tau,
 * beta_x = sum_a (a_{x-e_a,a}^2 + a_{x+e_a,a}^2) / (4 h_a^2), w_k the trilinear
 * weight of node k.  (J e_k)_v is a sum of six neighbour terms; the NGF part
 * keeps the sum of their squares.  Entries that come out as 0 are set to 1. */
static double node_weight(const orc_problem *p, int a, int i, int k) {
    int c;
    double f;
    axis_weight(i, ratio(p, a), &c, &f);
    if (c == k) return 1.0 - f;
    if (c == k - 1) return f;
    return 0.0;
}

void orc_gn_diag(const orc_problem *p, const orc_lin *L, double tau, double *diag) {
    long N = nvox(p), M = nnod(p);
    const int *n = p->n, *m = p->m;
    double hb = hbar(p), G = ghat(p), g2[3];
    for (int a = 0; a < 3; ++a) g2[a] = gsp(p, a) * gsp(p, a);
    /* beta_x */
    double *beta = malloc(sizeof(double) * N);
#pragma omp parallel for collapse(2)
    for (int i3 = 0; i3 < n[2]; ++i3)
        for (int i2 = 0; i2 < n[1]; ++i2)
            for (int i1 = 0; i1 < n[0]; ++i1) {
                int ii[3] = {i1, i2, i3};
                long st[3] = {1, n[0], (long)n[0] * n[1]};
                long x = IDX(n, i1, i2, i3);
                double b = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double s = 0.0;
                    if (ii[a] - 1 >= 0) s += L->a[a * N + x - st[a]] * L->a[a * N + x - st[a]];
                    if (ii[a] + 1 <= n[a] - 1) s += L->a[a * N + x + st[a]] * L->a[a * N + x + st[a]];
                    b += s / (4.0 * p->h[a] * p->h[a]);
                }
                beta[x] = b;
            }
    /* NGF part and curvature part, gathered per node */
#pragma omp parallel for collapse(2)
    for (int k3 = 0; k3 < m[2]; ++k3)
        for (int k2 = 0; k2 < m[1]; ++k2)
            for (int k1 = 0; k1 < m[0]; ++k1) {
                int kk[3] = {k1, k2, k3};
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    int rho = ratio(p, a);
                    lo[a] = (kk[a] - 1) * rho; if (lo[a] < 0) lo[a] = 0;
                    hi[a] = (kk[a] + 1) * rho - 1; if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
                }
                double acc[3] = {0, 0, 0};
                for (int i3 = lo[2]; i3 <= hi[2]; ++i3)
                    for (int i2 = lo[1]; i2 <= hi[1]; ++i2)
                        for (int i1 = lo[0]; i1 <= hi[0]; ++i1) {
                            double w = node_weight(p, 0, i1, k1) * node_weight(p, 1, i2, k2) * node_weight(p, 2, i3, k3);
                            if (w == 0.0) continue;
                            long x = IDX(n, i1, i2, i3);
                            for (int c = 0; c < 3; ++c) acc[c] += w * w * L->dT[c * N + x] * L->dT[c * N + x] * beta[x];
                        }
                double own = 0.0, nb = 0.0;
                for (int a = 0; a < 3; ++a) {
                    if (node_interior_axis(m, kk, a)) own += -2.0 / g2[a];
                    int km[3] = {k1, k2, k3}, kp[3] = {k1, k2, k3};
                    km[a] -= 1; kp[a] += 1;
                    if (km[a] >= 0 && node_interior_axis(m, km, a)) nb += 1.0 / (g2[a] * g2[a]);
                    if (kp[a] <= m[a] - 1 && node_interior_axis(m, kp, a)) nb += 1.0 / (g2[a] * g2[a]);
                }
                long node = IDX(m, k1, k2, k3);
                for (int c = 0; c < 3; ++c) diag[c * M + node] = 2.0 * hb * acc[c] + p->alpha * G * (own * own + nb);
            }
    free(beta);
    /* VCC part: per cell, psi''(d) (d d / d u_{k,c})^2 for its 8 corners */
    if (p->gamma != 0.0) {
        double *vd = malloc(sizeof(double) * 3 * M);
        orc_vcc_diag(p, L->u, vd);
        for (long i = 0; i < 3 * M; ++i) diag[i] += p->gamma * vd[i];
        free(vd);
    }
    if (p->nk > 0 && p->delta != 0.0)
        for (int i = 0; i < p->nk; ++i) {
            int c[3];
            double f[3];
            kp_weights(p, p->kx + 3 * i, c, f);
            for (int o3 = 0; o3 < 2; ++o3)
                for (int o2 = 0; o2 < 2; ++o2)
                    for (int o1 = 0; o1 < 2; ++o1) {
                        double w = (o1 ? f[0] : 1 - f[0]) * (o2 ? f[1] : 1 - f[1]) * (o3 ? f[2] : 1 - f[2]);
                        long node = IDX(m, c[0] + o1, c[1] + o2, c[2] + o3);
                        for (int comp = 0; comp < 3; ++comp) diag[comp * M + node] += 2.0 * p->delta * w * w;
                    }
        }
    for (long i = 0; i < 3 * M; ++i) {
        diag[i] += tau;
        if (!(diag[i] > 0.0)) diag[i] = 1.0;
    }
}

static double vdot(long n, const double *a, const double *b) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Preconditioned conjugate gradients, s0 = 0, exactly `iters` steps unless
 * the residual vanishes or the curvature p.Hp is not positive, with full
 * reorthogonalisation: each new residual r is made orthogonal to all earlier
 * preconditioned residuals z_j, r <- r - sum_j (r.z_j / r_j.z_j) r_j with
 * every coefficient taken from the same r (classical Gram-Schmidt) (same
 * iterates as plain PCG in exact arithmetic; keeps them so in floating point).
 * stats = {steps done, |r0|, |r_final|}. */
int orc_pcg(const orc_problem *p, const orc_lin *L, const double *g, double *s, int iters,
            double tau, double *stats) {
    long n3 = 3 * nnod(p);
    double *R = malloc(sizeof(double) * n3 * (iters + 1));   /* residual history r_0..r_iters */
    double *Z = malloc(sizeof(double) * n3 * (iters + 1));   /* preconditioned residuals */
    double *rz = malloc(sizeof(double) * (iters + 1));
    double *d = malloc(sizeof(double) * n3), *q = malloc(sizeof(double) * n3);
    double *Md = malloc(sizeof(double) * n3);
    orc_gn_diag(p, L, tau, Md);
    double *r = R, *z = Z;
    for (long i = 0; i < n3; ++i) { s[i] = 0.0; r[i] = -g[i]; z[i] = r[i] / Md[i]; d[i] = z[i]; }
    rz[0] = vdot(n3, r, z);
    double r0 = sqrt(vdot(n3, r, r));
    int k = 0;
    for (; k < iters; ++k) {
        if (rz[k] == 0.0) break;
        orc_gn_matvec(p, L, d, q);
        double dq = vdot(n3, d, q);
        if (!(dq > 0.0)) break;
        double al = rz[k] / dq;
        double *rn = R + (k + 1) * n3, *zn = Z + (k + 1) * n3, *rk = R + k * n3;
        for (long i = 0; i < n3; ++i) { s[i] += al * d[i]; rn[i] = rk[i] - al * q[i]; }
        /* classical Gram-Schmidt: all coefficients from the same r_{k+1} */
        double *cj = malloc(sizeof(double) * (k + 1));
        for (int j = 0; j <= k; ++j) cj[j] = rz[j] != 0.0 ? vdot(n3, rn, Z + j * n3) / rz[j] : 0.0;
        for (int j = 0; j <= k; ++j) {
            const double *rj = R + j * n3;
            for (long i = 0; i < n3; ++i) rn[i] -= cj[j] * rj[i];
        }
        free(cj);
        for (long i = 0; i < n3; ++i) zn[i] = rn[i] / Md[i];
        rz[k + 1] = vdot(n3, rn, zn);
        double be = rz[k + 1] / rz[k];
        for (long i = 0; i < n3; ++i) d[i] = zn[i] + be * d[i];
    }
    if (stats) { stats[0] = k; stats[1] = r0; stats[2] = sqrt(vdot(n3, R + k * n3, R + k * n3)); }
    free(R); free(Z); free(rz); free(d); free(q); free(Md);
    return k;
}

/* One level: fixed number of Gauss-Newton steps, each a fixed-length PCG
 * solve and an Armijo backtracking line search (t = 1, 1/2, ..., 2^-ls_max;
 * a step with J = +inf is rejected; if none is accepted, u is kept).
 * report[8*it + .] = {it, J, g.s, t accepted (0 = none), J new, evaluations,
 *                     pcg steps, status}. */
int orc_gn_solve(orc_problem *p, double *u, int gn_iters, int pcg_iters, int ls_max,
                 double armijo_c, double tau, int delta_adaptive, double *report) {
    long n3 = 3 * nnod(p);
    double *g = malloc(sizeof(double) * n3), *s = malloc(sizeof(double) * n3);
    double *ut = malloc(sizeof(double) * n3);
    double terms[5];
    if (delta_adaptive) {
        /* delta such that D = delta K at the start (Sec. II-D2) */
        double D0, K0 = 0.0;
        orc_ngf_gradient(p, u, &D0, NULL);
        if (p->nk > 0) orc_keypoints(p, u, NULL, &K0, NULL);
        p->delta = K0 > 0.0 ? D0 / K0 : 0.0;
    }
    int status = 0;
    for (int it = 0; it < gn_iters; ++it) {
        double *rep = report ? report + 8 * it : NULL;
        int st = orc_gradient(p, u, terms, g);
        double J0 = terms[4];
        if (st != 0) { status = st; if (rep) { rep[0] = it; rep[1] = J0; rep[7] = st; } break; }
        orc_lin *L = orc_linearize(p, u);
        double pst[3];
        orc_pcg(p, L, g, s, pcg_iters, tau, pst);
        orc_lin_free(L);
        double slope = vdot(n3, g, s);
        double t = 1.0, acc_t = 0.0, Jn = J0;
        int evals = 0;
        for (int k = 0; k <= ls_max; ++k) {
            for (long i = 0; i < n3; ++i) ut[i] = u[i] + t * s[i];
            double tt[5];
            int fs = orc_objective(p, ut, tt);
            ++evals;
            if (fs == 0 && tt[4] <= J0 + armijo_c * t * slope) { acc_t = t; Jn = tt[4]; break; }
            t *= 0.5;
        }
        if (acc_t > 0.0) memcpy(u, ut, sizeof(double) * n3);
        if (rep) {
            rep[0] = it; rep[1] = J0; rep[2] = slope; rep[3] = acc_t; rep[4] = Jn;
            rep[5] = evals; rep[6] = pst[0]; rep[7] = 0;
        }
    }
    free(g); free(s); free(ut);
    return status;
}

/* ------------------------------------------------------------------ */
/* Multilevel scheme (Sec. II-D3).                                     */
/* ------------------------------------------------------------------ */
void orc_restrict_image(const int *n, const float *in, float *out) {
    int nc[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
#pragma omp parallel for collapse(2)
    for (int j3 = 0; j3 < nc[2]; ++j3)
        for (int j2 = 0; j2 < nc[1]; ++j2)
            for (int j1 = 0; j1 < nc[0]; ++j1) {
                double s = 0.0;
                for (int o3 = 0; o3 < 2; ++o3)
                    for (int o2 = 0; o2 < 2; ++o2)
                        for (int o1 = 0; o1 < 2; ++o1) s += in[IDX(n, 2 * j1 + o1, 2 * j2 + o2, 2 * j3 + o3)];
                out[IDX(nc, j1, j2, j3)] = (float)(s / 8.0);
            }
}

/* Coarse node k sits at fine node 2k; odd fine nodes take the average of
 * their two coarse neighbours (exact trilinear interpolation, per axis). */
void orc_prolong_grid(const int *mc, const double *uc, const int *mf, double *uf) {
    long Mc = (long)mc[0] * mc[1] * mc[2], Mf = (long)mf[0] * mf[1] * mf[2];
    for (int comp = 0; comp < 3; ++comp)
        for (int k3 = 0; k3 < mf[2]; ++k3)
            for (int k2 = 0; k2 < mf[1]; ++k2)
                for (int k1 = 0; k1 < mf[0]; ++k1) {
                    int kk[3] = {k1, k2, k3}, lo[3], hi[3];
                    for (int a = 0; a < 3; ++a) { lo[a] = kk[a] / 2; hi[a] = (kk[a] + 1) / 2; }
                    double s = 0.0;
                    for (int o3 = 0; o3 < 2; ++o3)
                        for (int o2 = 0; o2 < 2; ++o2)
                            for (int o1 = 0; o1 < 2; ++o1) {
                                int c1 = o1 ? hi[0] : lo[0], c2 = o2 ? hi[1] : lo[1], c3 = o3 ? hi[2] : lo[2];
                                s += uc[comp * Mc + IDX(mc, c1, c2, c3)];
                            }
                    uf[comp * Mf + IDX(mf, k1, k2, k3)] = s / 8.0;
                }
}

int orc_register_pyramid(orc_problem *fin, int levels, double *u, int gn_iters, int pcg_iters,
                         int ls_max, double armijo_c, double tau, int delta_adaptive, double *report) {
    if (levels < 1) return -1;
    for (int a = 0; a < 3; ++a)
        if (fin->n[a] % (1 << (levels - 1)) || (fin->m[a] - 1) % (1 << (levels - 1))) return -1;
    float *R[8] = {0}, *T[8] = {0};
    int nl[8][3], ml[8][3];
    for (int a = 0; a < 3; ++a) { nl[0][a] = fin->n[a]; ml[0][a] = fin->m[a]; }
    R[0] = (float *)fin->R; T[0] = (float *)fin->T;
    for (int l = 1; l < levels; ++l) {
        for (int a = 0; a < 3; ++a) { nl[l][a] = nl[l - 1][a] / 2; ml[l][a] = (ml[l - 1][a] - 1) / 2 + 1; }
        long Nl = (long)nl[l][0] * nl[l][1] * nl[l][2];
        R[l] = malloc(sizeof(float) * Nl);
        T[l] = malloc(sizeof(float) * Nl);
        orc_restrict_image(nl[l - 1], R[l - 1], R[l]);
        orc_restrict_image(nl[l - 1], T[l - 1], T[l]);
    }
    /* start: injection of u onto the coarsest grid (node k <- fine node 2^L k) */
    int Lc = levels - 1;
    long Mc = (long)ml[Lc][0] * ml[Lc][1] * ml[Lc][2], Mf = (long)fin->m[0] * fin->m[1] * fin->m[2];
    double *ul = malloc(sizeof(double) * 3 * Mc);
    int sc = 1 << Lc;
    for (int comp = 0; comp < 3; ++comp)
        for (int k3 = 0; k3 < ml[Lc][2]; ++k3)
            for (int k2 = 0; k2 < ml[Lc][1]; ++k2)
                for (int k1 = 0; k1 < ml[Lc][0]; ++k1)
                    ul[comp * Mc + IDX(ml[Lc], k1, k2, k3)] = u[comp * Mf + IDX(fin->m, sc * k1, sc * k2, sc * k3)];
    double delta = fin->delta;
    int status = 0;
    for (int l = Lc; l >= 0; --l) {
        orc_problem pl = *fin;
        for (int a = 0; a < 3; ++a) { pl.n[a] = nl[l][a]; pl.m[a] = ml[l][a]; pl.h[a] = fin->h[a] * (1 << l); }
        pl.R = R[l]; pl.T = T[l]; pl.delta = delta;
        int adapt = delta_adaptive && l == Lc;
        status = orc_gn_solve(&pl, ul, gn_iters, pcg_iters, ls_max, armijo_c, tau, adapt,
                              report ? report + (long)(Lc - l) * gn_iters * 8 : NULL);
        delta = pl.delta;
        if (status != 0) break;
        if (l > 0) {
            long Mn = (long)ml[l - 1][0] * ml[l - 1][1] * ml[l - 1][2];
            double *un = malloc(sizeof(double) * 3 * Mn);
            orc_prolong_grid(ml[l], ul, ml[l - 1], un);
            free(ul);
            ul = un;
        }
    }
    if (status == 0) memcpy(u, ul, sizeof(double) * 3 * Mf);
    free(ul);
    for (int l = 1; l < levels; ++l) { free(R[l]); free(T[l]); }
    fin->delta = delta;
    return status;
}
