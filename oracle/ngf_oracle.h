/*
 * FP64 CPU oracle for the dense continuous registration objective of
 * Ruehaak et al., "Estimation of Large Motion in Lung CT by Integrating
 * Regularized Keypoint Correspondences into Dense Deformable Registration"
 * (arXiv 1807.00467), Sec. II-D, Eqs. (1), (5), (7)-(11).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference the
 * GPU path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the GPU
 * library and must never be used as a fallback for it.
 *
 * Conventions (the discretisation the paper leaves open; each choice is a
 * documented reading):
 *   - Images are [n3][n2][n1] with x fastest, cell-centred voxels:
 *     voxel i has centre (i + 1/2) * h (mm).  Domain [0, n*h].
 *   - The displacement grid has m nodes per axis spanning the domain exactly,
 *     node spacing g = n*h/(m-1); rho = n/(m-1) must be a power of two.
 *     u is stored component-major [3][m3][m2][m1] (mm); y(x) = x + (P u)(x),
 *     P = trilinear interpolation (first-order B-spline, Sec. II-D1/II-D3).
 *   - Status: 0 ok, 1 fold (some Jacobian bound d <= 0, objective +inf),
 *     negative on invalid arguments.
 */
#ifndef NGF_ORACLE_H
#define NGF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n[3];            /* voxels per axis (x, y, z) */
    double h[3];         /* voxel spacing, mm */
    int m[3];            /* grid nodes per axis */
    const float *R;      /* reference (fixed) image F */
    const float *T;      /* template (moving) image M */
    double eta;          /* NGF edge parameter, Eq. (1) */
    double alpha;        /* curvature weight, Eq. (11) */
    double gamma;        /* volume-change weight, Eq. (11) */
    double delta;        /* keypoint weight, Eq. (11) */
    int nk;              /* number of keypoints */
    const double *kx;    /* [nk][3] keypoint positions x_i (mm) */
    const double *ky;    /* [nk][3] keypoint targets y_KP(x_i) (mm) */
} orc_problem;

typedef struct orc_lin orc_lin;   /* stored linearisation (Gauss-Newton point) */

int orc_check(const orc_problem *p);

/* Trilinear prolongation of a grid field onto voxel centres: disp [3][N]. */
void orc_prolong(const orc_problem *p, const double *u, double *disp);

/* The sample cell of every voxel along each axis, k[a][v] = i_a + floor(s_a)
 * before clamping, as decided in FP32 (the integer decision both the GPU
 * kernels and orc_warp take; exported for its pin against the FP64 floor). */
void orc_cells(const orc_problem *p, const double *u, int *k);

/* Warped template Tw = T(y) and its derivative dT = dT/dy ([3][N]), Eq. (1). */
void orc_warp(const orc_problem *p, const double *u, double *Tw, double *dT);

/* NGF distance D, Eq. (1); r and a = dr/dg at interior voxels (may be NULL). */
double orc_ngf_distance(const orc_problem *p, const double *Tw, double *r, double *a);

/* terms = {D, R, V, K, J}; returns 1 on fold.  grad may be NULL. */
int orc_objective(const orc_problem *p, const double *u, double *terms);
int orc_gradient(const orc_problem *p, const double *u, double *terms, double *grad);
int orc_ngf_gradient(const orc_problem *p, const double *u, double *D, double *grad);

/* Regularisers.  v == NULL: out = gradient; else out = (GN) Hessian times v. */
void orc_curvature(const orc_problem *p, const double *u, const double *v, double *energy, double *out);
int orc_vcc(const orc_problem *p, const double *u, const double *v, double *energy, double *out,
            double *dminmax);
/* The 64 bounds d_abc of one grid cell; edge e of axis a joins the nodes
 * offset by (e & 1, e >> 1) along the other two axes in increasing axis order. */
void orc_vcc_cell_dets(const orc_problem *p, const double *u, const int *cell, double *d64);
void orc_keypoints(const orc_problem *p, const double *u, const double *v, double *energy, double *out);

/* Gauss-Newton matrix H = H_D + alpha H_R + gamma H_V + delta H_K at u. */
orc_lin *orc_linearize(const orc_problem *p, const double *u);
void orc_lin_free(orc_lin *L);
void orc_ngf_gn_matvec(const orc_problem *p, const orc_lin *L, const double *v, double *Hv);
void orc_gn_matvec(const orc_problem *p, const orc_lin *L, const double *v, double *Hv);
/* Jacobi preconditioner at the linearisation: NGF diagonal without the
 * adjoint's cross terms, exact curvature / VCC / keypoint diagonals, + tau. */
void orc_gn_diag(const orc_problem *p, const orc_lin *L, double tau, double *diag);
void orc_vcc_diag(const orc_problem *p, const double *u, double *out);

/* Jacobi-preconditioned CG on H s = -g, fixed iteration count, s0 = 0. */
int orc_pcg(const orc_problem *p, const orc_lin *L, const double *g, double *s, int iters,
            double tau, double *stats);

/* Fixed Gauss-Newton schedule with Armijo backtracking; report[it*8 + k]. */
int orc_gn_solve(orc_problem *p, double *u, int gn_iters, int pcg_iters, int ls_max,
                 double armijo_c, double tau, int delta_adaptive, double *report);

/* Pyramid helpers (2x2x2 box restriction; dyadic grid prolongation). */
void orc_restrict_image(const int *n, const float *in, float *out);
void orc_prolong_grid(const int *mc, const double *uc, const int *mf, double *uf);
int orc_register_pyramid(orc_problem *finest, int levels, double *u, int gn_iters, int pcg_iters,
                         int ls_max, double armijo_c, double tau, int delta_adaptive, double *report);

int orc_num_threads(void);
void orc_set_threads(int n);   /* OpenMP threads of the following calls (timing on fewer cores) */

#ifdef __cplusplus
}
#endif
#endif
