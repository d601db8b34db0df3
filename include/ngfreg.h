/*
 * ngfreg: GB300 (sm_103a) library for the dense continuous registration stage
 * of Ruehaak et al., "Estimation of Large Motion in Lung CT by Integrating
 * Regularized Keypoint Correspondences into Dense Deformable Registration"
 * (arXiv 1807.00467), Sec. II-D.
 *
 * The objective (Eq. (11), with the mask term B left out, beta = 0) is
 *     J(u) = D(u) + alpha R(u) + gamma V(u) + delta K(u)
 *   D  normalized gradient fields distance, Eq. (1)
 *   R  curvature regulariser, Eq. (5) (y_hat = identity)
 *   V  volume change control in the 64-bound form V-hat, Eqs. (7)-(9)
 *   K  quadratic keypoint penalty, Eq. (10)
 * over a displacement u on a node grid, y(x) = x + (P u)(x) with P trilinear
 * interpolation (first-order B-spline, Sec. II-D1 and II-D3).  The library
 * evaluates J, its gradient, Gauss-Newton matrix-vector products (the
 * "Hessian approximation" of Sec. II-D3), a fixed-length Jacobi PCG solve, a
 * fixed Gauss-Newton schedule with Armijo backtracking, and a multilevel
 * (pyramid) driver, all matrix-free (Sec. II-D3).
 *
 * Discretisation (the paper leaves these open):
 *   - Images are [n3][n2][n1] (x fastest), cell-centred voxels: voxel i has
 *     centre (i + 1/2) h, in mm.  D sums over interior voxels 1..n-2 of each
 *     axis with central differences of R and of the warped template.
 *   - The node grid has m nodes per axis spanning [0, n h] exactly, node
 *     spacing g = n h / (m - 1); rho = n / (m - 1) must be 1, 2, 4 or 8.
 *     Grid fields are float32 [3][m3][m2][m1] (x, y, z components, mm).
 *   - Out-of-domain samples of the template are clamped per axis, with zero
 *     derivative along a clamped axis.  The sample cell of each voxel is
 *     chosen in FP32 from the displacement interpolated along x, then y, then
 *     z (each step fma(w1, b, w0 * a)), times float(1/h), floor.
 *
 * Conventions for every call:
 *   - All pointers named *_dev are device pointers (cudaMalloc'd or torch
 *     tensors' data_ptr); the caller owns them.  Arrays are contiguous.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous unless
 *     stated otherwise.  Outputs are written on that stream.
 *   - The library allocates no device memory after rg_ctx_create: it carves
 *     all scratch from the caller's workspace (rg_workspace_size bytes).
 *   - Return value: RG_OK (0), RG_EFOLD (1: some Jacobian bound d <= 0, the
 *     objective is +inf), or a negative error code.  Errors are latched in
 *     the context and described by rg_last_error().
 */
#ifndef NGFREG_H
#define NGFREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RG_OK 0
#define RG_EFOLD 1
#define RG_EINVAL (-1)
#define RG_ECUDA (-2)
#define RG_ENOMEM (-3)
#define RG_ENONFINITE (-4)
#define RG_ETIMEOUT (-5)
#define RG_ESCRATCH (-6)

/* Largest PCG length a workspace can be sized for (pcg_max). */
#define RG_PCG_MAX 63

/* Which regulariser regularizer_apply evaluates. */
#define RG_CURV 1
#define RG_VCC 2
#define RG_KP 4

typedef struct {
    int32_t n[3];    /* voxels per axis (x, y, z), each >= 4 */
    double h[3];     /* voxel spacing, mm */
} rg_image_geom;

typedef struct {
    int32_t m[3];    /* grid nodes per axis; n[a] / (m[a] - 1) in {1, 2, 4, 8} */
} rg_grid_geom;

typedef enum { RG_F32 = 0, RG_F16 = 1 } rg_dtype;

typedef struct {
    double eta;           /* NGF edge parameter eta of Eq. (1) */
    double alpha;         /* curvature weight, Eq. (11) */
    double gamma;         /* volume-change weight, Eq. (11); 0 disables V */
    double delta;         /* keypoint weight, Eq. (11) */
    int32_t delta_adaptive; /* 1: delta = D(u0)/K(u0) at the start (Sec. II-D2) */
    double tau;           /* extra shift added to the PCG preconditioner diagonal (0 by default) */
    double det_lo, det_hi; /* reporting bounds on the Jacobian bounds d of Eq. (8) (e.g. 0.25, 4): the
                              solve reports whether min d >= det_lo and max d <= det_hi; psi is unchanged */
} rg_params;

/* Columns of a Gauss-Newton report row: {it, J, g.p, t (0 = rejected),
 * J new, evaluations, pcg steps, status, min d, max d, in bounds}, where
 * min d / max d are the extremes of the 64 Jacobian bounds d of Eq. (8) over
 * all grid cells at the iterate after the step, and "in bounds" is 1 when
 * det_lo <= min d and max d <= det_hi, else 0. */
#define RG_REPORT_COLS 11

typedef struct {
    int32_t levels;       /* pyramid levels (register_pyramid), >= 1 */
    int32_t gn_iters;     /* Gauss-Newton steps per level */
    int32_t pcg_iters;    /* PCG steps per Gauss-Newton step */
    int32_t ls_max;       /* line search tries t = 1, 1/2, ..., 2^-ls_max */
    double armijo_c;      /* Armijo constant */
    int32_t flags;        /* 0: host-driven line search; RG_SCHED_DEVICE / RG_SCHED_GRAPH below */
} rg_schedule;

/* rg_schedule.flags.  RG_SCHED_DEVICE: the slope g.p, the Armijo test and the
 * update run on the device, so an iteration needs no host synchronisation
 * (every line-search try is launched; the tries after the accepted one skip
 * their work).  RG_SCHED_GRAPH: as RG_SCHED_DEVICE, with one iteration's
 * launches captured once into a CUDA graph and replayed gn_iters times.
 * Both run on a private stream of the context ordered after and before the
 * caller's stream, give the same bits as the host-driven loop, synchronise
 * once at the end, and apply when 1 <= gn_iters <= 256 and profiling is off
 * (otherwise the host-driven loop runs). */
#define RG_SCHED_DEVICE 1
#define RG_SCHED_GRAPH 2
/* rg_schedule.flags: run rg_autotune on each level's context (at the start
 * iterate) before its Gauss-Newton steps.  Combines with the flags above. */
#define RG_SCHED_AUTOTUNE 4
/* rg_schedule.flags, register_pyramid_batch only: the PCG steps of every pair
 * whose level the column GN-product kernel covers (volumes at least 68 voxels
 * wide and 20 high, whole grid cells per axis) run in one persistent
 * cooperative kernel per level iteration (up to 24 pairs per launch), whose
 * CTAs take (pair, tile) items from a work counter, each waiting (bounded;
 * RG_ETIMEOUT when a wait runs out) for the previous phase of its own pair.
 * Same bits per pair as without the flag.  RG_SCHED_HOOK_BARRIER is a test
 * hook: the first item's completion is withheld, so the waits on it run out
 * after a short poll count (no fault, no hang). */
#define RG_SCHED_PERSISTENT 8
#define RG_SCHED_HOOK_BARRIER 16

typedef struct rg_ctx rg_ctx;

/* Workspace bytes a context for this problem needs (nk_max: the largest
 * keypoint count rg_set_keypoints will be given, at most 2^27, with a grid of
 * fewer than 2^31 nodes when nonzero; pcg_max: the longest PCG solve,
 * 0..RG_PCG_MAX, whose residual history the workspace keeps).
 * Returns RG_EINVAL on bad geometry or sizes. */
int rg_workspace_size(const rg_image_geom *img, const rg_grid_geom *grid, rg_dtype dtype,
                      int32_t nk_max, int32_t pcg_max, size_t *bytes);

/* Create a context.  workspace_dev: caller-owned device memory of at least
 * rg_workspace_size bytes, 256-byte aligned, kept alive until destroy.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream). */
int rg_ctx_create(rg_ctx **ctx, const rg_image_geom *img, const rg_grid_geom *grid, rg_dtype dtype,
                  const rg_params *params, int32_t nk_max, int32_t pcg_max, void *workspace_dev,
                  size_t ws_bytes, void *cuda_stream);
int rg_ctx_destroy(rg_ctx *ctx);
int rg_set_params(rg_ctx *ctx, const rg_params *params);
int rg_get_params(const rg_ctx *ctx, rg_params *params);
int rg_set_stream(rg_ctx *ctx, void *cuda_stream);

/* Tile height (voxel rows per CTA, 8 or 16; default 16) of the NGF kernels,
 * for tuning.  The workspace covers both; results do not depend on it beyond
 * FP32 summation order.  Invalidates the stored preconditioner. */
int rg_set_tile(rg_ctx *ctx, int32_t tile_y);

/* Tile autotuner (the paper has no counterpart: it picks launch shapes).
 * Candidates (tile_y, general): (16, 2) the specialised kernels with the
 * column-marching objective/gradient pass (where the volume allows it),
 * (16, 3) the specialised kernels with the z-chunked tile pass, (16, 1) and
 * (8, 1) the general column kernel with 16- and 8-row tiles; untuned contexts
 * use (16, 0), the specialised kernels with the pass chosen by size (the
 * column pass with at least one 60 x 16 voxel column per SM).  Each is timed
 * with CUDA events on the context's stream at u_dev (one linearisation pass
 * and three GN products, after one untimed round; the stream is synchronised)
 * and scored as one Gauss-Newton iteration, gradient pass + 30 products; the
 * fastest is kept in the context (tile_y / general, either may be NULL,
 * report it) and cached per process by image and grid shape, image type and
 * active terms, so later contexts of the same problem skip the timing.
 * Results of the candidates agree within the stated tolerances, not bit for
 * bit. The linearisation is discarded: call gn_linearize again before
 * gn_matvec / gn_pcg_solve. */
int rg_autotune(rg_ctx *ctx, const float *u_dev, int32_t *tile_y, int32_t *general);

/* Borrow the reference R (fixed image F) and template T (moving image M),
 * [n3][n2][n1], float32 for RG_F32, IEEE half of (HU + 1024) for RG_F16.
 * The pointers must stay valid while the context uses them. */
int rg_set_images(rg_ctx *ctx, const void *R_dev, const void *T_dev);

/* Borrow keypoints: x_dev, ykp_dev are float32 [nk][3] (mm), Eq. (10).
 * Also indexes the keypoints' cells on the context stream (the trilinear
 * weights of x_i are fixed), so the penalty's node sums are gathered in a
 * fixed order, without atomics: the same bits on every call.  The index
 * ranks the keypoints by pairwise comparison (nk^2 comparisons: about a
 * millisecond at 10^5 keypoints).  x_dev's contents must not change while
 * set; call again after changing them. */
int rg_set_keypoints(rg_ctx *ctx, int32_t nk, const float *x_dev, const float *ykp_dev);

/* terms_dev: double[5] = {D, R, V, K, J}, Eq. (11).  J = +inf on a fold. */
int ngf_objective(rg_ctx *ctx, const float *u_dev, double *terms_dev);

/* As ngf_objective, plus grad_dev = dJ/du, float32 [3][m3][m2][m1]. */
int ngf_gradient(rg_ctx *ctx, const float *u_dev, double *terms_dev, float *grad_dev);

/* Store the Gauss-Newton linearisation at u (per-voxel dT/dy and dr/dg, and
 * u itself for the VCC term) for subsequent gn_matvec / gn_pcg_solve calls.
 * If grad_dev / terms_dev are not NULL the gradient and terms at u are
 * produced by the same pass. */
int gn_linearize(rg_ctx *ctx, const float *u_dev, double *terms_dev, float *grad_dev);

/* Hv = H v with H = H_D + alpha H_R + gamma H_V + delta H_K at the stored
 * linearisation; H_D = 2 hbar J^T J, J = dr/du (NGF residual Jacobian). */
int gn_matvec(rg_ctx *ctx, const float *v_dev, float *Hv_dev);

/* One regulariser (which = RG_CURV, RG_VCC or RG_KP) at u: v_dev == NULL
 * gives out = gradient, else out = (GN) Hessian times v; energy_dev: one
 * double (unweighted energy).  Weights alpha, gamma, delta are NOT applied. */
int regularizer_apply(rg_ctx *ctx, int32_t which, const float *u_dev, const float *v_dev,
                      double *energy_dev, float *out_dev);

/* Fixed-length Jacobi-preconditioned CG on H p = -g at the stored
 * linearisation, p0 = 0, iters <= pcg_max; stops early only if r.z or p.Hp
 * stop being positive.  Each new residual is reorthogonalised against all
 * earlier preconditioned residuals (classical Gram-Schmidt): the iterates of
 * plain PCG in exact arithmetic, kept so in FP32.  Preconditioner: the
 * diagonal of H, with the NGF part taken
 * without the cross terms of the central-difference adjoint
 * (2 hbar sum_x w_k(x)^2 dT_c(x)^2 sum_a (a_{x-e_a,a}^2 + a_{x+e_a,a}^2)/(4 h_a^2)),
 * plus tau; non-positive entries use 1.  g_dev and p_dev must be 16-byte
 * aligned (cudaMalloc and PyTorch allocations are), else RG_EINVAL.
 * stats_dev: double[3] = {steps, |r0|, |r_end|} (may be NULL). */
int gn_pcg_solve(rg_ctx *ctx, const float *g_dev, float *p_dev, int32_t iters, double *stats_dev);

/* Fixed Gauss-Newton schedule on one level: gn_iters x (gradient +
 * linearisation, PCG, Armijo backtracking).  u_dev is updated in place.
 * report_host: double[gn_iters][RG_REPORT_COLS] (see RG_REPORT_COLS) or NULL.  Host-driven (flags 0):
 * synchronises the stream once per line-search try; see RG_SCHED_DEVICE. */
int gn_solve(rg_ctx *ctx, float *u_dev, const rg_schedule *sched, double *report_host);

/* Multilevel registration (Sec. II-D3): levels-1 times 2x2x2 box restriction
 * of R and T and halving of the grid, coarse-to-fine gn_solve, dyadic grid
 * prolongation between levels.  R_dev, T_dev, u_inout_dev are at the finest
 * level; u_inout's start value is injected onto the coarsest grid.
 * workspace_dev: rg_pyramid_workspace_size bytes.  report_host:
 * double[levels][gn_iters][RG_REPORT_COLS] (coarsest first) or NULL. */
int rg_pyramid_workspace_size(const rg_image_geom *img, const rg_grid_geom *finest, rg_dtype dtype,
                              int32_t levels, int32_t nk_max, int32_t pcg_max, size_t *bytes);
int register_pyramid(const rg_image_geom *img, const void *R_dev, const void *T_dev, rg_dtype dtype,
                     const rg_grid_geom *finest, const rg_params *params, const rg_schedule *sched,
                     int32_t nk, const float *kx_dev, const float *ky_dev, float *u_inout_dev,
                     double *report_host, void *workspace_dev, size_t ws_bytes, void *cuda_stream);

/* Many pairs through register_pyramid's schedule in lockstep (batching; the
 * paper has no counterpart).  Per pair p: img[p], R[p], T[p] (dtype shared),
 * fin[p], u_inout[p] and a workspace ws[p] of rg_pyramid_workspace_size(...,
 * nk_max = 0, ...) bytes (ws_bytes[p]); params and sched are shared, no
 * keypoints; 1 <= gn_iters <= 256; of sched->flags only RG_SCHED_PERSISTENT
 * and RG_SCHED_HOOK_BARRIER apply.  At each level
 * one CUDA graph holds every pair's Gauss-Newton iteration (line search
 * decided on the device) as a parallel branch and is replayed gn_iters times:
 * one graph launch advances all pairs.  Per pair the results have the bits of
 * register_pyramid with RG_SCHED_GRAPH.  report_host: double
 * [npairs][levels][gn_iters][RG_REPORT_COLS] or NULL.  A pair whose schedule
 * halts (a fold at the iterate, RG_EFOLD, or a non-finite objective,
 * RG_ENONFINITE) leaves the batch after that level: its u_inout keeps its start
 * value and its report rows stop at the halting row (status in column 7,
 * later rows zero); the other pairs run to the end and get their results.
 * Returns RG_OK, else the halting code of the lowest-numbered pair that halted;
 * other errors (RG_EINVAL, RG_ECUDA, RG_ETIMEOUT) abort the whole batch with no
 * output written.  Synchronises the stream once per level. */
int register_pyramid_batch(int32_t npairs, const rg_image_geom *img, const void *const *R, const void *const *T,
                           rg_dtype dtype, const rg_grid_geom *finest, const rg_params *params,
                           const rg_schedule *sched, float *const *u_inout, double *report_host,
                           void *const *workspace_dev, const size_t *ws_bytes, void *cuda_stream);

/* 2x2x2 box restriction of an image (float32 or half as dtype), n even. */
int rg_restrict_image(const int32_t *n, rg_dtype dtype, const void *in_dev, void *out_dev, void *cuda_stream);
/* Dyadic trilinear prolongation of a grid field from mc nodes to mf = 2 mc - 1. */
int rg_prolong_grid(const int32_t *mc, const float *uc_dev, float *uf_dev, void *cuda_stream);

/* NGF distance D of Eq. (1) at u without any device allocation (the paper
 * has no counterpart: this serves callers that cannot allocate device
 * memory, e.g. while a stream is being captured, inside a host application
 * that owns all device buffers, or under a fixed memory budget).  Images are
 * float32 [n3][n2][n1]; u is float32 [3][m3][m2][m1]; D_dev receives one
 * double.  Its only scratch is a file-scope device array of
 * RG_NOALLOC_MAX_CTAS doubles (512 KB on every GPU that loads the library,
 * held until the process exits), one partial sum per CTA: problems needing
 * more CTAs return RG_ESCRATCH.  A CTA covers a tile of 28 - 28 % rho_x voxels
 * in x (rho_x = n[0] / (m[0] - 1)), 16 in y and a z chunk of at most 32 slices
 * (fewer, whole grid cells, for large ratios), so the CTA count is
 * ceil(n[0] / tx) x ceil(n[1] / 16) x ceil(n[2] / tz).  Each call overwrites
 * the partials before reading them.  All calls share that array, so calls
 * whose kernels overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.
 * The first call on each device looks the array's device address up with
 * cudaGetSymbolAddress on the current device; make that first call before
 * any stream capture.  Enqueued on cuda_stream; asynchronous. */
#define RG_NOALLOC_MAX_CTAS 65536
int ngf_distance_noalloc(const rg_image_geom *img, const rg_grid_geom *grid, const float *R_dev,
                         const float *T_dev, const float *u_dev, double eta, double *D_dev,
                         void *cuda_stream);

/* Per-kernel timing with CUDA events recorded on the context stream around
 * every kernel launch while enabled.  Kernel ids: 0 NGF Gauss-Newton product
 * tile kernel, 1 NGF gradient/linearisation tile kernel, 2 NGF objective tile
 * kernel, 3 VCC gradient, 4 VCC Gauss-Newton product, 5 curvature L, 6 node
 * finaliser, 7 keypoints, 8 objective terms, 9 PCG/vector kernels, 10 other.
 * rg_profile_read synchronises on the recorded events, returns the summed
 * elapsed milliseconds and launch count of one id, and forgets them. */
int rg_profile(rg_ctx *ctx, int32_t enable);
int rg_profile_read(rg_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches);
/* Number of kernels this library has launched in the process so far. */
int64_t rg_launch_count(void);

/* Synchronise the context's stream and return the status its kernels
 * latched on the device since the last call: RG_ETIMEOUT if a kernel gave up
 * a bounded wait for a TMA transfer (its results are not valid), else
 * RG_ENONFINITE if an objective (ngf_objective, ngf_gradient, gn_linearize,
 * or a line-search evaluation) came out NaN, or +inf without a fold (non-finite
 * values in the images, keypoints or u), else RG_OK.  Clears the latches.
 * The asynchronous entry points return before their kernels run; this is where
 * their device-side failures surface. */
int rg_sync(rg_ctx *ctx);

/* Test hooks (no counterpart in the paper), for exercising the failure
 * paths without a GPU fault.  RG_HOOK_NO_TMA (value 0/1): the GN-product
 * kernels issue no TMA copy, so each of their bounded waits on a TMA barrier
 * runs out (the results are garbage and RG_ETIMEOUT is latched; no copy is
 * ever in flight).  RG_HOOK_POLL_LIMIT (value > 0): polls of a TMA barrier
 * before such a wait gives up (default 2^20).  RG_HOOK_PASS (value 0, 1, 2):
 * the objective / gradient / linearisation pass chosen by the volume's size
 * (0, the default: the column-marching pass when it has at least one column
 * of 60 x 16 voxels per SM), always the column-marching pass where it applies
 * (1), or always the tile pass (2); the results agree within rounding. */
#define RG_HOOK_NO_TMA 1
#define RG_HOOK_POLL_LIMIT 2
#define RG_HOOK_PASS 3
int rg_debug_hook(rg_ctx *ctx, int32_t what, int32_t value);

/* Latched error text of the last failing call on this context. */
const char *rg_last_error(const rg_ctx *ctx);
/* Library build/version string. */
const char *rg_version(void);

/* ------------------------------------------------------------------------
 * Discrete keypoint stage (Sec. II-C).  Images F (fixed) and M (moving) are
 * float32 [n[2]][n[1]][n[0]] at 1 mm isotropic spacing (Sec. II-C resamples
 * both scans to 1 mm^3); keypoints are int32 [nk][3] voxel positions
 * (x, y, z), 2 <= nk <= 65535.  Displacement labels: d = 2 (i - 16) mm per
 * axis, i = 0..32 (Sec. II-C2: {0, +-2, ..., +-32}^3 mm, 35 937 labels),
 * label index l = (i_z 33 + i_y) 33 + i_x.  Positions outside the volume read
 * the nearest voxel.  All pointers are device memory unless stated; calls are
 * asynchronous on cuda_stream except where they say they synchronise.
 * ------------------------------------------------------------------------ */
#define KP_LABELS 35937

typedef struct {
    double eta;           /* NGF edge parameter (Eq. 1, as used in Eq. 2) */
    double alpha;         /* alpha_KP of Eq. 3 */
    double sigma_i;       /* sigma_I of Eq. 3 (150 in the paper) */
} kp_params;

/* Workspace bytes of kp_match (two feature volumes of n voxels x 16 bytes,
 * four [nk][35937] float volumes, tree and MST scratch). */
int kp_workspace_size(const int32_t *n, int32_t nk, size_t *bytes);
/* Scratch bytes of kp_mst and kp_bp_marginals (one [nk][35937] message
 * volume plus tree and MST scratch). */
int kp_scratch_size(int32_t nk, size_t *bytes);

/* NGF features of Eq. 2: feat[z][y][x] = (grad I, eta) / ||(grad I, eta)||
 * as float4 (16-byte aligned), grad I by central differences over clamped
 * neighbours, so that the NGF cosine of two images is the dot product. */
int kp_ngf_features(const int32_t *n, const float *img, double eta, float *feat4, void *cuda_stream);

/* Eq. 2: D[k][l] = (1/64) sum_p (1 - (n_M(k + p + d_l) . n_F(k + p))^2) over
 * the 7^3 patch at stride 2 (p in {-3, -1, 1, 3}^3), float [nk][35937]. */
int kp_cost_volume(const int32_t *n, const float *feat_fixed, const float *feat_moving, int32_t nk,
                   const int32_t *kps, float *D, void *cuda_stream);

/* Minimum spanning tree over the keypoints with the edge weight of Eq. 3's
 * denominator, w = ||x_k - x_q|| + |I(k) - I(q)| / sigma_i (intensity: float
 * [nk]), evaluated in FP32 with each operation rounded once; ties broken by
 * (smaller index, larger index), so the tree is unique.  edges: int32
 * [nk - 1][2] (smaller, larger), sorted.  Synchronises the stream; RG_ECUDA
 * if the tree is incomplete. */
int kp_mst(int32_t nk, const int32_t *kps, const float *intensity, double sigma_i, int32_t *edges, void *scratch,
           size_t scratch_bytes, void *cuda_stream);

/* Exact min-marginals of sum_k D(k, d_k) + sum_edges alpha ||d_k - d_q||^2 /
 * w_kq (Eqs. 3-4) by two passes of min-sum belief propagation on the tree
 * rooted at its centre (the middle of a longest path, which minimises the
 * number of levels; exact min-marginals do not depend on the root); messages
 * are squared-distance min-convolutions over
 * the label grid (axis by axis).  marginals: float [nk][35937].
 * Synchronises the stream once (tree levels). */
int kp_bp_marginals(int32_t nk, const float *D, const int32_t *kps, const float *intensity, const int32_t *edges,
                    double sigma_i, double alpha, float *marginals, void *scratch, size_t scratch_bytes,
                    void *cuda_stream);

/* Sec. II-C2-4: features, cost volume, MST (intensities of F), marginals and
 * their argmin; symmetric != 0 adds the backward search from x_k + d*_k with
 * M fixed and F moving (intensities of M) and takes the argmin of
 * (E_fw(k, d) + E_bw(k, -d)) / 2 (lowest label among equal energies).
 * disp: int32 [nk][3] displacements in voxels (mm).  marginals: NULL, or
 * float [nk][35937] forward marginals followed (symmetric) by [nk][35937]
 * backward ones.  Synchronises the stream. */
int kp_match(const int32_t *n, const float *F, const float *M, int32_t nk, const int32_t *kps, const kp_params *p,
             int32_t symmetric, int32_t *disp, float *marginals, void *workspace, size_t ws_bytes,
             void *cuda_stream);

/* Keypoints of Sec. II-C1 (Foerstner operator) in the fixed image F:
 * F_D = 1 / trace((G_sigma * grad F grad F^T)^-1) in FP64 (central
 * differences, separable Gaussian with taps -5..5, weights exp(-i^2 /
 * (2 sigma^2)) normalised; nearest voxel outside the volume), F_D* its
 * maximum over the 6^3 window of offsets -3..2 per axis, keypoints = voxels
 * with mask != 0 (mask: uint8 [N], or NULL for all) and F_D = F_D* > 0, in
 * linear index order.  kps: int32 [max_kp][3] (x, y, z); *count (host) gets
 * the number found (only the first max_kp are written).  response: NULL or
 * double [N] for F_D.  Synchronises the stream. */
int kp_forstner_workspace_size(const int32_t *n, size_t *bytes);
int kp_forstner(const int32_t *n, const float *F, const uint8_t *mask, double sigma, int32_t max_kp, int32_t *kps,
                int32_t *count, double *response, void *workspace, size_t ws_bytes, void *cuda_stream);

/* Kernels launched by the kp_* entry points in this process so far. */
int64_t kp_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
