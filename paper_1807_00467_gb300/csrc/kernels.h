// Kernel launchers of the ngfreg library (internal).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ngf {

enum TileMode { MODE_OBJ = 0, MODE_LIN = 1, MODE_GRAD = 2, MODE_GRADLIN = 3, MODE_MATVEC = 4, MODE_DIAG = 5 };

size_t tile_smem_bytes(const TileGeom &g, int mode);
cudaError_t launch_ngf_tile(int mode, const TileArgs<float> &a, cudaStream_t st);
cudaError_t launch_ngf_tile(int mode, const TileArgs<__half> &a, cudaStream_t st);
// Dedicated GN-product kernel (stored linearisation streamed by TMA); same
// tile and node-box layout as MODE_MATVEC (diag: MODE_DIAG) of the general kernel.
bool gn_matvec_supported(const TileGeom &g);
// Objective / gradient / linearisation pass (MODE_OBJ, MODE_GRAD, MODE_GRADLIN,
// MODE_LIN as GRADLIN) on persistent CTAs; same tile and node-box layout.
bool ngf_grad_supported(const TileGeom &g);
cudaError_t launch_ngf_grad(int mode, const TileArgs<float> &a, cudaStream_t st);
cudaError_t launch_ngf_grad(int mode, const TileArgs<__half> &a, cudaStream_t st);
cudaError_t launch_gn_matvec(const TileArgs<float> &a, bool diag, cudaStream_t st);
// Column-marching GN product / diagonal (packed FP32, two x columns per lane).
bool gn_product_supported(const ColGeom &g);
cudaError_t launch_gn_product(const ColArgs &a, bool diag, cudaStream_t st);

// Column-marching objective / gradient / linearisation pass (ngf_gcol.cu):
// MODE_OBJ, MODE_GRAD, MODE_GRADLIN (MODE_LIN as GRADLIN); node boxes in the
// GN product's column layout, one D partial per column.
template <typename TImg>
struct GcolArgs {
    ColGeom g;
    float invh[3];          // float(1 / h), the FP32 cell decision
    float invh_rel[3];      // 1 - h float(1 / h)
    float eta2;
    const TImg *R, *T;
    const float *u;
    float *st_dT, *st_a;    // stored linearisation (GRADLIN)
    float *boxes;           // per-column node boxes [column][3][m3][C1 + 1][C0 + 1]
    double *dpart;          // per-column partial sums of 1 - r^2
    const int *skip = nullptr;
};
bool ngf_gcol_supported(const ColGeom &g);
cudaError_t launch_ngf_gcol(int mode, const GcolArgs<float> &a, cudaStream_t st);
cudaError_t launch_ngf_gcol(int mode, const GcolArgs<__half> &a, cudaStream_t st);

// Volume change control, Eqs. (7)-(9): per grid cell the 64 bounds d_abc.
struct VccArgs {
    int m[3];
    float ig[3];           // 1 / g_a
    int nb[3];             // cell tiles per axis
    int box;               // nodes per box
    const float *u;        // linearisation point [3][M]
    const float *v;        // direction for the GN product (NULL: gradient)
    int diag;              // 1: diagonal of the GN matrix instead
    float wscale;          // multiplies the node contributions (e.g. gamma * ghat)
    float *boxes;          // per-CTA node boxes [cta][3][box]
    double *epart;         // per-CTA partial sums of psi(d)
    int *fold;             // per-CTA count of d <= 0
    float *dmin, *dmax;    // per-CTA min / max of d
    const int *skip = nullptr;   // nonzero: the launch does nothing
};
constexpr int kVccTile[3] = {8, 4, 4};
cudaError_t launch_vcc(const VccArgs &a, cudaStream_t st);
cudaError_t launch_vcc_cells(const VccArgs &a, cudaStream_t st);   // gradient / GN product / diagonal

// Node passes: w = L v with the curvature operator L of Eq. (5) and
// per-block partials of |L v|^2 (launch_curv); out = sA (NGF boxes) +
// sB (VCC boxes) + sC L^T w (launch_nodes).
struct NodeArgs {
    int m[3];
    float ig2[3];          // 1 / g_a^2
    const float *boxA; BoxGeom gA; float sA;   // NGF boxes (scale hbar), may be NULL
    const float *boxB; BoxGeom gB; float sB;   // VCC boxes (scale gamma ghat), may be NULL
    const float *v;        // curvature input [3][M] (launch_curv)
    float *w;              // L v [3][M]: written by launch_curv, read by launch_nodes (may be NULL there)
    float sC;              // scale of L^T w (alpha ghat)
    double *rpart;         // per-block partial sums of |L v|^2, may be NULL
    float *out;            // [3][M] (launch_nodes)
    const float *dvec = nullptr;   // with dpart: per-block partials of dvec . out (launch_nodes)
    double *dpart = nullptr;
    const int *skip = nullptr;   // nonzero: the launch does nothing
};
int node_blocks(const int *m);
cudaError_t launch_curv(const NodeArgs &a, cudaStream_t st);
cudaError_t launch_nodes(const NodeArgs &a, cudaStream_t st);

// Keypoint penalty, Eq. (10).
// The keypoint index (launch_kp_index, once per set of keypoints): every
// keypoint's cell (linear index of its lowest node) and fractions, the
// keypoints sorted by (cell, keypoint index), and for every cell the sorted
// position of its first keypoint (-1: none).  The node sums gather through it
// without atomics.
struct KpIndex {
    int *cell;             // [nk]
    float *frac;           // [nk][3]
    int *sb, *perm;        // [nk]: sorted cells, keypoint at each sorted position
    int *soc;              // [M]: first sorted position of each cell, -1 if none
    float *src;            // [nk][3]: per-call scratch (res_i, or (P v)(x_i))
};
struct KpArgs {
    int m[3];
    float ig[3];           // 1 / g_a
    int nk;
    const float *kx, *ky;  // [nk][3]
    const float *u;        // [3][M]
    const float *v;        // NULL: gradient 2 P^T res; else 2 P^T P v
    float scale;           // multiplies the node contributions (delta)
    float *out;            // the node contributions are added to it (NULL: energy only)
    double *part;          // per-CTA partial sums of |res|^2
    KpIndex ix;
    const int *skip = nullptr;   // nonzero: the launch does nothing
};
int kp_blocks(int nk);
// index steps 0 (cells and fractions), 1 (ranks), 2 (first rank per cell)
cudaError_t launch_kp_index(const KpArgs &a, int step, cudaStream_t st);
cudaError_t launch_kp(const KpArgs &a, cudaStream_t st);          // residuals, energy, sources
cudaError_t launch_kp_gather(const KpArgs &a, cudaStream_t st);   // node sums into a.out

// Objective terms {D, R, V, K, J} from the partial sums.
struct TermsArgs {
    const double *dpart; int nd; double dscale;
    const double *rpart; int nr; double rscale;
    const double *vpart; int nv; double vscale; const int *fold;
    const double *kpart; int nkp;
    double alpha, gamma, delta;
    const float *dmin, *dmax; double *dminmax;
    double *terms;         // [5]
    const int *skip = nullptr;   // nonzero: the launch does nothing
    int *nonfinite = nullptr;    // set to 1 when J is NaN, or +inf without a fold
};
cudaError_t launch_terms(const TermsArgs &a, cudaStream_t st);

// PCG vector kernels (device-resident FP64 scalars).
struct PcgScalars {
    double rz, rz_new, pq, alpha, beta, r0, rend;
    int stop, steps;
};
int vec_blocks(long n);
cudaError_t launch_jacobi_diag(int alpha_on, const int *m, const float *ig2, double alpha_ghat, double tau,
                               float *minv, cudaStream_t st);
cudaError_t launch_kp_diag(const KpArgs &a, double two_delta, float *diag, cudaStream_t st);
cudaError_t launch_invert(long n, float *d, cudaStream_t st);
cudaError_t launch_dot(long n, const float *x, const float *y, double *part, cudaStream_t st);
cudaError_t launch_pcg_scalar(int which, const double *part, int nparts, PcgScalars *sc, cudaStream_t st,
                              double *rzh = nullptr);
cudaError_t launch_dot_slot(long n, const float *Rh, long stride, const PcgScalars *sc, double *part,
                            cudaStream_t st);

// Reorthogonalised PCG (float4 streams; FP64 per-block partials that the
// blocks of the next kernel reduce in a fixed order).  Residual history
// r_0..r_k in slots of `stride` floats.
struct PcgArgs {
    long n, stride;        // vector length, history slot stride (pcg_stride(n))
    const float *minv;     // inverse preconditioner diagonal
    float *Rh;             // residual history
    float *d;              // search direction
    double *part;          // Gram-Schmidt coefficient partials: (pcg_max + 2) x pcg_blocks(n)
    double *rzpart;        // r.z partials of the reorthogonalised residual: pcg_blocks(n)
    double *apart;         // d.q partials: max(pcg_blocks(n), node_blocks(m))
    unsigned *ticket;      // last-block ticket of the start kernel (zero between launches)
    PcgScalars *sc;
    double *rzh;           // r_j . z_j
};
int pcg_blocks(long n);
long pcg_stride(long n);
cudaError_t launch_pcg_start(const PcgArgs &a, const float *g, float *s, cudaStream_t st);
// d.q partials into a.apart (their count into *napart)
cudaError_t launch_pcg_alpha(const PcgArgs &a, const float *q, int *napart, cudaStream_t st);
// napart: the d.q partials in a.apart (from launch_pcg_alpha or the node pass)
cudaError_t launch_pcg_step(const PcgArgs &a, const float *q, int napart, int k, cudaStream_t st);
cudaError_t launch_pcg_reorth(const PcgArgs &a, int k, cudaStream_t st);
cudaError_t launch_pcg_dir(const PcgArgs &a, float *s, int k, cudaStream_t st);
cudaError_t launch_axpy_copy(long n, float t, const float *x, const float *p, float *y, cudaStream_t st,
                             const int *skip = nullptr);

// Device side of one Gauss-Newton iteration (line search without host reads).
struct GnState {
    double J0, Jn, slope, acc_t;
    double dmin, dmax;   // extremes of the Jacobian bounds d at the iterate after the step
    int done;      // the line search has finished (or the schedule halted): later tries skip
    int evals;     // objective evaluations of the line search
    int halted;    // a non-finite objective stopped the schedule
    int halt_it;   // ... at this iteration
    int status;    // RG_OK, RG_EFOLD or RG_ENONFINITE
    int it;        // iterations run (report row index)
};
constexpr int kGnRows = 256;   // report rows the workspace keeps for device-driven schedules
// dminmax: the {min d, max d} the objective's terms kernel wrote for the same evaluation
cudaError_t launch_gn_begin(GnState *s, const double *terms, const double *dminmax, cudaStream_t st);
cudaError_t launch_gn_slope(GnState *s, const double *part, int nparts, cudaStream_t st);
cudaError_t launch_gn_armijo(GnState *s, const double *terms, const double *dminmax, double t, double c,
                             cudaStream_t st);
cudaError_t launch_gn_accept(const GnState *s, long n, const float *tu, float *u, cudaStream_t st);
cudaError_t launch_gn_range(GnState *s, const double *dminmax, cudaStream_t st);   // d range at the new iterate
cudaError_t launch_gn_report(GnState *s, const double *pcg_stats, double *rep, int rows, double det_lo, double det_hi,
                             cudaStream_t st);

// Persistent batched PCG (pcg_batch.cu): the PCG steps of several volumes'
// Gauss-Newton systems in one cooperative launch.  Per volume the operands of
// one reorthogonalised PCG step after launch_pcg_start: the GN product of the
// NGF term (column kernel, v = the search direction), the VCC product, the
// curvature and node passes (out = q, d . q partials) and the vector state.
struct BatchPair {
    ColArgs col;           // GN product: v = d, boxes; its err flag also reports a barrier that gave up
    VccArgs vcc;           // VCC product (u = linearisation point, v = d), used when vcc_on
    NodeArgs nodes;        // curvature (v = d, w) and node pass (out = q, dpart = d . q partials)
    PcgArgs pcg;           // vectors and device scalars
    float *s;              // the solution (PCG iterate)
    int vcc_on;
};
constexpr int kBatchMax = 24;   // volumes per launch (the descriptors travel as kernel parameters)
// control words of one launch, zeroed before it: the work counter, the abort
// flag and per volume one completion counter per phase, each group on a
// 128-byte line of its own
constexpr size_t kBatchCtlWords = 64 + 32 * (size_t)kBatchMax;
bool pcg_batch_supported(const ColGeom &g);
// hook_skip: test hook, the first item's completion is withheld (the waits on
// it run out; RG_ETIMEOUT)
cudaError_t launch_pcg_batch(const BatchPair *pairs, int npairs, int iters, unsigned *ctl, int poll_limit,
                             int hook_skip, cudaStream_t st);

// Pyramid.
cudaError_t launch_restrict(const int *n, bool half, const void *in, void *out, cudaStream_t st);
cudaError_t launch_prolong_grid(const int *mc, const float *uc, float *uf, cudaStream_t st);
cudaError_t launch_inject_grid(const int *mf, int step, const float *uf, const int *mc, float *uc, cudaStream_t st);

}  // namespace ngf
