// Device side of one Gauss-Newton iteration of the fixed schedule
// (Sec. II-D3): the slope g.p, the Armijo test of each line-search try and
// the iterate update run on the GPU, so an iteration needs no host
// synchronisation and its launches can be captured once and replayed.
//
// Every decision is taken as on the host: the slope is the same sequential
// FP64 sum of the same block partials, the Armijo bound is one fused
// multiply-add J0 + (c t) g.p on both sides (c t is exact: t = 2^-k), so the
// device-driven and host-driven loops give the same bits.
#include <math.h>

#include "kernels.h"
#include "ngfreg.h"

namespace ngf {

namespace {

// after the objective and gradient at the iterate: start the iteration, or
// stop the schedule on a non-finite objective (fold or NaN)
__global__ void gn_begin_kernel(GnState *s, const double *terms, const double *dminmax) {
    if (s->halted) {
        s->done = 1;
        return;
    }
    const double J0 = terms[4];
    s->J0 = J0;
    s->dmin = dminmax[0];   // the iterate's d range, kept if no step is accepted
    s->dmax = dminmax[1];
    s->Jn = J0;
    s->acc_t = 0.0;
    s->slope = 0.0;
    s->evals = 0;
    s->done = 0;
    if (!isfinite(J0)) {
        s->status = isinf(J0) ? RG_EFOLD : RG_ENONFINITE;
        s->halted = 1;
        s->halt_it = s->it;
        s->done = 1;   // no line-search try runs
    }
}

// slope g.p: the block partials summed in index order (as the host does)
__global__ void gn_slope_kernel(GnState *s, const double *part, int nparts) {
    double acc = 0.0;
    for (int i = 0; i < nparts; ++i) acc += part[i];
    s->slope = acc;
}

// one line-search try at step t: accept the first t with
// J(u + t p) <= J0 + c t g.p; later tries see done and skip all their work
__global__ void gn_armijo_kernel(GnState *s, const double *terms, const double *dminmax, double t, double c) {
    if (s->done) return;
    s->evals += 1;
    const double J = terms[4];
    if (isfinite(J) && J <= fma(c * t, s->slope, s->J0)) {
        s->done = 1;
        s->acc_t = t;
        s->Jn = J;
        s->dmin = dminmax[0];
        s->dmax = dminmax[1];
    }
}

// the d range of the iterate after the step, from a separate range pass (when
// the objective does not evaluate the volume term)
__global__ void gn_range_kernel(GnState *s, const double *dminmax) {
    if (s->halted) return;
    s->dmin = dminmax[0];
    s->dmax = dminmax[1];
}

// u = u + t p (the accepted try's iterate) when a step was accepted
__global__ void gn_accept_kernel(const GnState *s, long n, const float *tu, float *u) {
    if (!(s->acc_t > 0.0)) return;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) u[i] = tu[i];
}

// report row {it, J, g.p, t, J new, evaluations, pcg steps, status, min d, max d, in bounds}
__global__ void gn_report_kernel(GnState *s, const double *pcg_stats, double *rep, int rows, double det_lo,
                                 double det_hi) {
    const int it = s->it;
    if (it < rows) {
        double *r = rep + RG_REPORT_COLS * (long)it;
        if (s->halted && s->halt_it == it) {
            for (int k = 0; k < RG_REPORT_COLS; ++k) r[k] = 0.0;
            r[0] = it; r[1] = s->J0; r[7] = s->status;
        } else if (!s->halted) {
            r[0] = it; r[1] = s->J0; r[2] = s->slope; r[3] = s->acc_t; r[4] = s->Jn; r[5] = s->evals;
            r[6] = pcg_stats[0]; r[7] = 0.0;
            r[8] = s->dmin; r[9] = s->dmax; r[10] = (s->dmin >= det_lo && s->dmax <= det_hi) ? 1.0 : 0.0;
        }
    }
    s->it = it + 1;
}

}  // namespace

cudaError_t launch_gn_begin(GnState *s, const double *terms, const double *dminmax, cudaStream_t st) {
    gn_begin_kernel<<<1, 1, 0, st>>>(s, terms, dminmax);
    return cudaGetLastError();
}
cudaError_t launch_gn_slope(GnState *s, const double *part, int nparts, cudaStream_t st) {
    gn_slope_kernel<<<1, 1, 0, st>>>(s, part, nparts);
    return cudaGetLastError();
}
cudaError_t launch_gn_armijo(GnState *s, const double *terms, const double *dminmax, double t, double c,
                             cudaStream_t st) {
    gn_armijo_kernel<<<1, 1, 0, st>>>(s, terms, dminmax, t, c);
    return cudaGetLastError();
}
cudaError_t launch_gn_accept(const GnState *s, long n, const float *tu, float *u, cudaStream_t st) {
    gn_accept_kernel<<<vec_blocks(n), 256, 0, st>>>(s, n, tu, u);
    return cudaGetLastError();
}
cudaError_t launch_gn_range(GnState *s, const double *dminmax, cudaStream_t st) {
    gn_range_kernel<<<1, 1, 0, st>>>(s, dminmax);
    return cudaGetLastError();
}
cudaError_t launch_gn_report(GnState *s, const double *pcg_stats, double *rep, int rows, double det_lo, double det_hi,
                             cudaStream_t st) {
    gn_report_kernel<<<1, 1, 0, st>>>(s, pcg_stats, rep, rows, det_lo, det_hi);
    return cudaGetLastError();
}

}  // namespace ngf
