// Vector kernels of the reorthogonalised PCG (Sec. II-D: the Gauss-Newton
// system is solved by preconditioned conjugate gradients).
//
// Every kernel streams the node vectors as float4 with the same partition:
// block b owns quads [b Q, (b + 1) Q), Q = kVT qpt, thread t its quads
// b Q + i kVT + t (i < qpt <= kQmax), so each thread keeps up to kQmax
// independent 16-byte loads in flight per stream.  Sums are FP32 within a
// warp and FP64 across warps and blocks.  A kernel publishes one FP64 partial
// per block and sum; the blocks of the NEXT kernel each reduce those partials
// in the same fixed order, so every block derives the same scalar (block 0
// records it in the device scalars), no block waits for another and no kernel
// ends in a serial reduction.  One PCG step k, after q = H d:
//   step:   alpha = r_k . z_k / d . q;  r' = r_k - alpha q;  partials of
//           (M^-1 r') . r_j, j = 0..k (the classical Gram-Schmidt coefficients)
//   reorth: c_j = (M^-1 r') . r_j / (r_j . z_j);  r_{k+1} = r' - sum_j c_j r_j,
//           the history read newest first (the step kernel has just streamed
//           it oldest first, so its newest slots are still in L2);  partials of
//           r_{k+1} . z_{k+1}
//   dir:    beta = r_{k+1} . z_{k+1} / r_k . z_k;  s += alpha d;  d = z_{k+1} + beta d
// The d . q partials come from the node pass that forms q (no later pass adds
// to it) or from pcg_alpha_kernel.
//
// The preconditioner is diagonal, so z_j = M^-1 r_j is not stored: the
// Gram-Schmidt coefficients use r . z_j = (M^-1 r) . r_j.
#include "pcg_body.cuh"

namespace ngf {

namespace {

using namespace pcgk;

// ---------------------------------------------------------------------------
// start: s = 0, r_0 = -g, d = z_0 = M^-1 r_0; scalars reset, |g|, r_0 . z_0
__global__ void __launch_bounds__(kVT, 2) pcg_start_kernel(Part P, const float *g, const float *minv, float *s, float *r,
                                                        float *d, double *part, unsigned *ticket, PcgScalars *sc,
                                                        double *rzh) {
    __shared__ double red[kVW];
    const VBlock b = cuda_block_1d();
    const int nb = gridDim.x;
    float gg = 0.f, rz = 0.f;
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long q = P.quad(i, b);
        if (i < P.qpt && q < P.n4) {
            const float4 gv = ldg4(g, q), m = ldg4(minv, q);
            const float4 rv = make_float4(-gv.x, -gv.y, -gv.z, -gv.w);
            const float4 zv = make_float4(m.x * rv.x, m.y * rv.y, m.z * rv.z, m.w * rv.w);
            st4(s, q, make_float4(0.f, 0.f, 0.f, 0.f));
            st4(r, q, rv);
            st4(d, q, zv);
            gg += dot4(gv, gv);
            rz += dot4(rv, zv);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < P.tail) {
        const long e = 4 * P.n4 + threadIdx.x;
        const float rv = -g[e], zv = minv[e] * rv;
        s[e] = 0.f; r[e] = rv; d[e] = zv;
        gg = fmaf(rv, rv, gg);
        rz = fmaf(rv, zv, rz);
    }
    const double tg = block_total(gg, red, b);
    const double tr = block_total(rz, red, b);
    if (threadIdx.x == 0) { part[blockIdx.x] = tg; part[nb + blockIdx.x] = tr; }
    if (!lb_last_block(ticket, gridDim.x)) return;
    if (threadIdx.x < 64) {
        const double v = lb_sum_parts(part + (threadIdx.x >> 5) * nb, nb);
        if (threadIdx.x == 0) {
            sc->pq = sc->alpha = sc->beta = sc->rend = sc->rz_new = 0.0;
            sc->stop = 0;
            sc->steps = 0;
            sc->r0 = sqrt(v);
        }
        if (threadIdx.x == 32) {
            sc->rz = v;
            rzh[0] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// partials of d . q (when a pass after the node pass still adds to q)
__global__ void __launch_bounds__(kVT, 2) pcg_alpha_kernel(Part P, const float *d, const float *q, double *apart) {
    __shared__ double red[kVW];
    const VBlock b = cuda_block_1d();
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long k = P.quad(i, b);
        if (i < P.qpt && k < P.n4) acc += dot4(ldg4(d, k), ldg4(q, k));
    }
    if (blockIdx.x == 0 && threadIdx.x < P.tail) {
        const long e = 4 * P.n4 + threadIdx.x;
        acc = fmaf(d[e], q[e], acc);
    }
    const double t = block_total(acc, red, b);
    if (threadIdx.x == 0) apart[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// step, reorthogonalisation and direction: the bodies of pcg_body.cuh
__global__ void __launch_bounds__(kVT, 2) pcg_step_kernel(Part P, PcgScalars *sc, const double *apart, int napart,
                                                       const float *q, const float *minv, float *Rh, long stride,
                                                       int k, double *part) {
    __shared__ PcgSmem sm;
    pcg_step_body(P, sc, apart, napart, q, minv, Rh, stride, k, part, cuda_block_1d(), sm);
}

__global__ void __launch_bounds__(kVT, 2) pcg_reorth_kernel(Part P, const PcgScalars *sc, const float *minv, float *Rh,
                                                         long stride, int k, const double *rzh, const double *cpart,
                                                         double *rzpart) {
    __shared__ PcgSmem sm;
    pcg_reorth_body(P, sc, minv, Rh, stride, k, rzh, cpart, rzpart, cuda_block_1d(), sm);
}

__global__ void __launch_bounds__(kVT, 2) pcg_dir_kernel(Part P, PcgScalars *sc, const float *minv, const float *r,
                                                      float *d, float *s, int k, double *rzh, const double *rzpart) {
    __shared__ PcgSmem sm;
    pcg_dir_body(P, sc, minv, r, d, s, k, rzh, rzpart, cuda_block_1d(), sm);
}

}  // namespace

int pcg_blocks(long n) {
    int nb;
    make_part(n, &nb);
    return nb;
}

long pcg_stride(long n) { return (n + 63) / 64 * 64; }

cudaError_t launch_pcg_start(const PcgArgs &a, const float *g, float *s, cudaStream_t st) {
    int nb;
    const Part P = make_part(a.n, &nb);
    pcg_start_kernel<<<nb, kVT, 0, st>>>(P, g, a.minv, s, a.Rh, a.d, a.part, a.ticket, a.sc, a.rzh);
    return cudaGetLastError();
}

cudaError_t launch_pcg_alpha(const PcgArgs &a, const float *q, int *napart, cudaStream_t st) {
    int nb;
    const Part P = make_part(a.n, &nb);
    pcg_alpha_kernel<<<nb, kVT, 0, st>>>(P, a.d, q, a.apart);
    *napart = nb;
    return cudaGetLastError();
}

cudaError_t launch_pcg_step(const PcgArgs &a, const float *q, int napart, int k, cudaStream_t st) {
    if (k < 0 || k + 1 >= kHist || napart < 1) return cudaErrorInvalidValue;
    int nb;
    const Part P = make_part(a.n, &nb);
    pcg_step_kernel<<<nb, kVT, 0, st>>>(P, a.sc, a.apart, napart, q, a.minv, a.Rh, a.stride, k, a.part);
    return cudaGetLastError();
}

cudaError_t launch_pcg_reorth(const PcgArgs &a, int k, cudaStream_t st) {
    if (k < 0 || k + 1 >= kHist) return cudaErrorInvalidValue;
    int nb;
    const Part P = make_part(a.n, &nb);
    pcg_reorth_kernel<<<nb, kVT, 0, st>>>(P, a.sc, a.minv, a.Rh, a.stride, k, a.rzh, a.part, a.rzpart);
    return cudaGetLastError();
}

cudaError_t launch_pcg_dir(const PcgArgs &a, float *s, int k, cudaStream_t st) {
    int nb;
    const Part P = make_part(a.n, &nb);
    pcg_dir_kernel<<<nb, kVT, 0, st>>>(P, a.sc, a.minv, a.Rh + (long)(k + 1) * a.stride, a.d, s, k, a.rzh,
                                       a.rzpart);
    return cudaGetLastError();
}

}  // namespace ngf
