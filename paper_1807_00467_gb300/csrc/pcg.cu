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
#include "ngfreg.h"
#include "common.cuh"
#include "kernels.h"
#include "lastblock.cuh"

namespace ngf {

namespace {

constexpr int kVT = 512;            // threads per block (two blocks per SM at the full size)
constexpr int kVW = kVT / 32;
constexpr int kQmax = 6;            // quads per thread at most
constexpr int kHist = RG_PCG_MAX + 1;

__device__ __forceinline__ float dot4(float4 a, float4 b) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// Block sum of a per-thread value (FP32 within a warp, FP64 across warps);
// the result is valid in thread 0.
__device__ __forceinline__ double block_total(float v, double *red) {
    v = lb_warp_sum_f(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kVW; ++i) t += red[i];
    __syncthreads();
    return t;
}

// Sum of the partials part[0..n) of the previous kernel by the whole block in
// a fixed order (thread-strided, a fixed shuffle tree, the warps in order):
// the same value in every block, valid in every thread.
__device__ __forceinline__ double block_sum_parts(const double *part, int n, double *red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kVT) s += __ldcg(part + i);
    s = lb_warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kVW; ++w) t += red[w];
    __syncthreads();
    return t;
}

struct Part {
    long n4;   // whole quads
    int tail;  // trailing floats (n % 4), handled by block 0
    int qpt;   // quads per thread
    __device__ __forceinline__ long quad(int i) const {
        return ((long)blockIdx.x * qpt + i) * kVT + threadIdx.x;
    }
};

__device__ __forceinline__ float4 ldg4(const float *p, long q) { return reinterpret_cast<const float4 *>(p)[q]; }
__device__ __forceinline__ void st4(float *p, long q, float4 v) { reinterpret_cast<float4 *>(p)[q] = v; }

// ---------------------------------------------------------------------------
// start: s = 0, r_0 = -g, d = z_0 = M^-1 r_0; scalars reset, |g|, r_0 . z_0
__global__ void __launch_bounds__(kVT, 2) pcg_start_kernel(Part P, const float *g, const float *minv, float *s, float *r,
                                                        float *d, double *part, unsigned *ticket, PcgScalars *sc,
                                                        double *rzh) {
    __shared__ double red[kVW];
    const int nb = gridDim.x;
    float gg = 0.f, rz = 0.f;
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long q = P.quad(i);
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
    const double tg = block_total(gg, red);
    const double tr = block_total(rz, red);
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
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long k = P.quad(i);
        if (i < P.qpt && k < P.n4) acc += dot4(ldg4(d, k), ldg4(q, k));
    }
    if (blockIdx.x == 0 && threadIdx.x < P.tail) {
        const long e = 4 * P.n4 + threadIdx.x;
        acc = fmaf(d[e], q[e], acc);
    }
    const double t = block_total(acc, red);
    if (threadIdx.x == 0) apart[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// alpha = r.z / d.q (stop on a non-positive curvature d.q or a vanishing r.z);
// r_{k+1} = r_k - alpha q; then the partials of (M^-1 r_{k+1}) . r_j, j = 0..k
__global__ void __launch_bounds__(kVT, 2) pcg_step_kernel(Part P, PcgScalars *sc, const double *apart, int napart,
                                                       const float *q, const float *minv, float *Rh, long stride,
                                                       int k, double *part) {
    __shared__ double wp[kHist][kVW];
    __shared__ double red[kVW];
    const int nb = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // every block forms the same alpha; a block that reads the stop flag block 0
    // has just set takes the same decision (the flag only ever turns on)
    const double pq = block_sum_parts(apart, napart, red);
    const int stop = (sc->stop || !(sc->rz != 0.0) || !(pq > 0.0)) ? 1 : 0;
    const double al64 = stop ? 0.0 : sc->rz / pq;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->pq = pq;
        sc->stop = stop;
        sc->alpha = al64;
    }
    const float al = (float)al64;
    const float *r = Rh + (long)k * stride;
    float *rn = Rh + (long)(k + 1) * stride;
    float4 zn[kQmax];
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long e = P.quad(i);
        zn[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < P.qpt && e < P.n4) {
            const float4 qv = ldg4(q, e), rv = ldg4(r, e), m = ldg4(minv, e);
            const float4 nv = make_float4(fmaf(-al, qv.x, rv.x), fmaf(-al, qv.y, rv.y), fmaf(-al, qv.z, rv.z),
                                          fmaf(-al, qv.w, rv.w));
            st4(rn, e, nv);
            zn[i] = make_float4(m.x * nv.x, m.y * nv.y, m.z * nv.z, m.w * nv.w);
        }
    }
    float zt = 0.f;
    const bool tail = blockIdx.x == 0 && threadIdx.x < P.tail;
    const long et = 4 * P.n4 + threadIdx.x;
    if (tail) {
        const float nv = fmaf(-al, q[et], r[et]);
        rn[et] = nv;
        zt = minv[et] * nv;
    }
#pragma unroll 1
    for (int j = 0; j <= k; ++j) {
        const float *rj = Rh + (long)j * stride;
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < kQmax; ++i) {
            const long e = P.quad(i);
            if (i < P.qpt && e < P.n4) acc += dot4(zn[i], ldg4(rj, e));
        }
        if (tail) acc = fmaf(zt, rj[et], acc);
        acc = lb_warp_sum_f(acc);
        if (lane == 0) wp[j][warp] = (double)acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= k; j += kVT) {
        double t = 0.0;
        for (int w = 0; w < kVW; ++w) t += wp[j][w];
        part[(long)j * nb + blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// c_j = (M^-1 r_{k+1}) . r_j / (r_j . z_j);  r_{k+1} -= sum_j c_j r_j;  then the
// partials of r.z with z = M^-1 r_{k+1}
__global__ void __launch_bounds__(kVT, 2) pcg_reorth_kernel(Part P, const PcgScalars *sc, const float *minv, float *Rh,
                                                         long stride, int k, const double *rzh, const double *cpart,
                                                         double *rzpart) {
    __shared__ float c[kHist];
    __shared__ double red[kVW];
    const int nb = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *r = Rh + (long)(k + 1) * stride;
    float4 rv[kQmax];
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long e = P.quad(i);
        rv[i] = (i < P.qpt && e < P.n4) ? ldg4(r, e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool tail = blockIdx.x == 0 && threadIdx.x < P.tail;
    const long et = 4 * P.n4 + threadIdx.x;
    float rt = tail ? r[et] : 0.f;
    // the coefficients, every block in the same order (one warp per coefficient)
    const bool stop = sc->stop != 0;
    for (int j = warp; j <= k; j += kVW) {
        const double v = lb_sum_parts(cpart + (long)j * nb, nb);
        if (lane == 0) c[j] = (stop || rzh[j] == 0.0) ? 0.f : (float)(v / rzh[j]);
    }
    __syncthreads();
#pragma unroll 2
    for (int j = k; j >= 0; --j) {
        const float *rj = Rh + (long)j * stride;
        const float cj = c[j];
#pragma unroll
        for (int i = 0; i < kQmax; ++i) {
            const long e = P.quad(i);
            if (i < P.qpt && e < P.n4) {
                const float4 x = ldg4(rj, e);
                rv[i].x = fmaf(-cj, x.x, rv[i].x); rv[i].y = fmaf(-cj, x.y, rv[i].y);
                rv[i].z = fmaf(-cj, x.z, rv[i].z); rv[i].w = fmaf(-cj, x.w, rv[i].w);
            }
        }
        if (tail) rt = fmaf(-cj, rj[et], rt);
    }
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long e = P.quad(i);
        if (i < P.qpt && e < P.n4) {
            const float4 m = ldg4(minv, e);
            st4(r, e, rv[i]);
            acc += dot4(rv[i], make_float4(m.x * rv[i].x, m.y * rv[i].y, m.z * rv[i].z, m.w * rv[i].w));
        }
    }
    if (tail) {
        r[et] = rt;
        acc = fmaf(rt, minv[et] * rt, acc);
    }
    const double t = block_total(acc, red);
    if (threadIdx.x == 0) rzpart[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// beta = r_{k+1}.z_{k+1} / r_k.z_k;  s += alpha d;  d = M^-1 r_{k+1} + beta d
__global__ void __launch_bounds__(kVT, 2) pcg_dir_kernel(Part P, PcgScalars *sc, const float *minv, const float *r,
                                                      float *d, float *s, int k, double *rzh, const double *rzpart) {
    __shared__ double red[kVW];
    const double v = block_sum_parts(rzpart, gridDim.x, red);
    // stop and alpha were set by the step kernel; rzh[k] = r_k . z_k while the
    // solve runs (block 0 appends rzh[k + 1], which no block reads here)
    const bool stop = sc->stop != 0;
    const double beta = stop ? 0.0 : v / rzh[k];
    const float al = (float)sc->alpha, be = (float)beta;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rz_new = v;
        sc->beta = beta;
        if (!stop) {
            sc->rz = v;
            sc->steps += 1;
            rzh[sc->steps] = v;
        }
    }
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long e = P.quad(i);
        if (i < P.qpt && e < P.n4) {
            const float4 m = ldg4(minv, e), rv = ldg4(r, e), dv = ldg4(d, e), sv = ldg4(s, e);
            st4(s, e, make_float4(fmaf(al, dv.x, sv.x), fmaf(al, dv.y, sv.y), fmaf(al, dv.z, sv.z),
                                  fmaf(al, dv.w, sv.w)));
            st4(d, e, make_float4(fmaf(be, dv.x, m.x * rv.x), fmaf(be, dv.y, m.y * rv.y), fmaf(be, dv.z, m.z * rv.z),
                                  fmaf(be, dv.w, m.w * rv.w)));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < P.tail) {
        const long e = 4 * P.n4 + threadIdx.x;
        const float dv = d[e];
        s[e] = fmaf(al, dv, s[e]);
        d[e] = fmaf(be, dv, minv[e] * r[e]);
    }
}

Part make_part(long n, int *nb) {
    Part P;
    P.n4 = n / 4;
    P.tail = (int)(n % 4);
    // two blocks per SM while that keeps at most kQmax quads per thread (more
    // waves beyond); short vectors take fewer blocks of one quad per thread
    const long fill = 2L * 152 * kVT;
    long blocks;
    if (P.n4 <= fill) blocks = P.n4 > 0 ? (P.n4 + kVT - 1) / kVT : 1;
    else blocks = 2L * 152 * ((P.n4 + fill * kQmax - 1) / (fill * kQmax));
    *nb = (int)blocks;
    P.qpt = (int)((P.n4 + blocks * kVT - 1) / (blocks * kVT));
    if (P.qpt < 1) P.qpt = 1;
    return P;
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
