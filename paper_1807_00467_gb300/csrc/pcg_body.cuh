// Bodies of the reorthogonalised PCG's step, reorthogonalisation and
// direction kernels (pcg.cu), shared with the persistent batched PCG kernel
// (pcg_batch.cu); the partition and the reductions are described in pcg.cu.
#pragma once

#include "ngfreg.h"
#include "common.cuh"
#include "kernels.h"
#include "lastblock.cuh"
#include "vblock.cuh"

namespace ngf {
namespace pcgk {

constexpr int kVT = 512;            // threads per block (two blocks per SM at the full size)
constexpr int kVW = kVT / 32;
constexpr int kQmax = 6;            // quads per thread at most
constexpr int kHist = RG_PCG_MAX + 1;

__device__ __forceinline__ float dot4(float4 a, float4 b) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// Block sum of a per-thread value (FP32 within a warp, FP64 across warps);
// the result is valid in thread 0.
__device__ __forceinline__ double block_total(float v, double *red, const VBlock &b) {
    v = lb_warp_sum_f(v);
    if ((b.tid & 31) == 0) red[b.tid >> 5] = (double)v;
    b.sync();
    double t = 0.0;
    if (b.tid == 0)
        for (int i = 0; i < kVW; ++i) t += red[i];
    b.sync();
    return t;
}

// Sum of the partials part[0..n) of the previous kernel by the whole block in
// a fixed order (thread-strided, a fixed shuffle tree, the warps in order):
// the same value in every block, valid in every thread.
__device__ __forceinline__ double block_sum_parts(const double *part, int n, double *red, const VBlock &b) {
    double s = 0.0;
    for (int i = b.tid; i < n; i += kVT) s += __ldcg(part + i);
    s = lb_warp_sum(s);
    if ((b.tid & 31) == 0) red[b.tid >> 5] = s;
    b.sync();
    double t = 0.0;
    for (int w = 0; w < kVW; ++w) t += red[w];
    b.sync();
    return t;
}

struct Part {
    long n4;   // whole quads
    int tail;  // trailing floats (n % 4), handled by block 0
    int qpt;   // quads per thread
    __device__ __forceinline__ long quad(int i, const VBlock &b) const {
        return ((long)b.bid * qpt + i) * kVT + b.tid;
    }
};

__device__ __forceinline__ float4 ldg4(const float *p, long q) { return reinterpret_cast<const float4 *>(p)[q]; }
__device__ __forceinline__ void st4(float *p, long q, float4 v) { reinterpret_cast<float4 *>(p)[q] = v; }

// shared scratch of one block of the step, reorthogonalisation and direction bodies
struct PcgSmem {
    double wp[kHist][kVW];
    double red[kVW];
    float c[kHist];
};

// ---------------------------------------------------------------------------
// alpha = r.z / d.q (stop on a non-positive curvature d.q or a vanishing r.z);
// r_{k+1} = r_k - alpha q; then the partials of (M^-1 r_{k+1}) . r_j, j = 0..k
__device__ __forceinline__ void pcg_step_body(const Part &P, PcgScalars *sc, const double *apart, int napart,
                                              const float *q, const float *minv, float *Rh, long stride, int k,
                                              double *part, const VBlock &b, PcgSmem &sm) {
    double (&wp)[kHist][kVW] = sm.wp;
    double *red = sm.red;
    const int nb = b.nblk, lane = b.tid & 31, warp = b.tid >> 5;
    // every block forms the same alpha; a block that reads the stop flag block 0
    // has just set takes the same decision (the flag only ever turns on)
    const double pq = block_sum_parts(apart, napart, red, b);
    const int stop = (sc->stop || !(sc->rz != 0.0) || !(pq > 0.0)) ? 1 : 0;
    const double al64 = stop ? 0.0 : sc->rz / pq;
    if (b.bid == 0 && b.tid == 0) {
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
        const long e = P.quad(i, b);
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
    const bool tail = b.bid == 0 && b.tid < P.tail;
    const long et = 4 * P.n4 + b.tid;
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
            const long e = P.quad(i, b);
            if (i < P.qpt && e < P.n4) acc += dot4(zn[i], ldg4(rj, e));
        }
        if (tail) acc = fmaf(zt, rj[et], acc);
        acc = lb_warp_sum_f(acc);
        if (lane == 0) wp[j][warp] = (double)acc;
    }
    b.sync();
    for (int j = b.tid; j <= k; j += kVT) {
        double t = 0.0;
        for (int w = 0; w < kVW; ++w) t += wp[j][w];
        part[(long)j * nb + b.bid] = t;
    }
}

// ---------------------------------------------------------------------------
// c_j = (M^-1 r_{k+1}) . r_j / (r_j . z_j);  r_{k+1} -= sum_j c_j r_j;  then the
// partials of r.z with z = M^-1 r_{k+1}
__device__ __forceinline__ void pcg_reorth_body(const Part &P, const PcgScalars *sc, const float *minv, float *Rh,
                                                long stride, int k, const double *rzh, const double *cpart,
                                                double *rzpart, const VBlock &b, PcgSmem &sm) {
    float *c = sm.c;
    double *red = sm.red;
    const int nb = b.nblk, lane = b.tid & 31, warp = b.tid >> 5;
    float *r = Rh + (long)(k + 1) * stride;
    float4 rv[kQmax];
#pragma unroll
    for (int i = 0; i < kQmax; ++i) {
        const long e = P.quad(i, b);
        rv[i] = (i < P.qpt && e < P.n4) ? ldg4(r, e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool tail = b.bid == 0 && b.tid < P.tail;
    const long et = 4 * P.n4 + b.tid;
    float rt = tail ? r[et] : 0.f;
    // the coefficients, every block in the same order (one warp per coefficient)
    const bool stop = sc->stop != 0;
    for (int j = warp; j <= k; j += kVW) {
        const double v = lb_sum_parts(cpart + (long)j * nb, nb);
        if (lane == 0) c[j] = (stop || rzh[j] == 0.0) ? 0.f : (float)(v / rzh[j]);
    }
    b.sync();
#pragma unroll 2
    for (int j = k; j >= 0; --j) {
        const float *rj = Rh + (long)j * stride;
        const float cj = c[j];
#pragma unroll
        for (int i = 0; i < kQmax; ++i) {
            const long e = P.quad(i, b);
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
        const long e = P.quad(i, b);
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
    const double t = block_total(acc, red, b);
    if (b.tid == 0) rzpart[b.bid] = t;
}

// ---------------------------------------------------------------------------
// beta = r_{k+1}.z_{k+1} / r_k.z_k;  s += alpha d;  d = M^-1 r_{k+1} + beta d
__device__ __forceinline__ void pcg_dir_body(const Part &P, PcgScalars *sc, const float *minv, const float *r, float *d,
                                             float *s, int k, double *rzh, const double *rzpart, const VBlock &b,
                                             PcgSmem &sm) {
    double *red = sm.red;
    const double v = block_sum_parts(rzpart, b.nblk, red, b);
    // stop and alpha were set by the step kernel; rzh[k] = r_k . z_k while the
    // solve runs (block 0 appends rzh[k + 1], which no block reads here)
    const bool stop = sc->stop != 0;
    const double beta = stop ? 0.0 : v / rzh[k];
    const float al = (float)sc->alpha, be = (float)beta;
    if (b.bid == 0 && b.tid == 0) {
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
        const long e = P.quad(i, b);
        if (i < P.qpt && e < P.n4) {
            const float4 m = ldg4(minv, e), rv = ldg4(r, e), dv = ldg4(d, e), sv = ldg4(s, e);
            st4(s, e, make_float4(fmaf(al, dv.x, sv.x), fmaf(al, dv.y, sv.y), fmaf(al, dv.z, sv.z),
                                  fmaf(al, dv.w, sv.w)));
            st4(d, e, make_float4(fmaf(be, dv.x, m.x * rv.x), fmaf(be, dv.y, m.y * rv.y), fmaf(be, dv.z, m.z * rv.z),
                                  fmaf(be, dv.w, m.w * rv.w)));
        }
    }
    if (b.bid == 0 && b.tid < P.tail) {
        const long e = 4 * P.n4 + b.tid;
        const float dv = d[e];
        s[e] = fmaf(al, dv, s[e]);
        d[e] = fmaf(be, dv, minv[e] * r[e]);
    }
}

// The partition of a vector of n floats: *nb blocks of kVT threads.
inline Part make_part(long n, int *nb) {
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

}  // namespace pcgk
}  // namespace ngf
