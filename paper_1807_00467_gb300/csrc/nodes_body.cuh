// Bodies of the node passes (nodes.cu), shared with the persistent batched
// PCG kernel (pcg_batch.cu).
//
// curv_body: w = L v per node and per-block partial sums of |L v|^2 (the
// curvature energy of Eq. (5)); L is the sum over axes of the nodal 3-point
// second differences at nodes interior to that axis, scaled by 1/g_a^2.
//
// node_body: per grid node k,
//   out_k = sA (sum of the NGF node boxes holding k) + sB (sum of the VCC node
//           boxes holding k) + sC (L^T w)_k,
// optionally with per-block partials of d . out (the PCG step length).
// The boxes holding a node come from per-axis lookups built once per block
// (box index, local index, 1 or 2 boxes), so the gather has no per-node
// integer division.  Blocks are 32 x 4 x 2 node tiles (256 threads).  No
// atomics: the result does not depend on scheduling.
#pragma once

#include "common.cuh"
#include "kernels.h"
#include "vblock.cuh"

namespace ngf {
namespace nodek {

constexpr int NX = 32, NY = 4, NZ = 2, NT = NX * NY * NZ;

// node tiles per axis
__host__ __device__ inline void node_grid(const int *m, int &gx, int &gy, int &gz) {
    gx = (m[0] + NX - 1) / NX;
    gy = (m[1] + NY - 1) / NY;
    gz = (m[2] + NZ - 1) / NZ;
}

// Loads of data that no thread of the launch writes (RO: the read-only data
// path), or that an earlier phase of the same persistent launch wrote (plain
// loads, ordered by its grid barriers).
template <bool RO>
__device__ __forceinline__ float ldn(const float *p) {
    if constexpr (RO) return __ldg(p);
    else return *p;
}

// boxes of geometry b holding node k along axis ax: lo | local index << 16 | count << 24
__device__ __forceinline__ int box_lookup(const BoxGeom &b, int ax, int k) {
    const int C = b.C[ax];
    const int hi = k / C;
    const int lo = (hi >= 1 && k - hi * C == 0) ? hi - 1 : hi;
    const int top = min(hi, b.nb[ax] - 1);
    return lo | ((k - lo * C) << 16) | ((top - lo + 1) << 24);
}

template <bool RO>
__device__ __forceinline__ void gather_boxes(const float *boxes, const BoxGeom &b, int tx, int ty, int tz, float &s0,
                                             float &s1, float &s2) {
    const int ncx = tx >> 24, ncy = ty >> 24, n = ncx * ncy * (tz >> 24);   // 1 or 2 boxes per axis
    const int BX = b.C[0] + 1, BY = b.C[1] + 1;
    // first box: its index and the node's offset in it; further boxes step back by one box and C nodes per axis
    const unsigned cta0 = ((unsigned)(tz & 0xffff) * b.nb[1] + (ty & 0xffff)) * b.nb[0] + (tx & 0xffff);
    const unsigned off0 = (((tz >> 16) & 0xff) * BY + ((ty >> 16) & 0xff)) * BX + ((tx >> 16) & 0xff);
    const unsigned sz = 3u * b.box;
#pragma unroll
    for (int i = 0; i < 8; ++i) {   // at most 2 boxes per axis; all loads issued together
        if (i >= n) break;
        const int ix = i & (ncx - 1), iy = (i >> (ncx - 1)) & (ncy - 1), iz = i >> (ncx + ncy - 2);
        const unsigned cta = cta0 + (iz * b.nb[1] + iy) * b.nb[0] + ix;
        const unsigned off = off0 - (iz * b.C[2] * BY + iy * b.C[1]) * BX - ix * b.C[0];
        const float *p = boxes + cta * sz + off;
        s0 += ldn<RO>(p);
        s1 += ldn<RO>(p + b.box);
        s2 += ldn<RO>(p + 2 * b.box);
    }
}

// shared scratch of one block
struct NodeSmem {
    int tabA[NX + NY + NZ], tabB[NX + NY + NZ];
    double red[NT / 32];
};

// w = L v per node (3 components) and per-block partials of |L v|^2; block
// (b.x, b.y, b.z) is a node tile of the node_grid tiling, b.bid its index.
template <bool RO>
__device__ __forceinline__ void curv_body(const NodeArgs &a, const VBlock &b, NodeSmem &sm) {
    const int bx = b.x, by = b.y, bz = b.z;
    const int mx = a.m[0], my = a.m[1], mz = a.m[2];
    const long mxy = (long)mx * my, M = mxy * mz;
    const int kx = bx * NX + b.tid % NX, ky = by * NY + (b.tid / NX) % NY;
    const int kz = bz * NZ + b.tid / (NX * NY);
    float e = 0.f;
    if (kx < mx && ky < my && kz < mz) {
        const long k = (long)kz * mxy + (long)ky * mx + kx;
        const bool ix = kx >= 1 && kx <= mx - 2, iy = ky >= 1 && ky <= my - 2, iz = kz >= 1 && kz <= mz - 2;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float *v = a.v + c * M + k;
            const float v0 = ldn<RO>(v);
            float w = 0.f;
            if (ix) w = fmaf(ldn<RO>(v + 1) - 2.f * v0 + ldn<RO>(v - 1), a.ig2[0], w);
            if (iy) w = fmaf(ldn<RO>(v + mx) - 2.f * v0 + ldn<RO>(v - mx), a.ig2[1], w);
            if (iz) w = fmaf(ldn<RO>(v + mxy) - 2.f * v0 + ldn<RO>(v - mxy), a.ig2[2], w);
            a.w[c * M + k] = w;
            e = fmaf(w, w, e);
        }
    }
    if (a.rpart) {
        // FP32 within the warp (a tree of non-negative terms: relative error <= 5 ulp), FP64 across warps
        for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
        if ((b.tid & 31) == 0) sm.red[b.tid >> 5] = (double)e;
        b.sync();
        if (b.tid == 0) {
            double s = 0.0;
            for (int i = 0; i < NT / 32; ++i) s += sm.red[i];
            a.rpart[b.bid] = s;
        }
    }
}

// out = sA (NGF boxes) + sB (VCC boxes) + sC L^T w (and, with dpart, the
// per-block partials of dvec . out)
template <bool RO>
__device__ __forceinline__ void node_body(const NodeArgs &a, const VBlock &b, NodeSmem &sm) {
    const int bx = b.x, by = b.y, bz = b.z;
    const int tid = b.tid;
    const int mx = a.m[0], my = a.m[1], mz = a.m[2];
    const long mxy = (long)mx * my, M = mxy * mz;
    const int x0 = bx * NX, y0 = by * NY, z0 = bz * NZ;
    if (tid < NX + NY + NZ) {
        const int ax = tid < NX ? 0 : (tid < NX + NY ? 1 : 2);
        const int k = ax == 0 ? x0 + tid : (ax == 1 ? y0 + tid - NX : z0 + tid - NX - NY);
        const int kc = min(k, a.m[ax] - 1);   // nodes beyond the grid are not written
        if (a.boxA) sm.tabA[tid] = box_lookup(a.gA, ax, kc);
        if (a.boxB) sm.tabB[tid] = box_lookup(a.gB, ax, kc);
    }
    b.sync();
    const int lx = tid % NX, ly = (tid / NX) % NY, lz = tid / (NX * NY);
    const int kx = x0 + lx, ky = y0 + ly, kz = z0 + lz;
    float dq = 0.f;   // dvec . out over this thread's node
    if (kx < mx && ky < my && kz < mz) {
        float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
        if (a.boxA) gather_boxes<RO>(a.boxA, a.gA, sm.tabA[lx], sm.tabA[NX + ly], sm.tabA[NX + NY + lz], sa[0], sa[1], sa[2]);
        if (a.boxB) gather_boxes<RO>(a.boxB, a.gB, sm.tabB[lx], sm.tabB[NX + ly], sm.tabB[NX + NY + lz], sb[0], sb[1], sb[2]);
        const unsigned k = ((unsigned)kz * my + ky) * mx + kx, Mu = (unsigned)M, sy = mx, sz = (unsigned)mxy;
        const bool ix = kx >= 1 && kx <= mx - 2, iy = ky >= 1 && ky <= my - 2, iz = kz >= 1 && kz <= mz - 2;
        const bool xm = kx - 1 >= 1, xp = kx + 1 <= mx - 2, ym = ky - 1 >= 1, yp = ky + 1 <= my - 2;
        const bool zm = kz - 1 >= 1, zp = kz + 1 <= mz - 2;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float o = a.sA * sa[c] + a.sB * sb[c];
            if (a.w) {
                // L^T w: the rows of L that reference node k along each axis
                const float *p = a.w + c * Mu + k;
                const float w0 = ldn<RO>(p);
                float tx = 0.f, ty = 0.f, tz = 0.f;
                if (ix) tx -= 2.f * w0;
                if (xm) tx += ldn<RO>(p - 1);
                if (xp) tx += ldn<RO>(p + 1);
                if (iy) ty -= 2.f * w0;
                if (ym) ty += ldn<RO>(p - sy);
                if (yp) ty += ldn<RO>(p + sy);
                if (iz) tz -= 2.f * w0;
                if (zm) tz += ldn<RO>(p - sz);
                if (zp) tz += ldn<RO>(p + sz);
                o = fmaf(a.sC, fmaf(tz, a.ig2[2], fmaf(ty, a.ig2[1], tx * a.ig2[0])), o);
            }
            a.out[c * Mu + k] = o;
            if (a.dpart) dq = fmaf(ldn<RO>(a.dvec + c * Mu + k), o, dq);
        }
    }
    if (a.dpart) {
        // FP32 within the warp, FP64 across warps (the PCG's d.q partials)
        for (int off = 16; off > 0; off >>= 1) dq += __shfl_xor_sync(0xffffffffu, dq, off);
        if ((tid & 31) == 0) sm.red[tid >> 5] = (double)dq;
        b.sync();
        if (tid == 0) {
            double s = 0.0;
            for (int i = 0; i < NT / 32; ++i) s += sm.red[i];
            a.dpart[b.bid] = s;
        }
    }
}

}  // namespace nodek
}  // namespace ngf
