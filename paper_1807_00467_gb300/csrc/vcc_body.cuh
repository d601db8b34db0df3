// Volume change control, Eqs. (7)-(9): gradient (and energy) of
// sum_cells sum_{a,b,c} psi(d_abc), its Gauss-Newton product
// sum psi''(d) (grad d . v) grad d and the diagonal of that product,
// sum psi''(d) (d d / d u_{k,c})^2, one thread per grid cell: the body of the
// kernels of vcc.cu, shared with the persistent batched PCG kernel
// (pcg_batch.cu).
//
// In a cell the 64 bounds are d_abc = det[e1_a, e2_b, e3_c] = e1_a . X_bc with
// the four x-, y- and z-edges e1_a, e2_b, e3_c (identity plus the scaled node
// differences) and X_bc = e2_b x e3_c.  With weights w_abc (psi'(d), or
// psi''(d) times the directional derivative along v) the edge gradients are
//   G1_a = sum_bc w X_bc,
//   G2_b = sum_c e3_c x W_bc,   G3_c = sum_b W_bc x e2_b,   W_bc = sum_a w e1_a,
// so each (b, c) pair costs one cross product (two for the directional
// derivative) plus four dot products.  For the diagonal, d d_abc / d u is
// +-X_bc / g_x at the ends of e1_a, +-(e3_c x e1_a) / g_y at the ends of e2_b
// and +-(e1_a x e2_b) / g_z at the ends of e3_c (summed where two of these
// edges share a corner).  Bounds with d <= 0 are folds: weight 0 here,
// counted for the energy pass (the objective is then +inf).
#pragma once

#include "common.cuh"
#include "kernels.h"
#include "vblock.cuh"

namespace ngf {
namespace vcck {

constexpr int TX = kVccTile[0], TY = kVccTile[1], TZ = kVccTile[2], NC = TX * TY * TZ;
constexpr int BX = TX + 1, BY = TY + 1, BZ = TZ + 1, NB = BX * BY * BZ;
constexpr unsigned FULL = 0xffffffffu;

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 cross(const V3 &a, const V3 &b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float dot(const V3 &a, const V3 &b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ void axpy(float w, const V3 &x, V3 &y) {
    y.x = fmaf(w, x.x, y.x); y.y = fmaf(w, x.y, y.y); y.z = fmaf(w, x.z, y.z);
}
__device__ __forceinline__ void add(const V3 &x, V3 &y) { y.x += x.x; y.y += x.y; y.z += x.z; }

// Packed FP32 (two lanes of f32x2: the bounds of two x-edges a = 2p, 2p + 1)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// corner offset (ox + 2 oy + 4 oz) of edge e = p + 2 q of axis `ax` at end `hi`;
// p, q are the offsets along the other two axes in increasing axis order
__host__ __device__ constexpr int corner_of(int ax, int e, int hi) {
    return ax == 0 ? hi + 2 * (e & 1) + 4 * (e >> 1) : ax == 1 ? (e & 1) + 2 * hi + 4 * (e >> 1) : (e & 1) + 2 * (e >> 1) + 4 * hi;
}

struct Kahan32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// shared scratch of one block of cells
struct VccSmem {
    float su[3][NB];
    float sv[3][NB];
    float scell[8 * 3][NC];
    double red[NC / 32];
    int sfold[NC / 32];
    float wmn[NC / 32], wmx[NC / 32];
};

// VM = 0: gradient of sum psi(d) (+ energy, folds, min / max d);
// VM = 1: GN product along v; VM = 2: diagonal of the GN matrix.
template <int VM>
__device__ __forceinline__ void vcc_cell_body(const VccArgs &a, const VBlock &vb, VccSmem &sm) {
    constexpr bool GN = VM == 1, DG = VM == 2;
    float (&su)[3][NB] = sm.su;
    float (&sv)[3][NB] = sm.sv;
    float (&scell)[8 * 3][NC] = sm.scell;
    const int tid = vb.tid;
    const int mx = a.m[0], my = a.m[1], mz = a.m[2];
    const long mxy = (long)mx * my, M = mxy * mz;
    const int cx0 = vb.x * TX, cy0 = vb.y * TY, cz0 = vb.z * TZ;
    for (int i = tid; i < NB; i += NC) {
        const int lz = i / (BX * BY), r = i - lz * BX * BY, ly = r / BX, lx = r - ly * BX;
        const int gx = cx0 + lx, gy = cy0 + ly, gz = cz0 + lz;
        const bool ok = gx < mx && gy < my && gz < mz;
        const long k = (long)gz * mxy + (long)gy * mx + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            su[c][i] = ok ? a.u[c * M + k] : 0.f;
            if (GN) sv[c][i] = ok ? a.v[c * M + k] : 0.f;
        }
    }
    vb.sync();
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    const bool valid = cx0 + lx < mx - 1 && cy0 + ly < my - 1 && cz0 + lz < mz - 1;
    const int base = (lz * BY + ly) * BX + lx;
    const float ig0 = a.ig[0], ig1 = a.ig[1], ig2 = a.ig[2];
    auto at = [&](const auto &s, int o) {
        const int i = base + (o & 1) + ((o >> 1) & 1) * BX + (o >> 2) * BX * BY;
        return V3{s[0][i], s[1][i], s[2][i]};
    };
    // edges (identity plus scaled differences) of u, and of v for the GN product
    V3 E1[4], E2[4], E3[4], D1[GN ? 4 : 1], D2[GN ? 4 : 1], D3[GN ? 4 : 1];
    {
        V3 cu[8], cv[GN ? 8 : 1];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            cu[o] = at(su, o);
            if constexpr (GN) cv[o] = at(sv, o);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const V3 &x0 = cu[corner_of(0, e, 0)], &x1 = cu[corner_of(0, e, 1)];
            const V3 &y0 = cu[corner_of(1, e, 0)], &y1 = cu[corner_of(1, e, 1)];
            const V3 &z0 = cu[corner_of(2, e, 0)], &z1 = cu[corner_of(2, e, 1)];
            E1[e] = {fmaf(x1.x - x0.x, ig0, 1.f), (x1.y - x0.y) * ig0, (x1.z - x0.z) * ig0};
            E2[e] = {(y1.x - y0.x) * ig1, fmaf(y1.y - y0.y, ig1, 1.f), (y1.z - y0.z) * ig1};
            E3[e] = {(z1.x - z0.x) * ig2, (z1.y - z0.y) * ig2, fmaf(z1.z - z0.z, ig2, 1.f)};
            if (GN) {
                const V3 &p0 = cv[corner_of(0, e, 0)], &p1 = cv[corner_of(0, e, 1)];
                const V3 &q0 = cv[corner_of(1, e, 0)], &q1 = cv[corner_of(1, e, 1)];
                const V3 &r0 = cv[corner_of(2, e, 0)], &r1 = cv[corner_of(2, e, 1)];
                D1[e] = {(p1.x - p0.x) * ig0, (p1.y - p0.y) * ig0, (p1.z - p0.z) * ig0};
                D2[e] = {(q1.x - q0.x) * ig1, (q1.y - q0.y) * ig1, (q1.z - q0.z) * ig1};
                D3[e] = {(r1.x - r0.x) * ig2, (r1.y - r0.y) * ig2, (r1.z - r0.z) * ig2};
            }
        }
    }
    V3 G1[4], G2[4], G3[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) G1[e] = G2[e] = G3[e] = V3{0.f, 0.f, 0.f};
    int fold = 0;
    float dmn = 3.4e38f, dmx = -3.4e38f;
    Kahan32 en;
    float out[8][3];
#pragma unroll
    for (int o = 0; o < 8; ++o) out[o][0] = out[o][1] = out[o][2] = 0.f;
    if constexpr (DG) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const V3 X = cross(E2[b], E3[c]);
                const V3 gx{X.x * ig0, X.y * ig0, X.z * ig0};
#pragma unroll
                for (int aa = 0; aa < 4; ++aa) {
                    const float d = dot(E1[aa], X);
                    const float rd = __fdividef(1.f, d);
                    const float w = d > 0.f ? 2.f * rd * rd * rd : 0.f;   // psi''(d)
                    const V3 Y = cross(E3[c], E1[aa]), Z = cross(E1[aa], E2[b]);
                    const V3 gy{Y.x * ig1, Y.y * ig1, Y.z * ig1}, gz{Z.x * ig2, Z.y * ig2, Z.z * ig2};
                    // corners and signs are compile-time once the loops are unrolled
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        const int sx = (o == corner_of(0, aa, 1)) - (o == corner_of(0, aa, 0));
                        const int sy = (o == corner_of(1, b, 1)) - (o == corner_of(1, b, 0));
                        const int sz = (o == corner_of(2, c, 1)) - (o == corner_of(2, c, 0));
                        if (sx == 0 && sy == 0 && sz == 0) continue;
                        V3 g{0.f, 0.f, 0.f};
                        bool first = true;
                        auto term = [&](int sg, const V3 &t) {
                            if (sg == 0) return;
                            const V3 st = sg > 0 ? t : V3{-t.x, -t.y, -t.z};
                            if (first) g = st;
                            else add(st, g);
                            first = false;
                        };
                        term(sx, gx);
                        term(sy, gy);
                        term(sz, gz);
                        out[o][0] = fmaf(w * g.x, g.x, out[o][0]);
                        out[o][1] = fmaf(w * g.y, g.y, out[o][1]);
                        out[o][2] = fmaf(w * g.z, g.z, out[o][2]);
                    }
                }
            }
        }
    } else if constexpr (GN) {
        // the x-edges in pairs (a = 2p, 2p + 1), one f32x2 lane each
        float2 e1x[2], e1y[2], e1z[2], d1x[2], d1y[2], d1z[2], g1x[2], g1y[2], g1z[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            e1x[p] = make_float2(E1[2 * p].x, E1[2 * p + 1].x);
            e1y[p] = make_float2(E1[2 * p].y, E1[2 * p + 1].y);
            e1z[p] = make_float2(E1[2 * p].z, E1[2 * p + 1].z);
            d1x[p] = make_float2(D1[2 * p].x, D1[2 * p + 1].x);
            d1y[p] = make_float2(D1[2 * p].y, D1[2 * p + 1].y);
            d1z[p] = make_float2(D1[2 * p].z, D1[2 * p + 1].z);
            g1x[p] = g1y[p] = g1z[p] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const V3 X = cross(E2[b], E3[c]);
                V3 Y = cross(D2[b], E3[c]);
                add(cross(E2[b], D3[c]), Y);
                const float2 Xx = bc2(X.x), Xy = bc2(X.y), Xz = bc2(X.z);
                float2 wx = make_float2(0.f, 0.f), wy = wx, wz = wx;   // W = sum_a w e1_a, per lane
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2 d = fma2(e1z[p], Xz, fma2(e1y[p], Xy, mul2(e1x[p], Xx)));
                    // grad d . v = d1_a . X + e1_a . Y
                    const float2 dd = fma2(e1z[p], bc2(Y.z), fma2(e1y[p], bc2(Y.y), fma2(e1x[p], bc2(Y.x),
                                      fma2(d1z[p], Xz, fma2(d1y[p], Xy, mul2(d1x[p], Xx))))));
                    const float r0 = __fdividef(1.f, d.x), r1 = __fdividef(1.f, d.y);
                    const float2 r = make_float2(r0, r1);
                    float2 w = mul2(mul2(mul2(r, r), mul2(r, bc2(2.f))), dd);   // psi''(d) (grad d . v)
                    w.x = d.x > 0.f ? w.x : 0.f;
                    w.y = d.y > 0.f ? w.y : 0.f;
                    g1x[p] = fma2(w, Xx, g1x[p]);
                    g1y[p] = fma2(w, Xy, g1y[p]);
                    g1z[p] = fma2(w, Xz, g1z[p]);
                    wx = fma2(w, e1x[p], wx);
                    wy = fma2(w, e1y[p], wy);
                    wz = fma2(w, e1z[p], wz);
                }
                const V3 W{wx.x + wx.y, wy.x + wy.y, wz.x + wz.y};
                add(cross(E3[c], W), G2[b]);
                add(cross(W, E2[b]), G3[c]);
            }
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            G1[2 * p] = V3{g1x[p].x, g1y[p].x, g1z[p].x};
            G1[2 * p + 1] = V3{g1x[p].y, g1y[p].y, g1z[p].y};
        }
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const V3 X = cross(E2[b], E3[c]);
                V3 W{0.f, 0.f, 0.f};
#pragma unroll
                for (int aa = 0; aa < 4; ++aa) {
                    const float d = dot(E1[aa], X);
                    const bool pos = d > 0.f;
                    dmn = fminf(dmn, d);
                    dmx = fmaxf(dmx, d);
                    fold += pos ? 0 : 1;
                    const float rd = __frcp_rn(d);
                    const float dm = d - 1.f;
                    en.add(pos ? dm * dm * rd : 0.f);               // psi(d) = (d - 1)^2 / d
                    const float w = pos ? dm * (d + 1.f) * rd * rd : 0.f;   // psi'(d) = 1 - 1/d^2
                    axpy(w, X, G1[aa]);
                    axpy(w, E1[aa], W);
                }
                add(cross(E3[c], W), G2[b]);
                add(cross(W, E2[b]), G3[c]);
            }
        }
    }
    // edge gradients onto the cell's corners (scaled by 1/g of the edge's axis)
#pragma unroll
    for (int e = 0; e < 4 && !DG; ++e) {
        const V3 g1{G1[e].x * ig0, G1[e].y * ig0, G1[e].z * ig0};
        const V3 g2{G2[e].x * ig1, G2[e].y * ig1, G2[e].z * ig1};
        const V3 g3{G3[e].x * ig2, G3[e].y * ig2, G3[e].z * ig2};
        const int x1 = corner_of(0, e, 1), x0 = corner_of(0, e, 0);
        const int y1 = corner_of(1, e, 1), y0 = corner_of(1, e, 0);
        const int z1 = corner_of(2, e, 1), z0 = corner_of(2, e, 0);
        out[x1][0] += g1.x; out[x1][1] += g1.y; out[x1][2] += g1.z;
        out[x0][0] -= g1.x; out[x0][1] -= g1.y; out[x0][2] -= g1.z;
        out[y1][0] += g2.x; out[y1][1] += g2.y; out[y1][2] += g2.z;
        out[y0][0] -= g2.x; out[y0][1] -= g2.y; out[y0][2] -= g2.z;
        out[z1][0] += g3.x; out[z1][1] += g3.y; out[z1][2] += g3.z;
        out[z0][0] -= g3.x; out[z0][1] -= g3.y; out[z0][2] -= g3.z;
    }
#pragma unroll
    for (int o = 0; o < 8; ++o)
#pragma unroll
        for (int k = 0; k < 3; ++k) scell[o * 3 + k][tid] = valid ? out[o][k] : 0.f;
    vb.sync();
    // gather per node of the box from the (up to) 8 cells of this tile
    const int cta = vb.bid;
    float *dst = a.boxes + (long)cta * 3 * a.box;
    for (int i = tid; i < NB; i += NC) {
        const int bz = i / (BX * BY), r = i - bz * BX * BY, by = r / BX, bx = r - by * BX;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int qx = bx - (o & 1), qy = by - ((o >> 1) & 1), qz = bz - (o >> 2);
            if (qx < 0 || qy < 0 || qz < 0 || qx >= TX || qy >= TY || qz >= TZ) continue;
            const int c = (qz * TY + qy) * TX + qx;
            s0 += scell[o * 3][c];
            s1 += scell[o * 3 + 1][c];
            s2 += scell[o * 3 + 2][c];
        }
        dst[i] = s0 * a.wscale;
        dst[a.box + i] = s1 * a.wscale;
        dst[2 * a.box + i] = s2 * a.wscale;
    }
    if (VM == 0) {
        // energy, fold count and min / max d of the block
        double (&red)[NC / 32] = sm.red;
        int (&sfold)[NC / 32] = sm.sfold;
        float (&wmn)[NC / 32] = sm.wmn;
        float (&wmx)[NC / 32] = sm.wmx;
        double e = valid ? (double)en.s - (double)en.c : 0.0;
        int f = valid ? fold : 0;
        if (!valid) { dmn = 3.4e38f; dmx = -3.4e38f; }
        for (int off = 16; off > 0; off >>= 1) {
            e += __shfl_xor_sync(FULL, e, off);
            f += __shfl_xor_sync(FULL, f, off);
            dmn = fminf(dmn, __shfl_xor_sync(FULL, dmn, off));
            dmx = fmaxf(dmx, __shfl_xor_sync(FULL, dmx, off));
        }
        const int w = tid >> 5;
        if ((tid & 31) == 0) { red[w] = e; sfold[w] = f; wmn[w] = dmn; wmx[w] = dmx; }
        vb.sync();
        if (tid == 0) {
            double t = 0.0;
            int ft = 0;
            float mn = 3.4e38f, mxv = -3.4e38f;
            for (int i = 0; i < NC / 32; ++i) {
                t += red[i];
                ft += sfold[i];
                mn = fminf(mn, wmn[i]);
                mxv = fmaxf(mxv, wmx[i]);
            }
            a.epart[cta] = t;
            a.fold[cta] = ft;
            a.dmin[cta] = mn;
            a.dmax[cta] = mxv;
        }
    }
}

}  // namespace vcck
}  // namespace ngf
