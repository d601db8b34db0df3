// Fused voxel-tile kernel for the NGF term of Eq. (1): trilinear warp of the
// template, central-difference gradients, per-voxel NGF residual, the adjoint
// of the central difference, and the gather of voxel contributions onto the
// grid nodes (P^T), in one pass over the volume.
//
// One CTA owns a tile of 32 x TY voxels in x-y (aligned to grid cells) and a
// chunk of TZ voxel planes along z, and marches through the chunk plane by
// plane with three pipelined stages:
//   W (plane p+2): y = x + P u, sample T(y) and dT/dy           (halo 2 in x-y)
//   C (plane p+1): f = grad R, g = grad T(y), r, c = d(1-r^2)/dg (halo 1)
//   A (plane p)  : b = -div-like adjoint of the central difference of c,
//                  z = b dT/dy, then P^T onto the CTA's node box.
// Shared-memory rings hold three planes of each stage's output, so every
// voxel is sampled once per CTA (plus the 2-voxel x-y halo) and R, T are read
// from HBM once.  Node contributions are reduced along x with warp shuffles
// (one lane per voxel column), along y through shared memory, and along z
// into a per-CTA node box in shared memory; boxes of neighbouring CTAs that
// share boundary nodes are summed by finalize_nodes (gather, no atomics).
//
// The same kernel, with different MODE, evaluates the objective only
// (line search), stores the Gauss-Newton linearisation, or applies the NGF
// Gauss-Newton matrix 2 hbar J^T J (stage W then forms dT . P v from the
// stored dT/dy, stage C forms 2 (a . G(dT . P v)) a from the stored a).
#include "common.cuh"
#include "kernels.h"

namespace ngf {

template <int MODE>
struct Mode {
    static constexpr bool grad = MODE == MODE_GRAD || MODE == MODE_GRADLIN || MODE == MODE_MATVEC;
    static constexpr bool store = MODE == MODE_LIN || MODE == MODE_GRADLIN;
    static constexpr bool matvec = MODE == MODE_MATVEC;
    static constexpr bool diag = MODE == MODE_DIAG;
    static constexpr bool reduce = grad || diag;   // stage A and the node box
    static constexpr int HW = grad ? 2 : 1;       // halo of stage W
    static constexpr int HC = HW - 1;             // halo of stage C
};

// Shared-memory carve-up (floats).  Host and device agree on it.
struct TileSmem {
    int tw, rr, cr, dtr, nodes, rows, box, total;
};

__host__ __device__ inline TileSmem tile_smem(const TileGeom &g, int mode) {
    const bool grad = mode == MODE_GRAD || mode == MODE_GRADLIN || mode == MODE_MATVEC;
    const bool matvec = mode == MODE_MATVEC, diag = mode == MODE_DIAG, reduce = grad || diag;
    const int HW = grad ? 2 : 1;
    TileSmem s;
    int RW = kTileX + 2 * HW, RH = g.TY + 2 * HW;
    int CW = kTileX + 2 * (HW - 1), CH = g.TY + 2 * (HW - 1);
    int off = 0;
    s.tw = off; off += diag ? 0 : 3 * RW * RH;
    s.rr = off; off += (matvec || diag) ? 0 : 3 * RW * RH;
    s.cr = off; off += grad ? 9 * CW * CH : (diag ? 9 * RW * RH : 0);
    s.dtr = off; off += reduce ? 9 * kTileX * g.TY : 0;
    s.nodes = off; off += diag ? 0 : 2 * 3 * g.nxt * g.nyt;
    s.rows = off; off += reduce ? 2 * g.TY * g.C[0] * 3 : 0;
    s.box = off; off += reduce ? 3 * g.box : 0;
    s.total = off;
    return s;
}

size_t tile_smem_bytes(const TileGeom &g, int mode) { return sizeof(float) * (size_t)tile_smem(g, mode).total; }

__device__ __forceinline__ int ring3(int p) { return (p + 6) % 3; }

// Per-axis placement of the template sample from the FP32 cell decision k.
// The sample is taken from voxel c0 and its neighbour c0 + step at fraction f
// in [0, 1), so voxel values are reproduced exactly at f = 0: on the last
// voxel (k = n-1, fraction 0) and above the domain the pair (n-1, n-2) is
// used with step -1 and the derivative sign flipped.
__device__ __forceinline__ void place_axis(int k, float fr, int n, int &c0, int &step, float &f, bool &in) {
    if (k < 0) {
        c0 = 0; step = 1; f = 0.f; in = false;
    } else if (k >= n - 1) {
        c0 = n - 1; step = -1; f = 0.f; in = k == n - 1 && fr == 0.f;
    } else {
        c0 = k; step = 1; f = fr; in = true;
    }
}

template <int TY, int MODE, typename TImg>
__global__ void __launch_bounds__(kThreads) ngf_tile_kernel(const TileArgs<TImg> a) {
    using M = Mode<MODE>;
    constexpr int HW = M::HW, HC = M::HC;
    constexpr int RW = kTileX + 2 * HW, RH = TY + 2 * HW;
    constexpr int CW = kTileX + 2 * HC, CH = TY + 2 * HC;
    constexpr int PPT = (RW * RH + kThreads - 1) / kThreads;   // W-stage points per thread
    extern __shared__ float smem[];
    const TileGeom &g = a.g;
    const TileSmem L = tile_smem(g, MODE);
    float *s_tw = smem + L.tw, *s_rr = smem + L.rr, *s_cr = smem + L.cr, *s_dt = smem + L.dtr;
    float *s_nodes = smem + L.nodes, *s_rows = smem + L.rows, *s_box = smem + L.box;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long sxy = (long)nx * ny, N = sxy * nz;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * TY, z0 = blockIdx.z * g.TZ;
    const int TZc = min(g.TZ, nz - z0);
    const int rx = g.rho[0], ry = g.rho[1], rz = g.rho[2];
    const int mx = g.m[0], my = g.m[1];
    const long mxy = (long)mx * my, Mn = mxy * g.m[2];
    const int CX = g.C[0], CY = g.C[1];
    const int kx_lo = max(x0 - HW, 0) / rx, ky_lo = max(y0 - HW, 0) / ry;
    const int nxt = g.nxt, nyt = g.nyt, nplane = nxt * nyt;

    if (M::reduce)
        for (int i = tid; i < 3 * g.box; i += kThreads) s_box[i] = 0.f;

    // Per-thread W-stage points and their x-y interpolated node values at the
    // two node planes bracketing the current voxel plane.
    float U[PPT][2][3];
    int cur_cz = -1000;
    float dsum = 0.f, dcomp = 0.f;   // Kahan sum of (1 - r^2) over own voxels

    const int nsteps = TZc + 2 * HW;
    for (int s = 0; s < nsteps; ++s) {
        const int pW = z0 - HW + s;
        // ---------------- node planes for the prolongation of plane pW
        if (!M::diag && pW >= 0 && pW < nz) {
            const int cz = pW / rz;
            if (cz != cur_cz) {
                const bool both = cz != cur_cz + 1;
                for (int kz = both ? cz : cz + 1; kz <= cz + 1; ++kz) {
                    float *dst = s_nodes + (kz & 1) * 3 * nplane;
                    for (int i = tid; i < 3 * nplane; i += kThreads) {
                        int comp = i / nplane, r = i - comp * nplane;
                        int ly = r / nxt, lx = r - ly * nxt;
                        int gx = kx_lo + lx, gy = ky_lo + ly;
                        float v = 0.f;
                        if (gx < mx && gy < my) v = __ldg(a.u + comp * Mn + (long)kz * mxy + (long)gy * mx + gx);
                        dst[i] = v;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const int pt = tid + j * kThreads;
                    const int ry_ = pt / RW, rx_ = pt - ry_ * RW;
                    const int gx = x0 - HW + rx_, gy = y0 - HW + ry_;
                    if (pt < RW * RH && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                        const int cx = gx / rx, cy = gy / ry;
                        const float fx = ((gx - cx * rx) + 0.5f) / rx, fy = ((gy - cy * ry) + 0.5f) / ry;
                        const int lx = cx - kx_lo, ly = cy - ky_lo;
                        if (both) {
                            const float *np_ = s_nodes + (cz & 1) * 3 * nplane;
#pragma unroll
                            for (int comp = 0; comp < 3; ++comp) {
                                const float *q = np_ + comp * nplane + ly * nxt + lx;
                                const float ux0 = lerp_fixed(q[0], q[1], 1.f - fx, fx);
                                const float ux1 = lerp_fixed(q[nxt], q[nxt + 1], 1.f - fx, fx);
                                U[j][0][comp] = lerp_fixed(ux0, ux1, 1.f - fy, fy);
                            }
                        } else {
#pragma unroll
                            for (int comp = 0; comp < 3; ++comp) U[j][0][comp] = U[j][1][comp];
                        }
                        const float *np_ = s_nodes + ((cz + 1) & 1) * 3 * nplane;
#pragma unroll
                        for (int comp = 0; comp < 3; ++comp) {
                            const float *q = np_ + comp * nplane + ly * nxt + lx;
                            const float ux0 = lerp_fixed(q[0], q[1], 1.f - fx, fx);
                            const float ux1 = lerp_fixed(q[nxt], q[nxt + 1], 1.f - fx, fx);
                            U[j][1][comp] = lerp_fixed(ux0, ux1, 1.f - fy, fy);
                        }
                    }
                }
                cur_cz = cz;
            }
        }
        // ---------------- stage W: plane pW on the halo-HW region
        if (M::diag) {
            // squares of the stored a = dr/dg around the tile, dT/dy on the tile
            float *ca = s_cr + ring3(pW) * 3 * RW * RH;
            float *dt = s_dt + ring3(pW) * 3 * kTileX * TY;
            const bool zin = pW >= 0 && pW < nz;
            for (int pt = tid; pt < RW * RH; pt += kThreads) {
                const int ry_ = pt / RW, rx_ = pt - ry_ * RW;
                const int gx = x0 - HW + rx_, gy = y0 - HW + ry_;
                const bool in = zin && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
                float q0 = 0.f, q1 = 0.f, q2 = 0.f;
                if (in) {
                    const long vox = (long)pW * sxy + (long)gy * nx + gx;
                    q0 = __ldg(a.lin_a + vox);
                    q1 = __ldg(a.lin_a + N + vox);
                    q2 = __ldg(a.lin_a + 2 * N + vox);
                    const bool own = rx_ >= HW && rx_ < HW + kTileX && ry_ >= HW && ry_ < HW + TY && pW >= z0 &&
                                     pW < z0 + TZc;
                    if (own) {
                        const int k = (ry_ - HW) * kTileX + (rx_ - HW);
                        dt[k] = __ldg(a.lin_dT + vox);
                        dt[kTileX * TY + k] = __ldg(a.lin_dT + N + vox);
                        dt[2 * kTileX * TY + k] = __ldg(a.lin_dT + 2 * N + vox);
                    }
                }
                ca[pt] = q0 * q0;
                ca[RW * RH + pt] = q1 * q1;
                ca[2 * RW * RH + pt] = q2 * q2;
            }
        } else {
            float *tw = s_tw + ring3(pW) * RW * RH;
            float *rr = s_rr + ring3(pW) * RW * RH;
            float *dt = s_dt + ring3(pW) * 3 * kTileX * TY;
            const bool zin = pW >= 0 && pW < nz;
            const int cz = zin ? pW / rz : 0;
            const float fz = zin ? ((pW - cz * rz) + 0.5f) / rz : 0.f;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int pt = tid + j * kThreads;
                if (pt >= RW * RH) continue;
                const int ry_ = pt / RW, rx_ = pt - ry_ * RW;
                const int gx = x0 - HW + rx_, gy = y0 - HW + ry_;
                const bool in = zin && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
                const bool own = in && rx_ >= HW && rx_ < HW + kTileX && ry_ >= HW && ry_ < HW + TY && pW >= z0 &&
                                 pW < z0 + TZc;
                float val = 0.f, rv = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
                if (in) {
                    const long vox = (long)pW * sxy + (long)gy * nx + gx;
                    float pu[3];
#pragma unroll
                    for (int comp = 0; comp < 3; ++comp) pu[comp] = lerp_fixed(U[j][0][comp], U[j][1][comp], 1.f - fz, fz);
                    if (M::matvec) {
                        d0 = __ldg(a.lin_dT + vox);
                        d1 = __ldg(a.lin_dT + N + vox);
                        d2 = __ldg(a.lin_dT + 2 * N + vox);
                        val = d0 * pu[0] + d1 * pu[1] + d2 * pu[2];
                    } else {
                        int c[3], stp[3];
                        float f[3];
                        bool ins[3];
                        const int ii[3] = {gx, gy, pW};
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            // cell decision: fixed-order FP32 product (shared definition with the oracle)
                            const float q = __fmul_rn(pu[ax], g.invh[ax]);
                            const float fl = floorf(q);
                            // fraction: add the exact rounding error of the product and the
                            // correction for float(1/h) (g.invh_rel = 1 - h * float(1/h))
                            const float e = __fmaf_rn(pu[ax], g.invh[ax], -q);
                            const float fr = (q - fl) + __fmaf_rn(q, g.invh_rel[ax], e);
                            place_axis(ii[ax] + (int)fl, q - fl, g.n[ax], c[ax], stp[ax], f[ax], ins[ax]);
                            if (stp[ax] > 0 && ins[ax]) f[ax] = fr;
                        }
                        const long sx = stp[0], sy = (long)stp[1] * nx, sz = (long)stp[2] * sxy;
                        const long b = (long)c[2] * sxy + (long)c[1] * nx + c[0];
                        const float t000 = ldimg(a.T, b), t100 = ldimg(a.T, b + sx);
                        const float t010 = ldimg(a.T, b + sy), t110 = ldimg(a.T, b + sy + sx);
                        const float t001 = ldimg(a.T, b + sz), t101 = ldimg(a.T, b + sz + sx);
                        const float t011 = ldimg(a.T, b + sz + sy), t111 = ldimg(a.T, b + sz + sy + sx);
                        const float dx00 = t100 - t000, dx10 = t110 - t010, dx01 = t101 - t001, dx11 = t111 - t011;
                        const float v00 = fmaf(f[0], dx00, t000), v10 = fmaf(f[0], dx10, t010);
                        const float v01 = fmaf(f[0], dx01, t001), v11 = fmaf(f[0], dx11, t011);
                        const float dy0 = v10 - v00, dy1 = v11 - v01;
                        const float w0 = fmaf(f[1], dy0, v00), w1 = fmaf(f[1], dy1, v01);
                        const float dz = w1 - w0;
                        val = fmaf(f[2], dz, w0);
                        const float ax0 = fmaf(f[1], dx10 - dx00, dx00), ax1 = fmaf(f[1], dx11 - dx01, dx01);
                        d0 = ins[0] ? fmaf(f[2], ax1 - ax0, ax0) * g.invh[0] * (float)stp[0] : 0.f;
                        d1 = ins[1] ? fmaf(f[2], dy1 - dy0, dy0) * g.invh[1] * (float)stp[1] : 0.f;
                        d2 = ins[2] ? dz * g.invh[2] * (float)stp[2] : 0.f;
                        rv = ldimg(a.R, vox);
                    }
                    if (M::store && own) {
                        a.st_dT[vox] = d0;
                        a.st_dT[N + vox] = d1;
                        a.st_dT[2 * N + vox] = d2;
                    }
                }
                tw[pt] = val;
                if (!M::matvec) rr[pt] = rv;
                if (M::grad && own) {
                    const int k = (ry_ - HW) * kTileX + (rx_ - HW);
                    dt[k] = d0;
                    dt[kTileX * TY + k] = d1;
                    dt[2 * kTileX * TY + k] = d2;
                }
            }
        }
        __syncthreads();
        // ---------------- stage C: plane pC on the halo-HC region
        const int pC = pW - 1;
        if (!M::diag && pC >= z0 - HC) {
            const float *tw_m = s_tw + ring3(pC - 1) * RW * RH, *tw_0 = s_tw + ring3(pC) * RW * RH,
                        *tw_p = s_tw + ring3(pC + 1) * RW * RH;
            const float *rr_m = s_rr + ring3(pC - 1) * RW * RH, *rr_0 = s_rr + ring3(pC) * RW * RH,
                        *rr_p = s_rr + ring3(pC + 1) * RW * RH;
            float *cr = s_cr + ring3(pC) * 3 * CW * CH;
            for (int pt = tid; pt < CW * CH; pt += kThreads) {
                const int cy_ = pt / CW, cx_ = pt - cy_ * CW;
                const int gx = x0 - HC + cx_, gy = y0 - HC + cy_;
                const bool interior = gx >= 1 && gx <= nx - 2 && gy >= 1 && gy <= ny - 2 && pC >= 1 && pC <= nz - 2;
                const int w = (cy_ + HW - HC) * RW + (cx_ + HW - HC);   // index in the W region
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                if (interior) {
                    const float g0 = (tw_0[w + 1] - tw_0[w - 1]) * g.inv2h[0];
                    const float g1 = (tw_0[w + RW] - tw_0[w - RW]) * g.inv2h[1];
                    const float g2 = (tw_p[w] - tw_m[w]) * g.inv2h[2];
                    const long vox = (long)pC * sxy + (long)gy * nx + gx;
                    if (M::matvec) {
                        const float a0 = __ldg(a.lin_a + vox), a1 = __ldg(a.lin_a + N + vox), a2 = __ldg(a.lin_a + 2 * N + vox);
                        const float dr = 2.f * (a0 * g0 + a1 * g1 + a2 * g2);
                        c0 = dr * a0; c1 = dr * a1; c2 = dr * a2;
                    } else {
                        const float f0 = (rr_0[w + 1] - rr_0[w - 1]) * g.inv2h[0];
                        const float f1 = (rr_0[w + RW] - rr_0[w - RW]) * g.inv2h[1];
                        const float f2 = (rr_p[w] - rr_m[w]) * g.inv2h[2];
                        // the same operation order for <f,g>, |f|^2, |g|^2: f = g gives equal values
                        const float fg = __fmaf_rn(f2, g2, __fmaf_rn(f1, g1, __fmaf_rn(f0, g0, g.eta2)));
                        const float ff = __fmaf_rn(f2, f2, __fmaf_rn(f1, f1, __fmaf_rn(f0, f0, g.eta2)));
                        const float gg = __fmaf_rn(g2, g2, __fmaf_rn(g1, g1, __fmaf_rn(g0, g0, g.eta2)));
                        const float rff = __frcp_rn(ff), rgg = __frcp_rn(gg);
                        // 1 - r^2 = (|f x g|^2 + eta^2 |f - g|^2) / (|f|_eta^2 |g|_eta^2)
                        // products rounded separately: exactly zero when f = g
                        const float x0_ = __fmul_rn(f1, g2) - __fmul_rn(f2, g1);
                        const float x1_ = __fmul_rn(f2, g0) - __fmul_rn(f0, g2);
                        const float x2_ = __fmul_rn(f0, g1) - __fmul_rn(f1, g0);
                        const float e0 = f0 - g0, e1 = f1 - g1, e2 = f2 - g2;
                        const float num = x0_ * x0_ + x1_ * x1_ + x2_ * x2_ + g.eta2 * (e0 * e0 + e1 * e1 + e2 * e2);
                        const float om = num * rff * rgg;
                        const bool own = gx >= x0 && gx < x0 + kTileX && gy >= y0 && gy < y0 + TY && pC >= z0 &&
                                         pC < z0 + TZc;
                        if (own) {   // Kahan summation
                            const float yk = om - dcomp;
                            const float tk = dsum + yk;
                            dcomp = (tk - dsum) - yk;
                            dsum = tk;
                        }
                        // a = dr/dg = (f |g|^2 - <f,g> g) / (|f| |g|^3) (norms with eta);
                        // q = f |g|^2 - <f,g> g, each product rounded once: 0 when f = g
                        const float q0 = __fmul_rn(f0, gg) - __fmul_rn(fg, g0);
                        const float q1 = __fmul_rn(f1, gg) - __fmul_rn(fg, g1);
                        const float q2 = __fmul_rn(f2, gg) - __fmul_rn(fg, g2);
                        if (M::grad) {   // c = d(1 - r^2)/dg = -2 r a = -2 <f,g> q / (|f|^2 |g|^4)
                            const float sc = -2.f * fg * rff * rgg * rgg;
                            c0 = sc * q0; c1 = sc * q1; c2 = sc * q2;
                        }
                        if (M::store && own) {
                            const float inv = rsqrtf(ff * gg) * rgg;
                            a.st_a[vox] = q0 * inv;
                            a.st_a[N + vox] = q1 * inv;
                            a.st_a[2 * N + vox] = q2 * inv;
                        }
                    }
                } else if (M::store) {
                    const bool own = gx >= x0 && gx < x0 + kTileX && gx < nx && gy >= y0 && gy < y0 + TY &&
                                     gy < ny && pC >= z0 && pC < z0 + TZc;
                    if (own) {
                        const long vox = (long)pC * sxy + (long)gy * nx + gx;
                        a.st_a[vox] = 0.f;
                        a.st_a[N + vox] = 0.f;
                        a.st_a[2 * N + vox] = 0.f;
                    }
                }
                if (M::grad) {
                    cr[pt] = c0;
                    cr[CW * CH + pt] = c1;
                    cr[2 * CW * CH + pt] = c2;
                }
            }
        }
        __syncthreads();
        if (!M::reduce) continue;
        // ---------------- stage A: plane pA, adjoint and P^T
        // (diagonal mode: beta * dT^2 and P^T with squared weights)
        const int pA = M::diag ? pW - 1 : pC - 1;
        if (pA >= z0) {
            constexpr int AW = M::diag ? RW : CW, AH = M::diag ? RH : CH, AO = M::diag ? HW : HC;
            const float *c_m = s_cr + ring3(pA - 1) * 3 * AW * AH, *c_0 = s_cr + ring3(pA) * 3 * AW * AH,
                        *c_p = s_cr + ring3(pA + 1) * 3 * AW * AH;
            const float *dt = s_dt + ring3(pA) * 3 * kTileX * TY;
            const int gx = x0 + lane;
            float fx = ((lane & (rx - 1)) + 0.5f) / rx, fx0 = 1.f - fx;
            if (M::diag) { fx0 *= fx0; fx *= fx; }
            for (int ty = warp; ty < TY; ty += kThreads / 32) {
                const int gy = y0 + ty;
                float z0_ = 0.f, z1_ = 0.f, z2_ = 0.f;
                if (gx < nx && gy < ny) {
                    const int w = (ty + AO) * AW + (lane + AO);
                    const int k = ty * kTileX + lane;
                    float b;
                    if (M::diag) {
                        b = (c_0[w - 1] + c_0[w + 1]) * (g.inv2h[0] * g.inv2h[0]) +
                            (c_0[AW * AH + w - AW] + c_0[AW * AH + w + AW]) * (g.inv2h[1] * g.inv2h[1]) +
                            (c_m[2 * AW * AH + w] + c_p[2 * AW * AH + w]) * (g.inv2h[2] * g.inv2h[2]);
                        const float d0 = dt[k], d1 = dt[kTileX * TY + k], d2 = dt[2 * kTileX * TY + k];
                        z0_ = b * d0 * d0;
                        z1_ = b * d1 * d1;
                        z2_ = b * d2 * d2;
                    } else {
                        b = (c_0[w - 1] - c_0[w + 1]) * g.inv2h[0] +
                            (c_0[AW * AH + w - AW] - c_0[AW * AH + w + AW]) * g.inv2h[1] +
                            (c_m[2 * AW * AH + w] - c_p[2 * AW * AH + w]) * g.inv2h[2];
                        z0_ = b * dt[k];
                        z1_ = b * dt[kTileX * TY + k];
                        z2_ = b * dt[2 * kTileX * TY + k];
                    }
                }
                float lo[3] = {fx0 * z0_, fx0 * z1_, fx0 * z2_};
                float hi[3] = {fx * z0_, fx * z1_, fx * z2_};
                for (int off = 1; off < rx; off <<= 1)
                    for (int comp = 0; comp < 3; ++comp) {
                        lo[comp] += __shfl_xor_sync(0xffffffffu, lo[comp], off);
                        hi[comp] += __shfl_xor_sync(0xffffffffu, hi[comp], off);
                    }
                if ((lane & (rx - 1)) == 0) {
                    const int cell = lane / rx;
                    for (int comp = 0; comp < 3; ++comp) {
                        s_rows[(ty * CX + cell) * 3 + comp] = lo[comp];
                        s_rows[((TY + ty) * CX + cell) * 3 + comp] = hi[comp];
                    }
                }
            }
            __syncthreads();
            const int lz = (pA - z0) / rz;
            const float fz = (((pA - z0) - lz * rz) + 0.5f) / rz;
            const int nbx = CX + 1, nby = CY + 1;
            for (int e = tid; e < 3 * nbx * nby; e += kThreads) {
                const int jx = e % nbx, t2 = e / nbx, jy = t2 % nby, comp = t2 / nby;
                float val = 0.f;
                const int ty_lo = max(0, (jy - 1) * ry), ty_hi = min(TY, (jy + 1) * ry);
                for (int ty = ty_lo; ty < ty_hi; ++ty) {
                    const int cyl = ty / ry;
                    const float fy = ((ty - cyl * ry) + 0.5f) / ry;
                    float wy = cyl == jy ? 1.f - fy : fy;
                    if (M::diag) wy *= wy;
                    float rv = 0.f;
                    if (jx < CX) rv += s_rows[(ty * CX + jx) * 3 + comp];
                    if (jx >= 1) rv += s_rows[((TY + ty) * CX + jx - 1) * 3 + comp];
                    val = fmaf(wy, rv, val);
                }
                float *bx = s_box + comp * g.box + (lz * nby + jy) * nbx + jx;
                const float wz0 = M::diag ? (1.f - fz) * (1.f - fz) : 1.f - fz, wz1 = M::diag ? fz * fz : fz;
                bx[0] += wz0 * val;
                bx[nby * nbx] += wz1 * val;
            }
        }
        __syncthreads();
    }

    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (M::reduce) {
        __syncthreads();
        float *dst = a.boxes + (long)cta * 3 * g.box;
        for (int i = tid; i < 3 * g.box; i += kThreads) dst[i] = s_box[i];
    }
    if (!M::matvec && !M::diag) {
        double v = (double)dsum - (double)dcomp;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        __shared__ double red[kThreads / 32];
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < kThreads / 32; ++i) t += red[i];
            a.dpart[cta] = t;
        }
    }
}

template <typename TImg>
static cudaError_t launch_mode(int mode, const TileArgs<TImg> &a, cudaStream_t st) {
    dim3 grid(a.g.nb[0], a.g.nb[1], a.g.nb[2]);
    size_t smem = tile_smem_bytes(a.g, mode);
#define NGF_LAUNCH(TYV, MV)                                                                              \
    do {                                                                                                 \
        auto k = ngf_tile_kernel<TYV, MV, TImg>;                                                         \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                  \
        k<<<grid, kThreads, smem, st>>>(a);                                                              \
        return cudaGetLastError();                                                                       \
    } while (0)
#define NGF_TY(TYV)                                     \
    switch (mode) {                                     \
        case MODE_OBJ: NGF_LAUNCH(TYV, MODE_OBJ);       \
        case MODE_LIN: NGF_LAUNCH(TYV, MODE_LIN);       \
        case MODE_GRAD: NGF_LAUNCH(TYV, MODE_GRAD);     \
        case MODE_GRADLIN: NGF_LAUNCH(TYV, MODE_GRADLIN); \
        case MODE_MATVEC: NGF_LAUNCH(TYV, MODE_MATVEC); \
        case MODE_DIAG: NGF_LAUNCH(TYV, MODE_DIAG);     \
        default: return cudaErrorInvalidValue;          \
    }
    switch (a.g.TY) {
        case 8: NGF_TY(8);
        case 16: NGF_TY(16);
        default: return cudaErrorInvalidValue;
    }
#undef NGF_TY
#undef NGF_LAUNCH
}

cudaError_t launch_ngf_tile(int mode, const TileArgs<float> &a, cudaStream_t st) { return launch_mode(mode, a, st); }
cudaError_t launch_ngf_tile(int mode, const TileArgs<__half> &a, cudaStream_t st) { return launch_mode(mode, a, st); }

}  // namespace ngf
