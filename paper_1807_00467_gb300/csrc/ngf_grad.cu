// NGF objective, gradient and Gauss-Newton linearisation (Eq. (1)) in one
// pass over the volume: trilinear warp of the template at y = x + P u (Eq. 11's
// transformation model), central-difference gradients of R and of the warped
// template, the per-voxel residual r and 1 - r^2, the adjoint of the central
// difference and P^T onto the grid nodes.
//
// Same tiling as the GN-product kernel (lane = x column, warp = y row, 2-voxel
// halo, 32-plane z chunks, persistent CTAs walking the tiles), with three
// pipelined stages per plane:
//   W (plane pW): y = x + P u, the FP32 cell decision (fixed operation order,
//                 shared with the oracle), 8 template samples, T(y), dT/dy; R(x)
//   C (plane pW - 1): f = grad R, g = grad T(y), 1 - r^2 in cancellation-free
//                 form, a = dr/dg (stored for the GN product), and
//                 c = d(1 - r^2)/dg scaled by 1/(2h) for the adjoint
//   A (plane pW - 2): adjoint of the central difference of c, times dT/dy,
//                 accumulated onto the column's two z-node planes
// The objective-only pass (ngf_obj_kernel) runs W and C (one plane of z halo)
// and issues each plane's template samples a plane early.  Samples outside
// the volume are placed on clamped cells (zero derivative along a clamped
// axis); voxels that are not interior contribute nothing and get a = 0.
#include "common.cuh"
#include "kernels.h"
#include "node_sweep.cuh"

namespace ngf {

namespace {

constexpr int kTY = 16, kNW = kTY + 4, kNT = 32 * kNW, kEx = kNW * 32;

struct GrSmem {
    int ext, exr, exc, nodes, rows, xr, total;
};

__host__ __device__ inline GrSmem gr_smem(const TileGeom &g, bool adj) {
    GrSmem s;
    int off = 0;
    s.ext = off; off += 2 * kEx;                                    // W value of plane C, double-buffered
    s.exr = off; off += 2 * kEx;                                    // R of plane C
    s.exc = off; off += adj ? 2 * kEx : 0;                          // c'_y of plane A
    s.nodes = off; off += g.nzt * g.nyt * g.nxt * 4;                // node planes of u, [plane][y][x][xyz_]
    s.rows = off; off += adj ? (g.C[2] + 1) * kTY * g.TXI * 3 : 0;  // parked z-node column sums
    s.xr = off; off += adj ? (g.C[2] + 1) * kTY * (g.C[0] + 1) * 3 : 0;
    s.total = off;
    return s;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

}  // namespace

// MODE: MODE_GRAD or MODE_GRADLIN (gradient + stored linearisation); the
// objective-only mode of this kernel is kept for reference, the launcher uses
// ngf_obj_kernel below.
template <int MODE, typename TImg, int RZ>
__global__ void __launch_bounds__(kNT, 1) ngf_grad_kernel(const __grid_constant__ TileArgs<TImg> a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    constexpr bool ADJ = MODE != MODE_OBJ, STORE = MODE == MODE_GRADLIN;
    constexpr int HZ = ADJ ? 2 : 1;   // z halo of stage W
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float smem[];
    const TileGeom &g = a.g;
    const GrSmem S = gr_smem(g, ADJ);

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int TXI = g.TXI, nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int sxy = nx * ny;
    const int N = sxy * nz;
    const int ntiles = g.nb[0] * g.nb[1] * g.nb[2];
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const int rzm = g.rho[2] - 1;
    const float irz = g.irho[2];
    const int nxt = g.nxt, nyt = g.nyt, nplane = nxt * nyt;
    float4 *s_nodes = reinterpret_cast<float4 *>(smem + S.nodes);
    float *rows = smem + S.rows, *xr = smem + S.xr;
    float *ex_t = smem + S.ext + w * 32 + L, *ex_r = smem + S.exr + w * 32 + L, *ex_c = smem + S.exc + w * 32 + L;
    const int up = w > 0 ? -32 : 0, dn = w < kNW - 1 ? 32 : 0;
    const bool own_col = w >= 2 && w < kTY + 2 && L >= 2 && L < TXI + 2;
    float *rowp = rows + ((w - 2) * TXI + (L - 2)) * 3;
    const float ih0 = g.invh[0], ih1 = g.invh[1], ih2 = g.invh[2];
    const float i2h0 = g.inv2h[0], i2h1 = g.inv2h[1], i2h2 = g.inv2h[2], eta2 = g.eta2;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int bx = t % g.nb[0], rr = t / g.nb[0];
        const int x0 = bx * TXI, y0 = (rr % g.nb[1]) * kTY, z0 = (rr / g.nb[1]) * g.TZ;
        const int TZc = min(g.TZ, nz - z0);
        const int nsteps = TZc + 2 * HZ;
        const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry, kz_lo = (z0 - HZ) >> lrz;

        // the previous tile's readers of the node tile, rows and xr are done
        __syncthreads();
        {
            const int mxy = g.m[0] * g.m[1], Mn = mxy * g.m[2];
            for (int i = tid; i < g.nzt * nplane; i += kNT) {
                const int pl = i / nplane, r = i - pl * nplane;
                const int ly = r / nxt, lx = r - ly * nxt;
                const int ux = kx_lo + lx, uy = ky_lo + ly, kz = kz_lo + pl;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ux < g.m[0] && uy < g.m[1] && kz >= 0 && kz < g.m[2]) {
                    const int q = kz * mxy + uy * g.m[0] + ux;
                    v.x = __ldg(a.u + q);
                    v.y = __ldg(a.u + Mn + q);
                    v.z = __ldg(a.u + 2 * Mn + q);
                }
                s_nodes[i] = v;
            }
        }
        // this column: position in the volume and in the node tile (clamped:
        // columns outside the volume are never interior and only need finite values)
        const int gx = x0 - 2 + L, gy = y0 - 2 + w;
        const bool colin = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        const bool intxy = colin && gx >= 1 && gx <= nx - 2 && gy >= 1 && gy <= ny - 2;
        const int col = colin ? gy * nx + gx : 0;
        const int cxg = gx >> lrx, cyg = gy >> lry;
        const float fx = ((gx - (cxg << lrx)) + 0.5f) * g.irho[0];
        const float fy = ((gy - (cyg << lry)) + 0.5f) * g.irho[1];
        const float4 *qcol = s_nodes + min(max(cyg - ky_lo, 0), nyt - 2) * nxt + min(max(cxg - kx_lo, 0), nxt - 2);
        // x, then y, fixed-order FP32 interpolation of node plane kz (the cell decision's definition)
        auto bilinear = [&](int kz, float *U) {
            const float4 *q = qcol + (kz - kz_lo) * nplane;
            const float4 n00 = q[0], n10 = q[1], n01 = q[nxt], n11 = q[nxt + 1];
            const float wx0 = 1.f - fx, wy0 = 1.f - fy;
            U[0] = lerp_fixed(lerp_fixed(n00.x, n10.x, wx0, fx), lerp_fixed(n01.x, n11.x, wx0, fx), wy0, fy);
            U[1] = lerp_fixed(lerp_fixed(n00.y, n10.y, wx0, fx), lerp_fixed(n01.y, n11.y, wx0, fx), wy0, fy);
            U[2] = lerp_fixed(lerp_fixed(n00.z, n10.z, wx0, fx), lerp_fixed(n01.z, n11.z, wx0, fx), wy0, fy);
        };
        __syncthreads();

        float U0[3], U1[3];
        bilinear((z0 - HZ) >> lrz, U0);
        bilinear(((z0 - HZ) >> lrz) + 1, U1);
        float tm = 0.f, t0 = 0.f, rm = 0.f, r0 = 0.f;           // W value and R at planes pC - 1, pC
        float d1[3] = {0.f, 0.f, 0.f}, d2[3] = {0.f, 0.f, 0.f};  // dT/dy at planes pW - 1, pW - 2
        float cxp = 0.f, czm2 = 0.f, czm1 = 0.f;                 // c' of the adjoint (as in the GN product)
        float acc0[3] = {0.f, 0.f, 0.f}, acc1[3] = {0.f, 0.f, 0.f};
        float dsum = 0.f, dcomp = 0.f;

        for (int s0 = 0; s0 < nsteps; s0 += 2) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int s = s0 + j;
                if (s >= nsteps) break;
                const int pW = z0 - HZ + s, pC = pW - 1;
                // z phase of plane pW (z0 is a multiple of rho_z; so is s0 when rho_z divides 2)
                const int phW = RZ ? ((j - HZ) & (RZ - 1)) : (pW & rzm);
                const float fz = RZ ? (phW + 0.5f) / (float)(RZ ? RZ : 1) : (phW + 0.5f) * irz;
                __syncthreads();
                if (phW == 0 && s > 0) {
                    U0[0] = U1[0]; U0[1] = U1[1]; U0[2] = U1[2];
                    bilinear((pW >> lrz) + 1, U1);
                }
                // ------------------------------------------------ stage W: plane pW
                float val, dw[3];
                {
                    const float pu0 = lerp_fixed(U0[0], U1[0], 1.f - fz, fz);
                    const float pu1 = lerp_fixed(U0[1], U1[1], 1.f - fz, fz);
                    const float pu2 = lerp_fixed(U0[2], U1[2], 1.f - fz, fz);
                    // per axis: FP32 cell decision, then the pair (c, c + step) and the
                    // fraction; at and beyond the last voxel the pair (n-1, n-2), step -1
                    int c[3], st[3];
                    float f[3];
                    bool in[3];
                    const float pu[3] = {pu0, pu1, pu2}, ih[3] = {ih0, ih1, ih2};
                    const int ii[3] = {gx, gy, pW}, nn[3] = {nx, ny, nz};
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const float q = __fmul_rn(pu[ax], ih[ax]);
                        const float fl = floorf(q);
                        // fraction: the exact rounding error of the product and the
                        // correction for float(1/h) (invh_rel = 1 - h float(1/h))
                        const float e = __fmaf_rn(pu[ax], ih[ax], -q);
                        const float fr = (q - fl) + __fmaf_rn(q, g.invh_rel[ax], e);
                        const int k = ii[ax] + (int)fl;
                        const bool lo = k < 0, hi = k >= nn[ax] - 1;
                        c[ax] = lo ? 0 : (hi ? nn[ax] - 1 : k);
                        st[ax] = hi ? -1 : 1;
                        in[ax] = !lo && (!hi || (k == nn[ax] - 1 && q - fl == 0.f));
                        f[ax] = (lo || hi) ? 0.f : fr;
                    }
                    const int sx = st[0], sy = st[1] * nx, sz = st[2] * sxy;
                    const TImg *T = a.T + (c[2] * sxy + c[1] * nx + c[0]);
                    const float t000 = ldimg(T, 0), t100 = ldimg(T, sx);
                    const float t010 = ldimg(T, sy), t110 = ldimg(T, sy + sx);
                    const float t001 = ldimg(T, sz), t101 = ldimg(T, sz + sx);
                    const float t011 = ldimg(T, sz + sy), t111 = ldimg(T, sz + sy + sx);
                    const float dx00 = t100 - t000, dx10 = t110 - t010, dx01 = t101 - t001, dx11 = t111 - t011;
                    const float v00 = fmaf(f[0], dx00, t000), v10 = fmaf(f[0], dx10, t010);
                    const float v01 = fmaf(f[0], dx01, t001), v11 = fmaf(f[0], dx11, t011);
                    const float dy0 = v10 - v00, dy1 = v11 - v01;
                    const float w0 = fmaf(f[1], dy0, v00), w1 = fmaf(f[1], dy1, v01);
                    const float dz = w1 - w0;
                    val = fmaf(f[2], dz, w0);
                    if (ADJ) {
                        const float ax0 = fmaf(f[1], dx10 - dx00, dx00), ax1 = fmaf(f[1], dx11 - dx01, dx01);
                        dw[0] = in[0] ? fmaf(f[2], ax1 - ax0, ax0) * ih0 * (float)st[0] : 0.f;
                        dw[1] = in[1] ? fmaf(f[2], dy1 - dy0, dy0) * ih1 * (float)st[1] : 0.f;
                        dw[2] = in[2] ? dz * ih2 * (float)st[2] : 0.f;
                        if (STORE && own_col && colin && pW >= z0 && pW < z0 + TZc) {
                            const int v = pW * sxy + col;
                            a.st_dT[v] = dw[0];
                            a.st_dT[N + v] = dw[1];
                            a.st_dT[2 * N + v] = dw[2];
                        }
                    }
                }
                const float rv = (colin && pW >= 0 && pW < nz) ? ldimg(a.R, pW * sxy + col) : 0.f;

                // ------------------------------------------------ stage C: plane pC
                const int b = (j & 1) * kEx;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                {
                    const float tl = __shfl_up_sync(FULL, t0, 1), tr = __shfl_down_sync(FULL, t0, 1);
                    const float rl = __shfl_up_sync(FULL, r0, 1), rr2 = __shfl_down_sync(FULL, r0, 1);
                    const float g0 = (tr - tl) * i2h0, g1 = (ex_t[b + dn] - ex_t[b + up]) * i2h1, g2 = (val - tm) * i2h2;
                    const float f0 = (rr2 - rl) * i2h0, f1 = (ex_r[b + dn] - ex_r[b + up]) * i2h1, f2 = (rv - rm) * i2h2;
                    // the same operation order for <f,g>, |f|^2, |g|^2: f = g gives equal values
                    const float fg = __fmaf_rn(f2, g2, __fmaf_rn(f1, g1, __fmaf_rn(f0, g0, eta2)));
                    const float ff = __fmaf_rn(f2, f2, __fmaf_rn(f1, f1, __fmaf_rn(f0, f0, eta2)));
                    const float gg = __fmaf_rn(g2, g2, __fmaf_rn(g1, g1, __fmaf_rn(g0, g0, eta2)));
                    const float rff = __frcp_rn(ff), rgg = __frcp_rn(gg);
                    const bool interior = intxy && pC >= 1 && pC <= nz - 2;
                    const bool own = own_col && pC >= z0 && pC < z0 + TZc;
                    // 1 - r^2 = (|f x g|^2 + eta^2 |f - g|^2) / (|f|_eta^2 |g|_eta^2); products
                    // rounded separately: exactly zero when f = g
                    const float x0_ = __fmul_rn(f1, g2) - __fmul_rn(f2, g1);
                    const float x1_ = __fmul_rn(f2, g0) - __fmul_rn(f0, g2);
                    const float x2_ = __fmul_rn(f0, g1) - __fmul_rn(f1, g0);
                    const float e0 = f0 - g0, e1 = f1 - g1, e2 = f2 - g2;
                    const float num = x0_ * x0_ + x1_ * x1_ + x2_ * x2_ + eta2 * (e0 * e0 + e1 * e1 + e2 * e2);
                    kahan_add(dsum, dcomp, (own && interior) ? num * rff * rgg : 0.f);
                    if (ADJ) {
                        // a = dr/dg = (f |g|^2 - <f,g> g) / (|f| |g|^3) (norms with eta);
                        // c = d(1 - r^2)/dg = -2 <f,g> q / (|f|^2 |g|^4), times 1/(2h) per axis
                        const float q0 = __fmul_rn(f0, gg) - __fmul_rn(fg, g0);
                        const float q1 = __fmul_rn(f1, gg) - __fmul_rn(fg, g1);
                        const float q2 = __fmul_rn(f2, gg) - __fmul_rn(fg, g2);
                        const float sc = interior ? -2.f * fg * rff * rgg * rgg : 0.f;
                        c0 = sc * q0 * i2h0; c1 = sc * q1 * i2h1; c2 = sc * q2 * i2h2;
                        if (STORE && own && colin && pC >= 0) {
                            const float inv = interior ? rsqrtf(ff * gg) * rgg : 0.f;
                            const int v = pC * sxy + col;
                            a.st_a[v] = q0 * inv * i2h0;   // a = dr/dg, stored with the scale 1 / (2 h)
                            a.st_a[N + v] = q1 * inv * i2h1;
                            a.st_a[2 * N + v] = q2 * inv * i2h2;
                        }
                    }
                }

                // ------------------------------------------------ stage A: plane pA = pW - 2
                if (ADJ) {
                    const float cxl = __shfl_up_sync(FULL, cxp, 1), cxr = __shfl_down_sync(FULL, cxp, 1);
                    if (s >= 4) {   // planes of the chunk (pA >= z0)
                        const int zl = s - 4, phA = zl & rzm;
                        const float wz1 = (phA + 0.5f) * irz;
                        const float bsum = (cxl - cxr) + (ex_c[b + up] - ex_c[b + dn]) + (czm2 - c2);
                        const float b1 = wz1 * bsum, b0 = bsum - b1;
                        acc0[0] = fmaf(b0, d2[0], acc0[0]); acc0[1] = fmaf(b0, d2[1], acc0[1]); acc0[2] = fmaf(b0, d2[2], acc0[2]);
                        acc1[0] = fmaf(b1, d2[0], acc1[0]); acc1[1] = fmaf(b1, d2[1], acc1[1]); acc1[2] = fmaf(b1, d2[2], acc1[2]);
                        if (phA == rzm) {
                            // node plane zl / rho_z is complete for this column: park it
                            if (own_col) {
                                float *r = rowp + (zl >> lrz) * (kTY * TXI * 3);
                                r[0] = acc0[0]; r[1] = acc0[1]; r[2] = acc0[2];
                            }
                            acc0[0] = acc1[0]; acc0[1] = acc1[1]; acc0[2] = acc1[2];
                            acc1[0] = acc1[1] = acc1[2] = 0.f;
                        }
                    }
                    ex_c[kEx - b] = c1;
                    czm2 = czm1; czm1 = c2;
                    cxp = c0;
                    d2[0] = d1[0]; d2[1] = d1[1]; d2[2] = d1[2];
                    d1[0] = dw[0]; d1[1] = dw[1]; d1[2] = dw[2];
                }
                // ------------------------------------------------ hand over to the next plane
                ex_t[kEx - b] = val;
                ex_r[kEx - b] = rv;
                tm = t0; t0 = val;
                rm = r0; r0 = rv;
            }
        }
        if (ADJ) {
            // the node plane above the chunk's last cell, then P^T along x and y
            if (own_col) {
                float *r = rowp + (TZc >> lrz) * (kTY * TXI * 3);
                r[0] = acc0[0]; r[1] = acc0[1]; r[2] = acc0[2];
            }
            __syncthreads();
            node_reduce_any<kTY, kNT, false>(g.rho[0], g.rho[1], rows, xr, a.boxes + (long)t * 3 * g.box, g.box,
                                             (TZc >> lrz) + 1, 1.f, tid);
        }
        // the tile's sum of 1 - r^2 (FP64 across the threads)
        {
            double v = (double)dsum - (double)dcomp;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
            __shared__ double red[kNW];
            if (L == 0) red[w] = v;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int i = 0; i < kNW; ++i) s += red[i];
                a.dpart[t] = s;
            }
        }
    }
}

// Objective only (line search): stages W and C with one plane of z halo.  The
// template samples of the next W plane (and R) are issued at the end of each
// plane, so that their latency overlaps the barrier.
template <typename TImg, int RZ>
__global__ void __launch_bounds__(kNT, 1) ngf_obj_kernel(const __grid_constant__ TileArgs<TImg> a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    constexpr int HZ = 1;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float smem[];
    const TileGeom &g = a.g;
    const GrSmem S = gr_smem(g, false);

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int TXI = g.TXI, nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int sxy = nx * ny;
    const int ntiles = g.nb[0] * g.nb[1] * g.nb[2];
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const int rzm = g.rho[2] - 1;
    const float irz = g.irho[2];
    const int nxt = g.nxt, nyt = g.nyt, nplane = nxt * nyt;
    float4 *s_nodes = reinterpret_cast<float4 *>(smem + S.nodes);
    float *ex_t = smem + S.ext + w * 32 + L, *ex_r = smem + S.exr + w * 32 + L;
    const int up = w > 0 ? -32 : 0, dn = w < kNW - 1 ? 32 : 0;
    const bool own_col = w >= 2 && w < kTY + 2 && L >= 2 && L < TXI + 2;
    const float ih0 = g.invh[0], ih1 = g.invh[1], ih2 = g.invh[2];
    const float i2h0 = g.inv2h[0], i2h1 = g.inv2h[1], i2h2 = g.inv2h[2], eta2 = g.eta2;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int bx = t % g.nb[0], rr = t / g.nb[0];
        const int x0 = bx * TXI, y0 = (rr % g.nb[1]) * kTY, z0 = (rr / g.nb[1]) * g.TZ;
        const int TZc = min(g.TZ, nz - z0);
        const int nsteps = TZc + 2 * HZ;
        const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry, kz_lo = (z0 - HZ) >> lrz;

        __syncthreads();
        {
            const int mxy = g.m[0] * g.m[1], Mn = mxy * g.m[2];
            for (int i = tid; i < g.nzt * nplane; i += kNT) {
                const int pl = i / nplane, r = i - pl * nplane;
                const int ly = r / nxt, lx = r - ly * nxt;
                const int ux = kx_lo + lx, uy = ky_lo + ly, kz = kz_lo + pl;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ux < g.m[0] && uy < g.m[1] && kz >= 0 && kz < g.m[2]) {
                    const int q = kz * mxy + uy * g.m[0] + ux;
                    v.x = __ldg(a.u + q);
                    v.y = __ldg(a.u + Mn + q);
                    v.z = __ldg(a.u + 2 * Mn + q);
                }
                s_nodes[i] = v;
            }
        }
        const int gx = x0 - 2 + L, gy = y0 - 2 + w;
        const bool colin = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        const bool intxy = colin && gx >= 1 && gx <= nx - 2 && gy >= 1 && gy <= ny - 2;
        const int col = colin ? gy * nx + gx : 0;
        const int cxg = gx >> lrx, cyg = gy >> lry;
        const float fx = ((gx - (cxg << lrx)) + 0.5f) * g.irho[0];
        const float fy = ((gy - (cyg << lry)) + 0.5f) * g.irho[1];
        const float4 *qcol = s_nodes + min(max(cyg - ky_lo, 0), nyt - 2) * nxt + min(max(cxg - kx_lo, 0), nxt - 2);
        auto bilinear = [&](int kz, float *U) {
            const float4 *q = qcol + (kz - kz_lo) * nplane;
            const float4 n00 = q[0], n10 = q[1], n01 = q[nxt], n11 = q[nxt + 1];
            const float wx0 = 1.f - fx, wy0 = 1.f - fy;
            U[0] = lerp_fixed(lerp_fixed(n00.x, n10.x, wx0, fx), lerp_fixed(n01.x, n11.x, wx0, fx), wy0, fy);
            U[1] = lerp_fixed(lerp_fixed(n00.y, n10.y, wx0, fx), lerp_fixed(n01.y, n11.y, wx0, fx), wy0, fy);
            U[2] = lerp_fixed(lerp_fixed(n00.z, n10.z, wx0, fx), lerp_fixed(n01.z, n11.z, wx0, fx), wy0, fy);
        };
        __syncthreads();

        float U0[3], U1[3];
        bilinear((z0 - HZ) >> lrz, U0);
        bilinear(((z0 - HZ) >> lrz) + 1, U1);
        float tm = 0.f, t0 = 0.f, rm = 0.f, r0 = 0.f;
        float dsum = 0.f, dcomp = 0.f;
        // pending samples of the next W plane: the 8 template values, the
        // fractions, and R
        float smp[8], sf[3], srv;
        auto issue_sample = [&](int pW, float fz) {
            const float pu[3] = {lerp_fixed(U0[0], U1[0], 1.f - fz, fz), lerp_fixed(U0[1], U1[1], 1.f - fz, fz),
                                 lerp_fixed(U0[2], U1[2], 1.f - fz, fz)};
            const float ih[3] = {ih0, ih1, ih2};
            const int ii[3] = {gx, gy, pW}, nn[3] = {nx, ny, nz};
            int c[3], st[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                // the same FP32 cell decision and placement as the gradient pass
                const float q = __fmul_rn(pu[ax], ih[ax]);
                const float fl = floorf(q);
                const float e = __fmaf_rn(pu[ax], ih[ax], -q);
                const float fr = (q - fl) + __fmaf_rn(q, g.invh_rel[ax], e);
                const int k = ii[ax] + (int)fl;
                const bool lo = k < 0, hi = k >= nn[ax] - 1;
                c[ax] = lo ? 0 : (hi ? nn[ax] - 1 : k);
                st[ax] = hi ? -1 : 1;
                sf[ax] = (lo || hi) ? 0.f : fr;
            }
            const int sx = st[0], sy = st[1] * nx, sz = st[2] * sxy;
            const TImg *T = a.T + (c[2] * sxy + c[1] * nx + c[0]);
            smp[0] = ldimg(T, 0); smp[1] = ldimg(T, sx); smp[2] = ldimg(T, sy); smp[3] = ldimg(T, sy + sx);
            smp[4] = ldimg(T, sz); smp[5] = ldimg(T, sz + sx); smp[6] = ldimg(T, sz + sy); smp[7] = ldimg(T, sz + sy + sx);
            srv = (colin && pW >= 0 && pW < nz) ? ldimg(a.R, pW * sxy + col) : 0.f;
        };
        issue_sample(z0 - HZ, (((z0 - HZ) & rzm) + 0.5f) * irz);

        for (int s0 = 0; s0 < nsteps; s0 += 2) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int s = s0 + j;
                if (s >= nsteps) break;
                const int pW = z0 - HZ + s, pC = pW - 1;
                __syncthreads();
                // ------------------------------------------------ stage W: plane pW (samples issued before)
                const float rv = srv;
                float val;
                {
                    const float dx00 = smp[1] - smp[0], dx10 = smp[3] - smp[2], dx01 = smp[5] - smp[4], dx11 = smp[7] - smp[6];
                    const float v00 = fmaf(sf[0], dx00, smp[0]), v10 = fmaf(sf[0], dx10, smp[2]);
                    const float v01 = fmaf(sf[0], dx01, smp[4]), v11 = fmaf(sf[0], dx11, smp[6]);
                    const float w0 = fmaf(sf[1], v10 - v00, v00), w1 = fmaf(sf[1], v11 - v01, v01);
                    val = fmaf(sf[2], w1 - w0, w0);
                }
                // ------------------------------------------------ stage C: 1 - r^2 at plane pC
                const int b = (j & 1) * kEx;
                {
                    const float tl = __shfl_up_sync(FULL, t0, 1), tr = __shfl_down_sync(FULL, t0, 1);
                    const float rl = __shfl_up_sync(FULL, r0, 1), rr2 = __shfl_down_sync(FULL, r0, 1);
                    const float g0 = (tr - tl) * i2h0, g1 = (ex_t[b + dn] - ex_t[b + up]) * i2h1, g2 = (val - tm) * i2h2;
                    const float f0 = (rr2 - rl) * i2h0, f1 = (ex_r[b + dn] - ex_r[b + up]) * i2h1, f2 = (rv - rm) * i2h2;
                    const float ff = __fmaf_rn(f2, f2, __fmaf_rn(f1, f1, __fmaf_rn(f0, f0, eta2)));
                    const float gg = __fmaf_rn(g2, g2, __fmaf_rn(g1, g1, __fmaf_rn(g0, g0, eta2)));
                    const float rff = __frcp_rn(ff), rgg = __frcp_rn(gg);
                    const bool interior = intxy && pC >= 1 && pC <= nz - 2;
                    const bool own = own_col && pC >= z0 && pC < z0 + TZc;
                    const float x0_ = __fmul_rn(f1, g2) - __fmul_rn(f2, g1);
                    const float x1_ = __fmul_rn(f2, g0) - __fmul_rn(f0, g2);
                    const float x2_ = __fmul_rn(f0, g1) - __fmul_rn(f1, g0);
                    const float e0 = f0 - g0, e1 = f1 - g1, e2 = f2 - g2;
                    const float num = x0_ * x0_ + x1_ * x1_ + x2_ * x2_ + eta2 * (e0 * e0 + e1 * e1 + e2 * e2);
                    kahan_add(dsum, dcomp, (own && interior) ? num * rff * rgg : 0.f);
                }
                // ------------------------------------------------ hand over to the next plane
                ex_t[kEx - b] = val;
                ex_r[kEx - b] = rv;
                tm = t0; t0 = val;
                rm = r0; r0 = rv;
                if (s + 1 < nsteps) {
                    const int phN = RZ ? ((j + 1 - HZ) & (RZ - 1)) : ((pW + 1) & rzm);
                    if (phN == 0) {
                        U0[0] = U1[0]; U0[1] = U1[1]; U0[2] = U1[2];
                        bilinear(((pW + 1) >> lrz) + 1, U1);
                    }
                    issue_sample(pW + 1, RZ ? (phN + 0.5f) / (float)(RZ ? RZ : 1) : (phN + 0.5f) * irz);
                }
            }
        }
        {
            double v = (double)dsum - (double)dcomp;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
            __shared__ double red[kNW];
            if (L == 0) red[w] = v;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int i = 0; i < kNW; ++i) s += red[i];
                a.dpart[t] = s;
            }
        }
    }
}

bool ngf_grad_supported(const TileGeom &g) {
    if (g.TY != kTY || g.nzt <= 0 || g.rho[0] < 2) return false;
    return (size_t)gr_smem(g, true).total * sizeof(float) <= 227u * 1024u;
}

template <typename TImg>
static cudaError_t launch_grad(int mode, const TileArgs<TImg> &a, cudaStream_t st) {
    if (!ngf_grad_supported(a.g)) return cudaErrorInvalidValue;
    const bool adj = mode != MODE_OBJ;
    const size_t smem = sizeof(float) * (size_t)gr_smem(a.g, adj).total;
    const int ntiles = a.g.nb[0] * a.g.nb[1] * a.g.nb[2];
    const int sms = device_sm_count();
    const int grid = ntiles < sms ? ntiles : sms;
    auto run = [&](auto kernel) {
        cudaError_t e = allow_max_dynamic_smem(kernel);
        if (e != cudaSuccess) return e;
        kernel<<<grid, kNT, smem, st>>>(a);
        return cudaGetLastError();
    };
    const bool r2 = a.g.rho[2] == 2;
    switch (mode) {
        case MODE_OBJ: return r2 ? run(ngf_obj_kernel<TImg, 2>) : run(ngf_obj_kernel<TImg, 0>);
        case MODE_GRAD: return r2 ? run(ngf_grad_kernel<MODE_GRAD, TImg, 2>) : run(ngf_grad_kernel<MODE_GRAD, TImg, 0>);
        case MODE_GRADLIN:
        case MODE_LIN:
            return r2 ? run(ngf_grad_kernel<MODE_GRADLIN, TImg, 2>) : run(ngf_grad_kernel<MODE_GRADLIN, TImg, 0>);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ngf_grad(int mode, const TileArgs<float> &a, cudaStream_t st) { return launch_grad(mode, a, st); }
cudaError_t launch_ngf_grad(int mode, const TileArgs<__half> &a, cudaStream_t st) { return launch_grad(mode, a, st); }

}  // namespace ngf
