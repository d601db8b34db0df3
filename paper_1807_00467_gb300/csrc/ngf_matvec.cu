// Gauss-Newton product of the NGF term, 2 hbar P^T J^T J P v (Eqs. (1), (11)),
// from the stored linearisation: dT/dy (the template gradient at the warped
// voxel) and a = dr/dg (the derivative of the NGF residual r w.r.t. the
// template gradient), one value per voxel and component.
//
// Per voxel x:  t(x)  = dT/dy(x) . (P v)(x)              (stage W)
//               c(x)  = 2 (a(x) . G t(x)) a(x)            (stage C, G = central differences)
//               z(x)  = (G^T c)(x) dT/dy(x)               (stage A)
// and the product is 2 hbar P^T z.
//
// The layout follows the general NGF tile kernel (lane = x column, warp = y
// row, 2-voxel halo, a chunk of TZ planes marched in z) with the GN-product
// specialisation:
//  - dT/dy and a of every plane arrive by TMA into a 4-stage ring (3 planes
//    ahead); planes outside the volume are zero-filled by the TMA unit, and a
//    is zero on the volume's boundary voxels, so no voxel needs a predicate:
//    zeros propagate to exactly the terms the adjoint leaves out;
//  - stage W reads both fields of its plane once; stages C and A take them
//    from registers one and two planes later, so a stage is free as soon as
//    stage W is done with it;
//  - the plane loop is unrolled by the ring depth: stage offsets, exchange
//    buffers and (for rho_z <= 4) the prolongation weights are constants, and
//    the per-plane register rings are renamings;
//  - one barrier per plane: the y-neighbour exchanges of t (for stage C) and
//    of c_y (for stage A) both use a double-buffered row written at the end of
//    the previous plane;
//  - the central-difference scale 1/(2h) is folded into a once per voxel
//    (a'_i = a_i / (2 h_i)), so stage C forms (a'.dt) a' and stage A sums
//    plain differences; the overall factor 2 x 2 / 4 leaves a factor 2 that is
//    applied once per node;
//  - P^T: each column accumulates its two z-node planes in registers and parks
//    a completed node plane in shared memory; the x and y reductions (hat
//    weights of the trilinear prolongation) run once per chunk.
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ngf {

namespace {

constexpr int kTY = 16;                   // voxel rows per tile
constexpr int kNW = kTY + 4;              // warps (rows incl. the 2-row halos)
constexpr int kNT = 32 * kNW;
constexpr int kStages = 4;                // TMA ring depth (planes) = loop unroll
constexpr int kAhead = 3;                 // planes in flight ahead of stage W
constexpr int kBoxF = ((kTmaBoxX * kNW * 3 * 4 + 127) / 128) * 32;   // floats per box, 128-byte padded
constexpr int kStageF = 2 * kBoxF;        // dT/dy box, then a box
constexpr int kComp = kNW * kTmaBoxX;     // floats between components in a box
constexpr int kEx = kNW * 32;             // floats per exchange row buffer
constexpr uint32_t kPlaneBytes = 2u * kTmaBoxX * kNW * 3 * 4;

struct MvSmem {
    int tma, ext, exc, nodes, rows, xr, total;
};

__host__ __device__ inline MvSmem mv_smem(const TileGeom &g) {
    MvSmem s;
    int off = 0;
    s.tma = off; off += kStages * kStageF + 32;          // + 128 bytes to align the base
    s.ext = off; off += 2 * kEx;                          // t of plane C, double-buffered
    s.exc = off; off += 2 * kEx;                          // c'_y of plane A, double-buffered
    s.nodes = off; off += g.nzt * g.nyt * g.nxt * 4;      // node planes of v, [plane][y][x][xyz_]
    s.rows = off; off += (g.C[2] + 1) * kTY * g.TXI * 3;  // z-reduced column sums per node plane
    s.xr = (g.C[2] + 1) * kTY * (g.C[0] + 1) * 3;         // x-reduced sums (reuse the TMA ring)
    s.total = off;
    return s;
}

// P^T along one axis for node j and every node plane p < np:
// dst[p dpl] = scale sum_i w_i src[p spl + (j - 1) R + i] (source index times sstride),
// i in [0, 2R), with the trilinear hat weights w_i of the ratio R and the
// source indices outside [0, nsrc) left out.
template <int R>
__device__ __forceinline__ void hat_sum(const float *src, int sstride, int spl, int j, int nsrc, float *dst, int dpl,
                                        int np, float scale) {
    float w[2 * R];
    int off[2 * R];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        const int c = (j - 1) * R + i;
        w[i] = (c >= 0 && c < nsrc) ? (i < R ? (i + 0.5f) / R : 1.f - (i - R + 0.5f) / R) : 0.f;
        off[i] = min(max(c, 0), nsrc - 1) * sstride;
    }
    for (int p = 0; p < np; ++p) {
        const float *q = src + p * spl;
        float v = 0.f;
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) v = fmaf(w[i], q[off[i]], v);
        dst[p * dpl] = scale * v;
    }
}

__device__ __forceinline__ void hat_sum_any(int R, const float *src, int sstride, int spl, int j, int nsrc, float *dst,
                                            int dpl, int np, float scale) {
    switch (R) {
        case 1: hat_sum<1>(src, sstride, spl, j, nsrc, dst, dpl, np, scale); break;
        case 2: hat_sum<2>(src, sstride, spl, j, nsrc, dst, dpl, np, scale); break;
        case 4: hat_sum<4>(src, sstride, spl, j, nsrc, dst, dpl, np, scale); break;
        default: hat_sum<8>(src, sstride, spl, j, nsrc, dst, dpl, np, scale); break;
    }
}

template <int RZ>
__global__ void __launch_bounds__(kNT, 1) gn_matvec_kernel(const __grid_constant__ TileArgs<float> a) {
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    const TileGeom &g = a.g;
    const MvSmem S = mv_smem(g);

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int TXI = g.TXI;
    const int x0 = blockIdx.x * TXI, y0 = blockIdx.y * kTY, z0 = blockIdx.z * g.TZ;
    const int TZc = min(g.TZ, g.n[2] - z0);
    const int nsteps = TZc + 4;
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const int rzm = g.rho[2] - 1;
    const float irz = g.irho[2];
    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;

    float *tma_base = smem + S.tma + ((128u - (smem_u32(smem + S.tma) & 127u)) & 127u) / 4;
    float *rows = smem + S.rows;
    float4 *s_nodes = reinterpret_cast<float4 *>(smem + S.nodes);

    // plane j of the chunk's sequence (voxel plane z0 - 2 + j) into stage j % kStages
    auto issue_plane = [&](int j) {
        const int st = j & (kStages - 1);
        float *dst = tma_base + st * kStageF;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[st], kPlaneBytes);
        tma_load_4d(dst, &a.map_dT, &bars[st], x0 - 4, y0 - 2, z0 - 2 + j, 0);
        tma_load_4d(dst + kBoxF, &a.map_a, &bars[st], x0 - 4, y0 - 2, z0 - 2 + j, 0);
    };
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int j = 0; j < kAhead && j < nsteps; ++j) issue_plane(j);
    }

    // node planes of v for P v, from floor((z0 - 2) / rho_z) on (zero outside the grid)
    const int nxt = g.nxt, nyt = g.nyt, nplane = nxt * nyt;
    const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry, kz_lo = (z0 - 2) >> lrz;
    {
        const long mxy = (long)g.m[0] * g.m[1], Mn = mxy * g.m[2];
        for (int i = tid; i < g.nzt * nplane; i += kNT) {
            const int pl = i / nplane, r = i - pl * nplane;
            const int ly = r / nxt, lx = r - ly * nxt;
            const int ux = kx_lo + lx, uy = ky_lo + ly, kz = kz_lo + pl;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ux < g.m[0] && uy < g.m[1] && kz >= 0 && kz < g.m[2]) {
                const long q = (long)kz * mxy + (long)uy * g.m[0] + ux;
                v.x = __ldg(a.u + q);
                v.y = __ldg(a.u + Mn + q);
                v.z = __ldg(a.u + 2 * Mn + q);
            }
            s_nodes[i] = v;
        }
    }

    // this column's bilinear position in the node tile (clamped: columns
    // outside the volume have dT/dy = 0 and only need finite values)
    const int gx = x0 - 2 + L, gy = y0 - 2 + w;
    const int cxg = gx >> lrx, cyg = gy >> lry;
    const float fx = ((gx - (cxg << lrx)) + 0.5f) * g.irho[0];
    const float fy = ((gy - (cyg << lry)) + 0.5f) * g.irho[1];
    const float4 *qcol = s_nodes + min(max(cyg - ky_lo, 0), nyt - 2) * nxt + min(max(cxg - kx_lo, 0), nxt - 2);
    auto bilinear = [&](int kz, float *U) {
        const float4 *q = qcol + (kz - kz_lo) * nplane;
        const float4 n00 = q[0], n10 = q[1], n01 = q[nxt], n11 = q[nxt + 1];
        float lo = fmaf(fx, n10.x - n00.x, n00.x), hi = fmaf(fx, n11.x - n01.x, n01.x);
        U[0] = fmaf(fy, hi - lo, lo);
        lo = fmaf(fx, n10.y - n00.y, n00.y); hi = fmaf(fx, n11.y - n01.y, n01.y);
        U[1] = fmaf(fy, hi - lo, lo);
        lo = fmaf(fx, n10.z - n00.z, n00.z); hi = fmaf(fx, n11.z - n01.z, n01.z);
        U[2] = fmaf(fy, hi - lo, lo);
    };

    const float i2h0 = g.inv2h[0], i2h1 = g.inv2h[1], i2h2 = g.inv2h[2];
    const bool own_col = w >= 2 && w < kTY + 2 && L >= 2 && L < TXI + 2;   // tile-owned column
    const float *sbase = tma_base + w * kTmaBoxX + L + 2;                  // this column in a TMA box
    // y-neighbours in the exchange rows (the outermost rows read themselves; unused)
    float *ex_t = smem + S.ext + w * 32 + L, *ex_c = smem + S.exc + w * 32 + L;
    const int up = w > 0 ? -32 : 0, dn = w < kNW - 1 ? 32 : 0;
    float *rowp = rows + ((w - 2) * TXI + (L - 2)) * 3;    // + node plane * kTY * TXI * 3

    __syncthreads();

    float U0[3], U1[3], D[3];   // P v at node planes cz, cz + 1 (x-y interpolated), D = U1 - U0
    {
        const int cz = (z0 - 2) >> lrz;
        bilinear(cz, U0);
        bilinear(cz + 1, U1);
        for (int k = 0; k < 3; ++k) D[k] = U1[k] - U0[k];
    }
    float tm = 0.f, t0 = 0.f;                  // t at planes pC - 1, pC
    float a1[3] = {0.f, 0.f, 0.f};             // a' at plane pC (read by stage W one plane earlier)
    float d1[3] = {0.f, 0.f, 0.f}, d2[3] = {0.f, 0.f, 0.f};   // dT/dy at planes pW - 1 (= pC), pW - 2 (= pA)
    float cxp = 0.f;                           // c'_x at plane pA (from the previous plane's stage C)
    float czm2 = 0.f, czm1 = 0.f;              // c'_z at planes pA - 1, pA
    float acc0[3] = {0.f, 0.f, 0.f}, acc1[3] = {0.f, 0.f, 0.f};   // z-node planes czl, czl + 1

    uint32_t phase = 0;
    for (int s0 = 0; s0 < nsteps; s0 += kStages, phase ^= 1u) {
#pragma unroll
        for (int j = 0; j < kStages; ++j) {
            const int s = s0 + j;
            if (s >= nsteps) break;
            const int pW = z0 - 2 + s;
            // z phase of planes pW and pA = pW - 2 within their cells (z0 is a
            // multiple of rho_z; so is s0 when rho_z divides the ring depth)
            const int phW = RZ ? ((j - 2) & (RZ - 1)) : (pW & rzm);
            const int phA = RZ ? (j & (RZ - 1)) : ((pW - 2) & rzm);
            const float fz = RZ ? (phW + 0.5f) / (float)(RZ ? RZ : 1) : (phW + 0.5f) * irz;
            const float wz1 = RZ ? (phA + 0.5f) / (float)(RZ ? RZ : 1) : (phA + 0.5f) * irz;

            // the stage of plane s - 1 was last read before this barrier
            __syncthreads();
            if (tid == 0 && s + kAhead < nsteps) issue_plane(s + kAhead);

            // ------------------------------------------------ P v: next node plane at a cell start
            if (phW == 0 && s > 0) {
                U0[0] = U1[0]; U0[1] = U1[1]; U0[2] = U1[2];
                bilinear((pW >> lrz) + 1, U1);
                D[0] = U1[0] - U0[0]; D[1] = U1[1] - U0[1]; D[2] = U1[2] - U0[2];
            }

            mbar_wait_bounded(&bars[j], phase, a.err);
            // ------------------------------------------------ stage W: t at plane pW
            const float *sW = sbase + j * kStageF;
            const float dw0 = sW[0], dw1 = sW[kComp], dw2 = sW[2 * kComp];
            const float aw0 = sW[kBoxF] * i2h0, aw1 = sW[kBoxF + kComp] * i2h1, aw2 = sW[kBoxF + 2 * kComp] * i2h2;
            const float tp = fmaf(dw2, fmaf(fz, D[2], U0[2]), fmaf(dw1, fmaf(fz, D[1], U0[1]), dw0 * fmaf(fz, D[0], U0[0])));

            // ------------------------------------------------ stage C: c' at plane pC = pW - 1
            const int b = (j & 1) * kEx;
            const float txl = __shfl_up_sync(FULL, t0, 1), txr = __shfl_down_sync(FULL, t0, 1);
            const float dr = fmaf(a1[2], tp - tm, fmaf(a1[1], ex_t[b + dn] - ex_t[b + up], a1[0] * (txr - txl)));
            const float c0 = dr * a1[0], c1 = dr * a1[1], c2 = dr * a1[2];

            // ------------------------------------------------ stage A: G^T c at plane pA = pW - 2, times dT/dy
            const float cxl = __shfl_up_sync(FULL, cxp, 1), cxr = __shfl_down_sync(FULL, cxp, 1);
            if (j >= 4 || s0 > 0) {   // planes of the chunk (pA >= z0)
                const float bsum = (cxl - cxr) + (ex_c[b + up] - ex_c[b + dn]) + (czm2 - c2);
                const float b1 = wz1 * bsum, b0 = bsum - b1;
                acc0[0] = fmaf(b0, d2[0], acc0[0]); acc0[1] = fmaf(b0, d2[1], acc0[1]); acc0[2] = fmaf(b0, d2[2], acc0[2]);
                acc1[0] = fmaf(b1, d2[0], acc1[0]); acc1[1] = fmaf(b1, d2[1], acc1[1]); acc1[2] = fmaf(b1, d2[2], acc1[2]);
                if (phA == (RZ ? RZ - 1 : rzm)) {
                    // node plane (pA - z0) / rho_z is complete for this column: park it
                    if (own_col) {
                        float *r = rowp + ((s - 4) >> lrz) * (kTY * TXI * 3);
                        r[0] = acc0[0]; r[1] = acc0[1]; r[2] = acc0[2];
                    }
                    acc0[0] = acc1[0]; acc0[1] = acc1[1]; acc0[2] = acc1[2];
                    acc1[0] = acc1[1] = acc1[2] = 0.f;
                }
            }
            // ------------------------------------------------ hand over to the next plane
            ex_t[kEx - b] = tp;
            ex_c[kEx - b] = c1;
            tm = t0; t0 = tp;
            czm2 = czm1; czm1 = c2;
            cxp = c0;
            d2[0] = d1[0]; d2[1] = d1[1]; d2[2] = d1[2];
            d1[0] = dw0; d1[1] = dw1; d1[2] = dw2;
            a1[0] = aw0; a1[1] = aw1; a1[2] = aw2;
        }
    }
    // the node plane above the chunk's last cell
    if (own_col) {
        float *r = rowp + (TZc >> lrz) * (kTY * TXI * 3);
        r[0] = acc0[0]; r[1] = acc0[1]; r[2] = acc0[2];
    }
    __syncthreads();

    // ---------------------------------------------------- x then y reduction onto the CTA's node box
    // (each thread keeps one (row, node, component) and walks the node planes)
    const int CX = g.C[0], CY = g.C[1];
    const int nplanes = (TZc >> lrz) + 1;
    float *xr = tma_base;   // [plane][ty][jx][comp]; every TMA copy has completed
    for (int e = tid; e < kTY * (CX + 1) * 3; e += kNT) {
        const int k = e % 3, t = e / 3, jx = t % (CX + 1), ty = t / (CX + 1);
        const float *src = rows + ty * TXI * 3 + k;
        float *dst = xr + (ty * (CX + 1) + jx) * 3 + k;
        hat_sum_any(g.rho[0], src, 3, kTY * TXI * 3, jx, TXI, dst, kTY * (CX + 1) * 3, nplanes, 1.f);
    }
    __syncthreads();
    {
        const int nc = (CY + 1) * (CX + 1) * 3, G = max(1, kNT / nc);
        for (int e = tid; e < nc * G; e += kNT) {
            const int c = e % nc, pg = e / nc;
            const int k = c % 3, t = c / 3, jx = t % (CX + 1), jy = t / (CX + 1);
            const float *src = xr + pg * kTY * (CX + 1) * 3 + jx * 3 + k;
            float *dst = a.boxes + ((long)cta * 3 + k) * g.box + (pg * (CY + 1) + jy) * (CX + 1) + jx;
            hat_sum_any(g.rho[1], src, (CX + 1) * 3, G * kTY * (CX + 1) * 3, jy, kTY, dst, G * (CY + 1) * (CX + 1),
                        (nplanes - pg + G - 1) / G, 2.f);
        }
    }
}

}  // namespace

bool gn_matvec_supported(const TileGeom &g) {
    if (!g.tma || g.TY != kTY || g.nzt <= 0 || g.rho[0] < 2) return false;
    const MvSmem s = mv_smem(g);
    return s.xr <= kStages * kStageF && (size_t)s.total * sizeof(float) <= 227u * 1024u;
}

cudaError_t launch_gn_matvec(const TileArgs<float> &a, cudaStream_t st) {
    if (!gn_matvec_supported(a.g)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)mv_smem(a.g).total;
    const dim3 grid(a.g.nb[0], a.g.nb[1], a.g.nb[2]);
    auto run = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kernel<<<grid, kNT, smem, st>>>(a);
        return cudaGetLastError();
    };
    switch (a.g.rho[2]) {
        case 1: return run(gn_matvec_kernel<1>);
        case 2: return run(gn_matvec_kernel<2>);
        case 4: return run(gn_matvec_kernel<4>);
        default: return run(gn_matvec_kernel<0>);   // rho_z = 8: phases from the plane index
    }
}

}  // namespace ngf
