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
//  - dT/dy and a of every plane arrive by TMA into a 6-stage ring (3 planes
//    ahead); planes outside the volume are zero-filled by the TMA unit, and a
//    is zero on the volume's boundary voxels, so no voxel needs a predicate:
//    zeros propagate to exactly the terms the adjoint leaves out;
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
constexpr int kStages = 6;                // TMA ring depth (planes)
constexpr int kAhead = 3;                 // planes in flight ahead of stage W
constexpr int kBoxF = ((kTmaBoxX * kNW * 3 * 4 + 127) / 128) * 32;   // floats per box, 128-byte padded
constexpr int kStageF = 2 * kBoxF;        // dT/dy box, then a box
constexpr int kComp = kNW * kTmaBoxX;     // floats between components in a box
constexpr uint32_t kPlaneBytes = 2u * kTmaBoxX * kNW * 3 * 4;

struct MvSmem {
    int tma, ext, exc, nodes, rows, xr, total;
};

__host__ __device__ inline MvSmem mv_smem(const TileGeom &g) {
    MvSmem s;
    int off = 0;
    s.tma = off; off += kStages * kStageF + 32;          // + 128 bytes to align the base
    s.ext = off; off += 2 * kNW * 32;                     // t of plane C, double-buffered
    s.exc = off; off += 2 * kNW * 32;                     // c_y of plane A, double-buffered
    s.nodes = off; off += g.nzt * 3 * g.nxt * g.nyt;      // node planes of P v
    s.rows = off; off += (g.C[2] + 1) * kTY * g.TXI * 3;  // z-reduced column sums per node plane
    s.xr = (g.C[2] + 1) * kTY * (g.C[0] + 1) * 3;         // x-reduced sums (reuse the TMA ring)
    s.total = off;
    return s;
}

}  // namespace

bool gn_matvec_supported(const TileGeom &g) {
    if (!g.tma || g.TY != kTY || g.nzt <= 0 || g.rho[0] < 2) return false;
    const MvSmem s = mv_smem(g);
    return s.xr <= kStages * kStageF && (size_t)s.total * sizeof(float) <= 227u * 1024u;
}

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
    float *ext = smem + S.ext, *exc = smem + S.exc, *s_nodes = smem + S.nodes, *rows = smem + S.rows;

    // plane j of the chunk's sequence (voxel plane z0 - 2 + j) into stage j % kStages
    auto issue_plane = [&](int j) {
        const int st = j % kStages;
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

    // node planes of v for P v (zero beyond the grid)
    const int nxt = g.nxt, nyt = g.nyt, nzt = g.nzt, nplane = nxt * nyt;
    const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry, kz_lo = max(z0 - 2, 0) >> lrz;
    {
        const long mxy = (long)g.m[0] * g.m[1], Mn = mxy * g.m[2];
        for (int i = tid; i < nzt * 3 * nplane; i += kNT) {
            const int pl = i / nplane, r = i - pl * nplane;   // pl = plane * 3 + comp
            const int kz = kz_lo + pl / 3, comp = pl - (pl / 3) * 3;
            const int ly = r / nxt, lx = r - ly * nxt;
            const int ux = kx_lo + lx, uy = ky_lo + ly;
            float v = 0.f;
            if (ux < g.m[0] && uy < g.m[1] && kz < g.m[2]) v = __ldg(a.u + comp * Mn + (long)kz * mxy + (long)uy * g.m[0] + ux);
            s_nodes[i] = v;
        }
    }

    // this column's bilinear position in the node tile (clamped: columns
    // outside the volume have dT/dy = 0 and only need finite values)
    const int gx = x0 - 2 + L, gy = y0 - 2 + w;
    const int cxg = gx >> lrx, cyg = gy >> lry;
    const float fx = ((gx - (cxg << lrx)) + 0.5f) * g.irho[0];
    const float fy = ((gy - (cyg << lry)) + 0.5f) * g.irho[1];
    const float *qcol = s_nodes + min(max(cyg - ky_lo, 0), nyt - 2) * nxt + min(max(cxg - kx_lo, 0), nxt - 2);
    auto bilinear = [&](int kz, int comp) {
        const float *q = qcol + ((kz - kz_lo) * 3 + comp) * nplane;
        const float lo = fmaf(fx, q[1] - q[0], q[0]);
        const float hi = fmaf(fx, q[nxt + 1] - q[nxt], q[nxt]);
        return fmaf(fy, hi - lo, lo);
    };

    const float i2h0 = g.inv2h[0], i2h1 = g.inv2h[1], i2h2 = g.inv2h[2];
    const bool rowC = w >= 1 && w < kNW - 1;          // rows whose c is needed
    const bool rowA = w >= 2 && w < kTY + 2;          // rows owned by the tile
    const bool colA = L >= 2 && L < TXI + 2;          // columns owned by the tile
    const int o = w * kTmaBoxX + L + 2;               // this column in a TMA box
    const int ex_me = w * 32 + L;

    float U0[3] = {0.f, 0.f, 0.f}, D[3] = {0.f, 0.f, 0.f};   // P v at node planes cz, cz + 1 (x-y interpolated)
    int cur_cz = -1000;
    float tm = 0.f, t0 = 0.f;          // t at planes pC - 1, pC
    float cxp = 0.f;                   // c'_x at plane pA (from the previous plane's stage C)
    float czm2 = 0.f, czm1 = 0.f;      // c'_z at planes pA - 1, pA
    float acc0[3] = {0.f, 0.f, 0.f}, acc1[3] = {0.f, 0.f, 0.f};   // z-node planes czl, czl + 1

    int stW = 0;            // stage of plane s
    uint32_t phW = 0;       // its phase parity
    for (int s = 0; s < nsteps; ++s) {
        const int pW = z0 - 2 + s, pA = pW - 2;
        const int b = s & 1;
        const int stC = stW == 0 ? kStages - 1 : stW - 1;
        const int stA = stC == 0 ? kStages - 1 : stC - 1;
        // the stage of plane s - 3 was last read before this barrier (at s = 0 it
        // publishes the barrier initialisation and the node planes)
        __syncthreads();
        if (tid == 0 && s + kAhead < nsteps) issue_plane(s + kAhead);

        // ------------------------------------------------ P v at plane pW (node planes on change)
        const int cz = min(max(pW >> lrz, kz_lo), kz_lo + nzt - 2);
        if (cz != cur_cz) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float u0 = cz == cur_cz + 1 ? U0[k] + D[k] : bilinear(cz, k);
                const float u1 = bilinear(cz + 1, k);
                U0[k] = u0;
                D[k] = u1 - u0;
            }
            cur_cz = cz;
        }
        const float fz = ((pW & rzm) + 0.5f) * irz;

        mbar_wait_bounded(&bars[stW], phW, a.err);
        const float *sW = tma_base + stW * kStageF;
        // ------------------------------------------------ stage W: t at plane pW
        const float tp = sW[o] * fmaf(fz, D[0], U0[0]) + sW[kComp + o] * fmaf(fz, D[1], U0[1]) +
                         sW[2 * kComp + o] * fmaf(fz, D[2], U0[2]);

        // ------------------------------------------------ stage C: c' at plane pC = pW - 1
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
        {
            const float txl = __shfl_up_sync(FULL, t0, 1), txr = __shfl_down_sync(FULL, t0, 1);
            if (rowC) {
                const float *e = ext + b * kNW * 32 + ex_me;
                const float *sC = tma_base + stC * kStageF + kBoxF;
                const float a0 = sC[o] * i2h0, a1 = sC[kComp + o] * i2h1, a2 = sC[2 * kComp + o] * i2h2;
                const float dr = fmaf(a2, tp - tm, fmaf(a1, e[32] - e[-32], a0 * (txr - txl)));
                c0 = dr * a0;
                c1 = dr * a1;
                c2 = dr * a2;
            }
        }
        // ------------------------------------------------ stage A: G^T c at plane pA, times dT/dy
        {
            const float cxl = __shfl_up_sync(FULL, cxp, 1), cxr = __shfl_down_sync(FULL, cxp, 1);
            if (rowA && pA >= z0) {
                const float *e = exc + b * kNW * 32 + ex_me;
                const float bsum = (cxl - cxr) + (e[-32] - e[32]) + (czm2 - c2);
                const float *sA = tma_base + stA * kStageF;
                const int zl = pA - z0, ph = zl & rzm;
                const float wz1 = (ph + 0.5f) * irz;
                const float b1 = wz1 * bsum, b0 = bsum - b1;
                const float d0 = sA[o], d1 = sA[kComp + o], d2 = sA[2 * kComp + o];
                acc0[0] = fmaf(b0, d0, acc0[0]); acc0[1] = fmaf(b0, d1, acc0[1]); acc0[2] = fmaf(b0, d2, acc0[2]);
                acc1[0] = fmaf(b1, d0, acc1[0]); acc1[1] = fmaf(b1, d1, acc1[1]); acc1[2] = fmaf(b1, d2, acc1[2]);
                if (ph == rzm) {
                    // node plane zl >> lrz is complete for this column: park it
                    if (colA) {
                        float *r = rows + (((zl >> lrz) * kTY + (w - 2)) * TXI + (L - 2)) * 3;
                        r[0] = acc0[0]; r[1] = acc0[1]; r[2] = acc0[2];
                    }
                    acc0[0] = acc1[0]; acc0[1] = acc1[1]; acc0[2] = acc1[2];
                    acc1[0] = acc1[1] = acc1[2] = 0.f;
                }
            }
        }
        // ------------------------------------------------ hand over to the next plane
        ext[(b ^ 1) * kNW * 32 + ex_me] = tp;
        exc[(b ^ 1) * kNW * 32 + ex_me] = c1;
        tm = t0; t0 = tp;
        czm2 = czm1; czm1 = c2;
        cxp = c0;
        if (++stW == kStages) { stW = 0; phW ^= 1u; }
    }
    // the node plane above the chunk's last cell
    if (rowA && colA) {
        float *r = rows + (((TZc >> lrz) * kTY + (w - 2)) * TXI + (L - 2)) * 3;
        r[0] = acc0[0]; r[1] = acc0[1]; r[2] = acc0[2];
    }
    __syncthreads();

    // ---------------------------------------------------- x then y reduction onto the CTA's node box
    const int CX = g.C[0], CY = g.C[1], rxm = g.rho[0] - 1, rym = g.rho[1] - 1;
    const int nplanes = (TZc >> lrz) + 1;
    float *xr = tma_base;   // [plane][ty][jx][comp]; every TMA copy has completed
    for (int e = tid; e < nplanes * kTY * (CX + 1) * 3; e += kNT) {
        const int k = e % 3, t1 = e / 3, jx = t1 % (CX + 1), t2 = t1 / (CX + 1);   // t2 = plane * kTY + ty
        const int lo = max(0, (jx - 1) << lrx), hi = min(TXI, (jx + 1) << lrx);
        const float *r = rows + (long)t2 * TXI * 3 + k;
        float v = 0.f;
        for (int tx = lo; tx < hi; ++tx) {
            float wx = ((tx & rxm) + 0.5f) * g.irho[0];
            if ((tx >> lrx) == jx) wx = 1.f - wx;
            v = fmaf(wx, r[tx * 3], v);
        }
        xr[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < 3 * nplanes * (CY + 1) * (CX + 1); e += kNT) {
        const int jx = e % (CX + 1), t1 = e / (CX + 1), jy = t1 % (CY + 1), t2 = t1 / (CY + 1);
        const int jz = t2 % nplanes, comp = t2 / nplanes;
        const int lo = max(0, (jy - 1) << lry), hi = min(kTY, (jy + 1) << lry);
        float v = 0.f;
        for (int ty = lo; ty < hi; ++ty) {
            float wy = ((ty & rym) + 0.5f) * g.irho[1];
            if ((ty >> lry) == jy) wy = 1.f - wy;
            v = fmaf(wy, xr[((jz * kTY + ty) * (CX + 1) + jx) * 3 + comp], v);
        }
        a.boxes[((long)cta * 3 + comp) * g.box + (jz * (CY + 1) + jy) * (CX + 1) + jx] = 2.f * v;
    }
}

cudaError_t launch_gn_matvec(const TileArgs<float> &a, cudaStream_t st) {
    if (!gn_matvec_supported(a.g)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)mv_smem(a.g).total;
    cudaError_t e = cudaFuncSetAttribute(gn_matvec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gn_matvec_kernel<<<dim3(a.g.nb[0], a.g.nb[1], a.g.nb[2]), kNT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ngf
