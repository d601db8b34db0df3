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
//  - the central-difference scale 1/(2h) is folded into a when the
//    linearisation stores it (a'_i = a_i / (2 h_i)), so stage C forms (a'.dt) a' and stage A sums
//    plain differences; the overall factor 2 x 2 / 4 leaves a factor 2 that is
//    applied once per node;
//  - P^T: each column accumulates its two z-node planes in registers and parks
//    a completed node plane in shared memory; the x and y reductions (hat
//    weights of the trilinear prolongation) run once per chunk as row sweeps;
//  - persistent CTAs: each CTA walks tiles strided by the grid and its TMA
//    plane sequence continues into the next tile, whose first planes and node
//    tile are fetched during the current tile's reduction.
#include "common.cuh"
#include "kernels.h"
#include "node_sweep.cuh"
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
    s.xr = off; off += (g.C[2] + 1) * kTY * (g.C[0] + 1) * 3;   // x-reduced sums
    s.total = off;
    return s;
}

// DG = false: the GN product (stages W, C, A above).  DG = true: the Jacobi
// diagonal of 2 hbar J^T J with the cross terms of the central-difference
// adjoint left out: per voxel beta = sum_a (a'_a^2 at x - e_a and x + e_a) with
// a' = a / (2 h), times (dT/dy)_k^2, onto the nodes with squared hat weights.
// It reuses the pipeline: stage C forms a'^2 instead of c', stage A sums
// instead of differencing, and P v is not needed.
template <int RZ, bool DG>
__global__ void __launch_bounds__(kNT, 1) gn_matvec_kernel(const __grid_constant__ TileArgs<float> a, int chain) {
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    const TileGeom &g = a.g;
    const MvSmem S = mv_smem(g);

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int TXI = g.TXI;
    const int ntiles = g.nb[0] * g.nb[1] * g.nb[2];
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const int rzm = g.rho[2] - 1;
    const float irz = g.irho[2];

    float *tma_base = smem + S.tma + ((128u - (smem_u32(smem + S.tma) & 127u)) & 127u) / 4;
    float *rows = smem + S.rows, *xr = smem + S.xr;
    float4 *s_nodes = reinterpret_cast<float4 *>(smem + S.nodes);

    // tile t: voxel origin (x0, y0, z0); tiles are numbered x fastest, then y, then z
    auto origin = [&](int t, int &x0, int &y0, int &z0) {
        const int bx = t % g.nb[0], r = t / g.nb[0];
        x0 = bx * TXI;
        y0 = (r % g.nb[1]) * kTY;
        z0 = (r / g.nb[1]) * g.TZ;
    };
    // plane j of tile (x0, y0, z0) (voxel plane z0 - 2 + j) into stage `st`
    auto issue_plane = [&](int x0, int y0, int z0, int j, int st) {
        if (a.no_tma) return;   // test hook: the waits run out instead
        float *dst = tma_base + st * kStageF;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[st], kPlaneBytes);
        tma_load_4d(dst, &a.map_dT, &bars[st], x0 - 4, y0 - 2, z0 - 2 + j, 0);
        tma_load_4d(dst + kBoxF, &a.map_a, &bars[st], x0 - 4, y0 - 2, z0 - 2 + j, 0);
    };
    // node planes of v for P v on tile (x0, y0, z0), from floor((z0 - 2) / rho_z)
    // on (zero outside the grid)
    const int nxt = g.nxt, nyt = g.nyt, nplane = nxt * nyt;
    auto load_nodes = [&](int x0, int y0, int z0) {
        const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry, kz_lo = (z0 - 2) >> lrz;
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
    };

    int t = blockIdx.x;
    if (t >= ntiles) return;
    {
        int x0, y0, z0;
        origin(t, x0, y0, z0);
        if (tid == 0) {
            for (int i = 0; i < kStages; ++i) mbar_init(&bars[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            const int ns = min(g.TZ, g.n[2] - z0) + 4;
            for (int j = 0; j < kAhead && j < ns; ++j) issue_plane(x0, y0, z0, j, j);
        }
        if (!DG) load_nodes(x0, y0, z0);
    }

    const bool own_col = w >= 2 && w < kTY + 2 && L >= 2 && L < TXI + 2;   // tile-owned column
    const float *sbase = tma_base + w * kTmaBoxX + L + 2;                  // this column in a TMA box
    // y-neighbours in the exchange rows (the outermost rows read themselves; unused)
    float *ex_t = smem + S.ext + w * 32 + L, *ex_c = smem + S.exc + w * 32 + L;
    const int up = w > 0 ? -32 : 0, dn = w < kNW - 1 ? 32 : 0;
    float *rowp = rows + ((w - 2) * TXI + (L - 2)) * 3;    // + node plane * kTY * TXI * 3
    uint32_t phase = 0;   // continues across the tiles of this CTA (each has a multiple of kStages planes)
    for (;;) {
        int x0, y0, z0, xn = 0, yn = 0, zn = 0;
        origin(t, x0, y0, z0);
        const int tn = t + gridDim.x;   // this CTA's next tile
        const bool has_next = chain && tn < ntiles;
        if (has_next) origin(tn, xn, yn, zn);
        const int TZc = min(g.TZ, g.n[2] - z0);
        const int nsteps = TZc + 4;
        const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry, kz_lo = (z0 - 2) >> lrz;

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

        // node tile loaded; the previous tile's reduction is done with rows and xr
        __syncthreads();

        float U0[3], U1[3], D[3];   // P v at node planes cz, cz + 1 (x-y interpolated), D = U1 - U0
        if (!DG) {
            const int cz = (z0 - 2) >> lrz;
            bilinear(cz, U0);
            bilinear(cz + 1, U1);
            for (int k = 0; k < 3; ++k) D[k] = U1[k] - U0[k];
        } else {
            for (int k = 0; k < 3; ++k) U0[k] = U1[k] = D[k] = 0.f;
        }
        float tm = 0.f, t0 = 0.f;                  // t at planes pC - 1, pC
        float a1[3] = {0.f, 0.f, 0.f};             // a' at plane pC (read by stage W one plane earlier)
        float d1[3] = {0.f, 0.f, 0.f}, d2[3] = {0.f, 0.f, 0.f};   // dT/dy at planes pW - 1 (= pC), pW - 2 (= pA)
        float cxp = 0.f;                           // c'_x at plane pA (from the previous plane's stage C)
        float czm2 = 0.f, czm1 = 0.f;              // c'_z at planes pA - 1, pA
        float acc0[3] = {0.f, 0.f, 0.f}, acc1[3] = {0.f, 0.f, 0.f};   // z-node planes czl, czl + 1

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
                if (tid == 0) {
                    // 3 planes ahead: of this tile, then the first planes of the next one
                    if (s + kAhead < nsteps) issue_plane(x0, y0, z0, s + kAhead, (j + kAhead) & (kStages - 1));
                    else if (has_next) issue_plane(xn, yn, zn, s + kAhead - nsteps, (j + kAhead) & (kStages - 1));
                }

                // ------------------------------------------------ P v: next node plane at a cell start
                if (!DG && phW == 0 && s > 0) {
                    U0[0] = U1[0]; U0[1] = U1[1]; U0[2] = U1[2];
                    bilinear((pW >> lrz) + 1, U1);
                    D[0] = U1[0] - U0[0]; D[1] = U1[1] - U0[1]; D[2] = U1[2] - U0[2];
                }

                mbar_wait_bounded(&bars[j], phase, a.err, a.poll_limit);
                // ------------------------------------------------ stage W: t at plane pW
                const float *sW = sbase + j * kStageF;
                const float dw0 = sW[0], dw1 = sW[kComp], dw2 = sW[2 * kComp];
                const float aw0 = sW[kBoxF], aw1 = sW[kBoxF + kComp], aw2 = sW[kBoxF + 2 * kComp];   // a' = a / (2 h)
                const float tp = fmaf(dw2, fmaf(fz, D[2], U0[2]),
                                      fmaf(dw1, fmaf(fz, D[1], U0[1]), dw0 * fmaf(fz, D[0], U0[0])));

                // ------------------------------------------------ stage C: c' at plane pC = pW - 1
                const int b = (j & 1) * kEx;
                const float txl = __shfl_up_sync(FULL, t0, 1), txr = __shfl_down_sync(FULL, t0, 1);
                float c0, c1, c2;
                if (DG) {   // a'^2 of plane pC
                    c0 = a1[0] * a1[0]; c1 = a1[1] * a1[1]; c2 = a1[2] * a1[2];
                } else {
                    const float dr = fmaf(a1[2], tp - tm, fmaf(a1[1], ex_t[b + dn] - ex_t[b + up], a1[0] * (txr - txl)));
                    c0 = dr * a1[0]; c1 = dr * a1[1]; c2 = dr * a1[2];
                }

                // ------------------------------------------------ stage A: G^T c at plane pA = pW - 2, times dT/dy
                const float cxl = __shfl_up_sync(FULL, cxp, 1), cxr = __shfl_down_sync(FULL, cxp, 1);
                if (j >= 4 || s0 > 0) {   // planes of the chunk (pA >= z0)
                    if (DG) {
                        // beta (x - e_a and x + e_a terms), times (dT/dy)^2, squared z weights
                        const float beta = (cxl + cxr) + (ex_c[b + up] + ex_c[b + dn]) + (czm2 + c2);
                        const float b1 = wz1 * wz1 * beta, b0 = (1.f - wz1) * (1.f - wz1) * beta;
                        const float q0 = d2[0] * d2[0], q1 = d2[1] * d2[1], q2 = d2[2] * d2[2];
                        acc0[0] = fmaf(b0, q0, acc0[0]); acc0[1] = fmaf(b0, q1, acc0[1]); acc0[2] = fmaf(b0, q2, acc0[2]);
                        acc1[0] = fmaf(b1, q0, acc1[0]); acc1[1] = fmaf(b1, q1, acc1[1]); acc1[2] = fmaf(b1, q2, acc1[2]);
                    } else {
                        const float bsum = (cxl - cxr) + (ex_c[b + up] - ex_c[b + dn]) + (czm2 - c2);
                        const float b1 = wz1 * bsum, b0 = bsum - b1;
                        acc0[0] = fmaf(b0, d2[0], acc0[0]); acc0[1] = fmaf(b0, d2[1], acc0[1]); acc0[2] = fmaf(b0, d2[2], acc0[2]);
                        acc1[0] = fmaf(b1, d2[0], acc1[0]); acc1[1] = fmaf(b1, d2[1], acc1[1]); acc1[2] = fmaf(b1, d2[2], acc1[2]);
                    }
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

        // the next tile's node planes (no thread reads the node tile any more),
        // while its first TMA planes are in flight
        if (!DG && has_next) load_nodes(xn, yn, zn);

        // ------------------------------------------------ x then y reduction onto the tile's node box
        {
            const int nplanes = (TZc >> lrz) + 1;
            float *box = a.boxes + (long)t * 3 * g.box;
            node_reduce_any<kTY, kNT, DG>(g.rho[0], g.rho[1], rows, xr, box, g.box, nplanes, DG ? 1.f : 2.f, tid);
        }
        if (!has_next) break;
        t = tn;
    }
}

}  // namespace

bool gn_matvec_supported(const TileGeom &g) {
    if (!g.tma || g.TY != kTY || g.nzt <= 0 || g.rho[0] < 2) return false;
    const MvSmem s = mv_smem(g);
    return (size_t)s.total * sizeof(float) <= 227u * 1024u;
}

cudaError_t launch_gn_matvec(const TileArgs<float> &a, bool diag, cudaStream_t st) {
    if (!gn_matvec_supported(a.g)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)mv_smem(a.g).total;
    const int ntiles = a.g.nb[0] * a.g.nb[1] * a.g.nb[2];
    // persistent CTAs (one per SM, tiles strided by the grid) when every tile's
    // plane sequence is a whole number of ring cycles, else one tile per CTA
    const int tail = a.g.n[2] - (a.g.nb[2] - 1) * a.g.TZ;
    const int chain = (a.g.TZ + 4) % kStages == 0 && (tail + 4) % kStages == 0;
    const int sms = device_sm_count();
    const int grid = chain ? (ntiles < sms ? ntiles : sms) : ntiles;
    auto run = [&](auto kernel) {
        cudaError_t e = allow_max_dynamic_smem(kernel);
        if (e != cudaSuccess) return e;
        kernel<<<grid, kNT, smem, st>>>(a, chain);
        return cudaGetLastError();
    };
    switch (a.g.rho[2] * 2 + (diag ? 1 : 0)) {
        case 2: return run(gn_matvec_kernel<1, false>);
        case 3: return run(gn_matvec_kernel<1, true>);
        case 4: return run(gn_matvec_kernel<2, false>);
        case 5: return run(gn_matvec_kernel<2, true>);
        case 8: return run(gn_matvec_kernel<4, false>);
        case 9: return run(gn_matvec_kernel<4, true>);
        case 17: return run(gn_matvec_kernel<0, true>);   // rho_z = 8: phases from the plane index
        default: return run(gn_matvec_kernel<0, false>);
    }
}

}  // namespace ngf
