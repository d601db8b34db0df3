// Gauss-Newton product of the NGF term, 2 hbar P^T J^T J P v (Eqs. (1), (11)),
// and the Jacobi diagonal of 2 hbar J^T J, from the stored linearisation
// (dT/dy and a = dr/dg per voxel and component): the column-marching form.
// The body of the kernels of gn_product.cu, shared with the persistent
// batched PCG kernel (pcg_batch.cu).
//
// Per voxel x:  t(x) = dT/dy(x) . (P v)(x)              (stage W)
//               c(x) = 2 (a(x) . G t(x)) a(x)            (stage C, G = central differences)
//               z(x) = (G^T c)(x) dT/dy(x)               (stage A)
// and the product is 2 hbar P^T z (the same three stages as the tile kernel
// of ngf_matvec.cu).
//
// Layout:
//  - a CTA owns a column of the volume: TXI (60, or 56 when rho_x = 8) x 16
//    voxels in x-y and every z plane.  Lane L holds the two adjacent x columns
//    x0 - 2 + 2L and x0 - 1 + 2L (packed FP32: one f32x2 instruction serves
//    both), warp w the row y0 - 2 + w; 20 warps cover the 16 rows and the
//    2-row halos, 32 lanes the 60 columns and the 2-column halos;
//  - the CTA marches z from plane -2 to n3 + 1, so every plane of the stored
//    linearisation is read once per column (no z halo is re-read); each
//    plane's dT/dy and a arrive by TMA (box 68 x 20 x 1 x 3, zero fill outside
//    the volume) into a 4-stage ring, 3 planes ahead, and the plane sequence
//    continues into the CTA's next column;
//  - one barrier per plane; x neighbours by warp shuffles (the other column of
//    a lane pair is local), y neighbours through double-buffered exchange
//    rows, z neighbours in registers;
//  - P v: the node planes of v stream through a 4-slot ring in shared memory
//    (each thread stages one node of a plane in registers two cells before it
//    is needed); each lane pair interpolates bilinearly in x-y at cell starts
//    and linearly in z per plane;
//  - P^T: every lane accumulates its columns' two z-node planes in registers.
//    When a node plane is complete, each lane of the interior warps parks its
//    pair's hat-weighted parts for the cell's lower and upper node (plain
//    stores, no shuffles); in the next plane all threads sum the parked lanes
//    of each (row, node column) (the x reduction), and in the plane after
//    that one thread per node of the column's box [3][m3][C1 + 1][C0 + 1]
//    sums its rows with the y hat weights and writes it (the y reduction), so
//    the reduction is spread over every warp and two barriers that the plane
//    loop has anyway; a node-parallel pass sums the boxes of neighbouring
//    columns (no atomics).
#pragma once

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ngf {
namespace gnpk {

constexpr int kTY = 16;                   // owned voxel rows per column
constexpr int kNW = kTY + 4;              // warps: rows incl. the 2-row halos
constexpr int kNT = 32 * kNW;
constexpr int kStages = 4;                // TMA ring depth (planes) = loop unroll
constexpr int kAhead = 3;                 // planes in flight ahead of stage W
constexpr int kBoxF = 4096;               // floats per field box (3 x 20 x 68 = 4080, 128-byte padded)
constexpr int kStageF = 2 * kBoxF;        // dT/dy box, then a box
constexpr int kComp = kNW * kColBoxX;     // floats between components in a box
constexpr int kEx = kNW * 64;             // floats per exchange buffer (a float2 per lane and warp)
constexpr uint32_t kPlaneBytes = 2u * kColBoxX * kNW * 3 * 4;
constexpr unsigned FULL = 0xffffffffu;

struct PcSmem {
    int tma, ext, exc, nodes, park, xr, total;
};

__host__ __device__ inline PcSmem pc_smem(const ColGeom &g) {
    PcSmem s;
    int off = 0;
    s.tma = off; off += kStages * kStageF + 32;            // + 128 bytes to align the base
    s.ext = off; off += 2 * kEx;                            // t of plane C, double-buffered
    s.exc = off; off += 2 * kEx;                            // c'_y of plane A, double-buffered
    s.nodes = off; off += 4 * ((g.nyt * g.nxt + 31) & ~31) * 4;   // node planes of v, [slot][y][x][xyz_]
    s.park = off; off += 2 * kTY * 32 * 6;                 // parked lane parts of 2 node planes, [slot][row][lane][3][lo, hi]
    s.xr = off; off += 2 * kTY * (g.C0 + 1) * 3;           // x-reduced rows of 2 node planes, [slot][row][node][3]
    s.total = off;
    return s;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// P^T along y for one node of a column box: node row jy receives the x-reduced
// rows of its lower cell (rows jy ry + i, weight 1 - f_i) and of its upper
// cell (rows (jy - 1) ry + i, weight f_i), f_i = (i + 1/2) / ry (squared
// weights for the diagonal); src points at row 0 of the node's column (stride ss).
template <int RY, bool SQ>
__device__ __forceinline__ float y_node(const float *src, int ss, int jy, int C1) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < RY; ++i) {
        const float f = (i + 0.5f) / RY;
        if (jy < C1) acc = fmaf(SQ ? (1.f - f) * (1.f - f) : 1.f - f, src[(jy * RY + i) * ss], acc);
        if (jy > 0) acc = fmaf(SQ ? f * f : f, src[((jy - 1) * RY + i) * ss], acc);
    }
    return acc;
}

template <bool SQ>
__device__ __forceinline__ float y_node_any(int ry, const float *src, int ss, int jy, int C1) {
    switch (ry) {
        case 1: return y_node<1, SQ>(src, ss, jy, C1);
        case 2: return y_node<2, SQ>(src, ss, jy, C1);
        case 4: return y_node<4, SQ>(src, ss, jy, C1);
        default: return y_node<8, SQ>(src, ss, jy, C1);
    }
}

// Bounded wait on a TMA barrier: one try (which suspends the thread for a
// while in hardware) and, rarely, the polling loop that gives up.
__device__ __forceinline__ void plane_wait(uint64_t *bar, uint32_t phase, int *err, int limit) {
    if (!mbar_try_wait(bar, phase)) mbar_wait_bounded(bar, phase, err, limit);
}

// DG = false: the GN product.  DG = true: the Jacobi diagonal of 2 hbar J^T J
// without the cross terms of the central-difference adjoint: per voxel
// beta = sum_a (a'_a^2 at x - e_a and x + e_a) with a' = a / (2 h), times
// (dT/dy)_k^2, onto the nodes with squared hat weights (stage C forms a'^2,
// stage A sums instead of differencing, P v is not needed).
// RZ: rho_z when it divides the ring depth (phases are constants), else 0.
// CHAIN: a column's plane count is a whole number of ring cycles (no bound
// checks inside a cycle), and CTAs walk several columns.
// RXY: 4 when rho_x = rho_y = 4 (the x and y passes are then straight-line
// code with constant extents), else 0 (extents from the geometry).
// The kernel body: the CTA's columns t0, t0 + tstep, ... (CHAIN) or column t0
// alone.  bars: the CTA's kStages TMA barriers, initialised here when
// init_bars; pbits: the parity of each barrier's next phase (bit j for stage
// j), carried from one call to the next when a CTA processes the columns of
// several volumes (MULTI: the persistent batched kernel of pcg_batch.cu, whose
// calls each end with no copy in flight).
template <int RZ, bool DG, bool CHAIN, int RXY, bool MULTI = false>
__device__ __forceinline__ void gn_product_body(const ColArgs &a, float *smem, uint64_t *bars, int t0, int tstep,
                                                bool init_bars, uint32_t &pbits) {
    const ColGeom &g = a.g;
    const PcSmem S = pc_smem(g);

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int ncols = g.nb[0] * g.nb[1];
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const int rx = g.rho[0], half = rx >> 1, rzm = g.rho[2] - 1;
    const float irz = g.irho[2];
    const int n3 = g.n[2], nsteps = n3 + 4;
    const int nxt = g.nxt, nplane = nxt * g.nyt, npad = (nplane + 31) & ~31;
    const int C0 = g.C0, C1 = g.C1, XR = (C0 + 1) * 3;
    const long mxy = (long)g.m[0] * g.m[1], Mn = mxy * g.m[2];

    float *tma_base = smem + S.tma + ((128u - (smem_u32(smem + S.tma) & 127u)) & 127u) / 4;
    float4 *s_nodes = reinterpret_cast<float4 *>(smem + S.nodes);
    float2 *park = reinterpret_cast<float2 *>(smem + S.park);   // [2 slots][16 rows][32 lanes][3] (lo, hi)
    float *xr = smem + S.xr;                                     // [2 slots][16 rows][C0 + 1][3]

    auto origin = [&](int t, int &x0, int &y0) {
        x0 = (t % g.nb[0]) * g.TXI;
        y0 = (t / g.nb[0]) * kTY;
    };
    // plane j (voxel plane j - 2) of column (x0, y0) into stage `st`; issued by
    // lane 0 of the last warp (a halo row with the least other work; callers
    // are warp-uniform)
    auto issue_plane = [&](int x0, int y0, int j, int st) {
        if (a.no_tma || L != 0) return;   // no_tma: test hook, the waits run out instead
        float *dst = tma_base + st * kStageF;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[st], kPlaneBytes);
        tma_load_4d(dst, &a.map_dT, &bars[st], x0 - 4, y0 - 2, j - 2, 0);
        tma_load_4d(dst + kBoxF, &a.map_a, &bars[st], x0 - 4, y0 - 2, j - 2, 0);
    };

    int t = t0;
    if (t >= ncols) return;
    {
        int x0, y0;
        origin(t, x0, y0);
        if (init_bars && tid == kNT - 32) {
            for (int i = 0; i < kStages; ++i) mbar_init(&bars[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (w == kNW - 1)
            for (int j = 0; j < kAhead && j < nsteps; ++j) issue_plane(x0, y0, j, j);
    }

    // this lane's pair of columns: local x index i0 = 2L - 2 (even) and i0 + 1
    const int i0 = 2 * L - 2;
    const bool interior_warp = w >= 2 && w < kTY + 2;
    const bool owner = interior_warp && i0 >= 0 && i0 < g.TXI;   // tile-owned pair
    const int ph = i0 & (rx - 1);   // x phase of the pair's first column in its cell (both share the cell)
    const float2 *sbase = reinterpret_cast<const float2 *>(tma_base + w * kColBoxX + 2 * L + 2);
    float2 *ex_t = reinterpret_cast<float2 *>(smem + S.ext) + w * 32 + L;
    float2 *ex_c = reinterpret_cast<float2 *>(smem + S.exc) + w * 32 + L;
    const int up = w > 0 ? -32 : 0, dn = w < kNW - 1 ? 32 : 0;   // in float2; the outer rows read themselves
    constexpr int exh = kEx / 2;                                   // float2 per exchange buffer
    const float2 *ex_t_up = ex_t + up, *ex_t_dn = ex_t + dn, *ex_c_up = ex_c + up, *ex_c_dn = ex_c + dn;
    float2 *park_lane = park + ((w - 2) * 32 + L) * 3;   // this lane's parked parts in a slot (interior warps)
    // the last warps (halo rows and the interior rows next to them) copy the node planes of v
    const bool node_warp = (kNW - 1 - w) * 32 < npad;
    const int ntid = tid - (kNT - npad);              // this thread's node of a plane (when node_warp)
    // work items of the x and y passes go to the threads lane-major, so that
    // every warp takes a share; quotients by the item extents from reciprocals
    // (exact for the item counts and extents here: below 2^11)
    const int lane_major = L * kNW + w;
    const float invXR = 1.f / XR, invNP = 1.f / ((C1 + 1) * (C0 + 1)), invC0 = 1.f / (C0 + 1);
    auto idiv = [](int a, float inv) { return __float2int_rz(((float)a + 0.5f) * inv); };

    uint32_t phase = 0;   // continues across the columns of this CTA (each has a multiple of kStages planes)
    for (;;) {
        int x0, y0, xn = 0, yn = 0;
        origin(t, x0, y0);
        const int tn = t + tstep;
        const bool has_next = CHAIN && tn < ncols;
        if (has_next) origin(tn, xn, yn);
        const int kx_lo = (x0 - 2) >> lrx, ky_lo = (y0 - 2) >> lry;
        float *box = a.boxes + (long)t * 3 * g.box;

        // P v: this thread's node of every node plane (threads of the node warps
        // beyond the plane fill padding), copied asynchronously into the ring
        // (zero outside the grid)
        int ngo = -1;   // offset of the node in a grid plane, -1 outside the grid or the plane
        if (ntid >= 0 && ntid < nplane) {
            const int ly = ntid / nxt, lx = ntid - ly * nxt;
            const int ux = kx_lo + lx, uy = ky_lo + ly;
            if (ux >= 0 && ux < g.m[0] && uy >= 0 && uy < g.m[1]) ngo = uy * g.m[0] + ux;
        }
        auto node_copy = [&](int kz) {   // node warps only (warp-uniform callers)
            const bool in = ngo >= 0 && kz >= 0 && kz < g.m[2];
            const float *p = in ? a.v + kz * mxy + ngo : a.v;
            const uint32_t dst = smem_u32(s_nodes + (kz & 3) * npad + ntid);
            const uint32_t n = in ? 4u : 0u;   // 0 source bytes: zero fill
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(p), "r"(n) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 4), "l"(p + Mn), "r"(n) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 8), "l"(p + 2 * Mn), "r"(n) : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        const int cz0 = (-2) >> lrz;   // node plane of voxel plane -2
        if (!DG && node_warp) {
            asm volatile("cp.async.wait_all;" ::: "memory");   // the last column's copies have landed
            for (int i = 0; i < 4; ++i) node_copy(cz0 + i);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }

        // this pair's bilinear position in a node plane
        const int qoff = (((y0 - 2 + w) >> lry) - ky_lo) * nxt + (((x0 + i0) >> lrx) - kx_lo);
        auto bilinear = [&](int kz, float2 *U) {
            const float4 *qp = s_nodes + (kz & 3) * npad + qoff;
            const float4 n00 = qp[0], n10 = qp[1], n01 = qp[nxt], n11 = qp[nxt + 1];
            const float2 fx2 = make_float2((ph + 0.5f) * g.irho[0], (ph + 1.5f) * g.irho[0]);
            const float2 fy2 = bc2((((y0 - 2 + w) & (g.rho[1] - 1)) + 0.5f) * g.irho[1]);
            float2 lo = fma2(fx2, bc2(n10.x - n00.x), bc2(n00.x)), hi = fma2(fx2, bc2(n11.x - n01.x), bc2(n01.x));
            U[0] = fma2(fy2, sub2(hi, lo), lo);
            lo = fma2(fx2, bc2(n10.y - n00.y), bc2(n00.y));
            hi = fma2(fx2, bc2(n11.y - n01.y), bc2(n01.y));
            U[1] = fma2(fy2, sub2(hi, lo), lo);
            lo = fma2(fx2, bc2(n10.z - n00.z), bc2(n00.z));
            hi = fma2(fx2, bc2(n11.z - n01.z), bc2(n01.z));
            U[2] = fma2(fy2, sub2(hi, lo), lo);
        };
        // park a completed node plane (interior warps): the pair's parts for its
        // cell's lower and upper node, hat weights 1 - f and f with f = fe and
        // fe + 1 / rho_x (squared for the diagonal), zero outside the tile
        auto park_plane = [&](const float2 *acc, int kz) {
            if (!interior_warp) return;
            float2 *dst = park_lane + (kz & 1) * (kTY * 32 * 3);
            const float irx = g.irho[0], fe = (ph + 0.5f) * irx;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float ve = owner ? acc[k].x : 0.f, vo = owner ? acc[k].y : 0.f;
                if (DG) {
                    const float fo = fe + irx;
                    dst[k] = make_float2(fmaf((1.f - fo) * (1.f - fo), vo, (1.f - fe) * (1.f - fe) * ve),
                                         fmaf(fo * fo, vo, fe * fe * ve));
                } else {
                    const float sum = ve + vo, hi = fmaf(fe, sum, vo * irx);
                    dst[k] = make_float2(sum - hi, hi);
                }
            }
        };
        // x reduction of a parked node plane (all threads): item (row, node jx,
        // component) sums the lower parts of the lanes of cell jx and the upper
        // parts of the lanes of cell jx - 1 (the lanes of cell c are
        // 1 + c rho_x / 2 .. + rho_x / 2 - 1; cell C0 lies outside the tile)
        auto x_pass = [&](int kz) {
            const float2 *src = park + (kz & 1) * (kTY * 32 * 3);
            float *dst = xr + (kz & 1) * (kTY * XR);
            if constexpr (RXY > 0) {   // consecutive threads take consecutive (row, node, component) items
                constexpr int H = RXY / 2, C0c = (60 - 60 % RXY) / RXY, XRc = (C0c + 1) * 3, NX = kTY * XRc;
#pragma unroll
                for (int i = 0; i < (NX + kNT - 1) / kNT; ++i) {
                    const int it = tid + i * kNT;
                    if (NX % kNT == 0 || it < NX) {
                        const int row = it / XRc, r = it % XRc, jx = r / 3, k = r % 3;
                        const float2 *p = src + (row * 32 + 1 + jx * H) * 3 + k;
                        const float2 *pl = jx < C0c ? p : p - 3 * H, *ph = jx > 0 ? p : p + 3 * H;
                        float lo = 0.f, hi = 0.f;
#pragma unroll
                        for (int q = 0; q < H; ++q) {
                            lo += pl[3 * q].x;
                            hi += ph[3 * (q - H)].y;
                        }
                        dst[it] = (jx < C0c ? lo : 0.f) + (jx > 0 ? hi : 0.f);
                    }
                }
            } else {
                for (int it = lane_major; it < kTY * XR; it += kNT) {
                    const int row = idiv(it, invXR), r = it - row * XR, jx = (r * 43) >> 7, k = r - jx * 3;
                    const float2 *p = src + (row * 32 + 1 + jx * half) * 3 + k;
                    // the lanes of cell jx (lower parts, none for jx = C0) and of cell
                    // jx - 1 (upper parts, none for jx = 0); a missing cell reads a
                    // neighbouring one inside the row and is discarded
                    const float2 *pl = jx < C0 ? p : p - 3 * half, *ph = jx > 0 ? p : p + 3 * half;
                    float lo, hi;
                    switch (half) {
                        case 1: lo = pl[0].x; hi = ph[-3].y; break;
                        case 2: lo = pl[0].x + pl[3].x; hi = ph[-6].y + ph[-3].y; break;
                        default: lo = (pl[0].x + pl[3].x) + (pl[6].x + pl[9].x); hi = (ph[-12].y + ph[-9].y) + (ph[-6].y + ph[-3].y);
                    }
                    dst[it] = (jx < C0 ? lo : 0.f) + (jx > 0 ? hi : 0.f);
                }
            }
        };
        // y reduction of an x-reduced node plane: one thread per node of the box
        auto y_pass = [&](int kz) {
            if constexpr (RXY > 0) {   // consecutive threads take consecutive nodes (coalesced stores)
                constexpr int C0c = (60 - 60 % RXY) / RXY, C1c = kTY / RXY, XRc = (C0c + 1) * 3;
                constexpr int NP = (C1c + 1) * (C0c + 1), NY = 3 * NP;
                const float *src = xr + (kz & 1) * (kTY * XRc);
                float *dst = box + (long)kz * NP;
#pragma unroll
                for (int i = 0; i < (NY + kNT - 1) / kNT; ++i) {
                    const int it = (tid + kNT - 64) % kNT + i * kNT;   // from the third warp on
                    if (it < NY) {
                        const int k = it / NP, r = it % NP, jy = r / (C0c + 1), jx = r % (C0c + 1);
                        const float v = y_node<RXY, DG>(src + jx * 3 + k, XRc, jy, C1c);
                        dst[(long)k * g.box + r] = (DG ? 1.f : 2.f) * v;
                    }
                }
            } else {
                const int np = (C1 + 1) * (C0 + 1);
                for (int it = lane_major; it < 3 * np; it += kNT) {
                    const int k = idiv(it, invNP), r = it - k * np;
                    const int jy = idiv(r, invC0), jx = r - jy * (C0 + 1);
                    const float v = y_node_any<DG>(g.rho[1], xr + (kz & 1) * (kTY * XR) + jx * 3 + k, XR, jy, C1);
                    box[(long)k * g.box + (long)kz * np + r] = (DG ? 1.f : 2.f) * v;
                }
            }
        };

        // the exchange rows read before this column has written them (stages C and A
        // of its first planes, which multiply them by zeros) must hold finite values
        {
            float *ex = smem + S.ext;
            for (int i = tid; i < 4 * kEx; i += kNT) ex[i] = 0.f;
        }
        __syncthreads();   // node ring filled, exchange rows cleared; the previous column's sweeps are done with xr

        // P v of the pair at node planes kz (U0) and kz + 1 (U0 + D) of the current cell
        float2 U0[3], D[3];
        if (!DG) {
            float2 U1[3];
            bilinear(cz0, U0);
            bilinear(cz0 + 1, U1);
            for (int k = 0; k < 3; ++k) D[k] = sub2(U1[k], U0[k]);
        } else {
            for (int k = 0; k < 3; ++k) U0[k] = D[k] = make_float2(0.f, 0.f);
        }
        const float2 z2 = make_float2(0.f, 0.f);
        float2 tm = z2, t0 = z2;                  // t at planes pC - 1, pC
        float2 a1[3] = {z2, z2, z2};              // a' at plane pC
        float2 d1[3] = {z2, z2, z2}, d2[3] = {z2, z2, z2};   // dT/dy at planes pC, pA
        float2 cxp = z2;                          // c'_x at plane pA
        float2 czm2 = z2, czm1 = z2;              // c'_z at planes pA - 1, pA
        float2 acc0[3] = {z2, z2, z2}, acc1[3] = {z2, z2, z2};   // z-node planes of pA's cell
        int xk = -1, yk = -1;                     // node planes due for the x pass, the y pass in this step

        for (int s0 = 0; s0 < nsteps; s0 += kStages, phase ^= 1u) {
#pragma unroll
            for (int j = 0; j < kStages; ++j) {
                const int s = s0 + j;
                if (!CHAIN && s >= nsteps) break;
                const int pW = s - 2;
                // z phases of planes pW and pA = pW - 2 (s0 is a multiple of rho_z when RZ != 0)
                const int phW = RZ ? ((j - 2) & (RZ - 1)) : (pW & rzm);
                const int phA = RZ ? (j & (RZ - 1)) : ((pW - 2) & rzm);
                const float fz = RZ ? (phW + 0.5f) / (float)(RZ ? RZ : 1) : (phW + 0.5f) * irz;
                const float wz1 = RZ ? (phA + 0.5f) / (float)(RZ ? RZ : 1) : (phA + 0.5f) * irz;
                const bool cell_start = !DG && phW == 0 && s > 0;

                // at a cell start, the node-plane copy issued two cells ago (the plane
                // read in this step) lands before this barrier; the last one stays in flight
                if (cell_start && node_warp) asm volatile("cp.async.wait_group 1;" ::: "memory");
                // the stage of plane s - 1 and the buffers of the last plane were last read before this barrier
                __syncthreads();
                if (w == kNW - 1) {
                    // 3 planes ahead: of this column, then the first planes of the next one
                    if (CHAIN ? s < nsteps - kAhead : s + kAhead < nsteps)
                        issue_plane(x0, y0, s + kAhead, (j + kAhead) & (kStages - 1));
                    else if (has_next)
                        issue_plane(xn, yn, s + kAhead - nsteps, (j + kAhead) & (kStages - 1));
                }
                // the node planes parked and x-reduced in the last steps move on
                if (yk >= 0) y_pass(yk);
                if (xk >= 0) x_pass(xk);
                yk = xk;
                xk = -1;

                // ------------------------------------------------ P v: the next node plane at a cell start
                if (cell_start) {
                    const int kz = pW >> lrz;
                    float2 U1[3];
                    bilinear(kz + 1, U1);
                    for (int k = 0; k < 3; ++k) {
                        U0[k] = add2(U0[k], D[k]);   // node plane kz (to one rounding)
                        D[k] = sub2(U1[k], U0[k]);
                    }
                    if (node_warp) node_copy(kz + 3);   // read at the start of cell kz + 2
                }

                if constexpr (MULTI) {
                    plane_wait(&bars[j], (pbits >> j) & 1u, a.err, a.poll_limit);
                    pbits ^= 1u << j;
                } else {
                    plane_wait(&bars[j], phase, a.err, a.poll_limit);
                }
                // ------------------------------------------------ stage W: t at plane pW
                const float2 *sW = sbase + j * (kStageF / 2);
                const float2 dw0 = sW[0], dw1 = sW[kComp / 2], dw2 = sW[kComp];
                // a' = a / (2 h), stored so by the linearisation
                const float2 aw0 = sW[kBoxF / 2], aw1 = sW[(kBoxF + kComp) / 2], aw2 = sW[(kBoxF + 2 * kComp) / 2];
                float2 tp;
                if (!DG) {
                    const float2 fz2 = bc2(fz);
                    tp = mul2(dw0, fma2(fz2, D[0], U0[0]));
                    tp = fma2(dw1, fma2(fz2, D[1], U0[1]), tp);
                    tp = fma2(dw2, fma2(fz2, D[2], U0[2]), tp);
                } else {
                    tp = z2;
                }

                // ------------------------------------------------ stage C: c' at plane pC = pW - 1
                const int bo = (j & 1) * exh;
                float2 c0, c1, c2;
                if (DG) {
                    c0 = mul2(a1[0], a1[0]); c1 = mul2(a1[1], a1[1]); c2 = mul2(a1[2], a1[2]);
                } else {
                    const float sU = __shfl_up_sync(FULL, t0.y, 1), sD = __shfl_down_sync(FULL, t0.x, 1);
                    const float2 dtx = make_float2(t0.y - sU, sD - t0.x);
                    const float2 dty = sub2(ex_t_dn[bo], ex_t_up[bo]);
                    const float2 dr = fma2(a1[2], sub2(tp, tm), fma2(a1[1], dty, mul2(a1[0], dtx)));
                    c0 = mul2(dr, a1[0]); c1 = mul2(dr, a1[1]); c2 = mul2(dr, a1[2]);
                }

                // ------------------------------------------------ stage A: G^T c at plane pA = pW - 2, times dT/dy
                // (planes before the volume have dT/dy = 0 and add nothing)
                {
                    const float cxl = __shfl_up_sync(FULL, cxp.y, 1), cxr = __shfl_down_sync(FULL, cxp.x, 1);
                    const float2 wz = bc2(wz1);
                    if (DG) {
                        const float2 bx = make_float2(cxl + cxp.y, cxp.x + cxr);
                        const float2 beta = add2(add2(bx, add2(ex_c_up[bo], ex_c_dn[bo])), add2(czm2, c2));
                        const float2 b1 = mul2(mul2(wz, wz), beta);
                        const float2 b0 = mul2(bc2((1.f - wz1) * (1.f - wz1)), beta);
                        for (int k = 0; k < 3; ++k) {
                            const float2 qk2 = mul2(d2[k], d2[k]);
                            acc0[k] = fma2(b0, qk2, acc0[k]);
                            acc1[k] = fma2(b1, qk2, acc1[k]);
                        }
                    } else {
                        const float2 bx = make_float2(cxl - cxp.y, cxp.x - cxr);
                        const float2 bsum = add2(add2(bx, sub2(ex_c_up[bo], ex_c_dn[bo])), sub2(czm2, c2));
                        const float2 b1 = mul2(wz, bsum), b0 = sub2(bsum, b1);
                        for (int k = 0; k < 3; ++k) {
                            acc0[k] = fma2(b0, d2[k], acc0[k]);
                            acc1[k] = fma2(b1, d2[k], acc1[k]);
                        }
                    }
                    if (phA == (RZ ? RZ - 1 : rzm) && s0 > 0) {
                        // node plane (pA >> lrz) is complete: park it (x pass next step, y pass after)
                        const int kz = (s - 4) >> lrz;
                        park_plane(acc0, kz);
                        xk = kz;
                        for (int k = 0; k < 3; ++k) {
                            acc0[k] = acc1[k];
                            acc1[k] = z2;
                        }
                    }
                }
                // ------------------------------------------------ hand over to the next plane
                ex_t[exh - bo] = tp;
                ex_c[exh - bo] = c1;
                tm = t0; t0 = tp;
                czm2 = czm1; czm1 = c2;
                cxp = c0;
                for (int k = 0; k < 3; ++k) d2[k] = d1[k];
                d1[0] = dw0; d1[1] = dw1; d1[2] = dw2;
                a1[0] = aw0; a1[1] = aw1; a1[2] = aw2;
            }
        }
        // the pending passes and the top node plane (above the last cell)
        __syncthreads();
        if (yk >= 0) y_pass(yk);
        if (xk >= 0) x_pass(xk);
        park_plane(acc0, g.m[2] - 1);
        __syncthreads();
        if (xk >= 0) y_pass(xk);
        x_pass(g.m[2] - 1);
        __syncthreads();
        y_pass(g.m[2] - 1);
        if (!has_next) break;
        t = tn;
    }
    if constexpr (MULTI) {   // the node-plane copies still in flight land before the CTA moves on
        if (!DG && node_warp) asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    }
}

}  // namespace gnpk
}  // namespace ngf
