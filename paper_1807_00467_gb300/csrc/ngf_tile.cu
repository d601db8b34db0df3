// Fused voxel-column kernel for the NGF term of Eq. (1): trilinear warp of
// the template, central-difference gradients, per-voxel NGF residual, the
// adjoint of the central difference, and the gather of voxel contributions
// onto the grid nodes (P^T), in one pass over the volume.
//
// A CTA owns an x-y tile of TXI x TY voxels (aligned to grid cells) and a
// chunk of TZ voxel planes.  Each thread owns one voxel column (x, y) of the
// tile plus a 2-voxel halo (lane = x, warp = y) and marches through the chunk
// plane by plane with three pipelined stages:
//   W (plane p+2): y = x + P u, sample T(y) and dT/dy   (all columns)
//   C (plane p+1): f = grad R, g = grad T(y), r, c = d(1 - r^2)/dg (halo 1)
//   A (plane p)  : adjoint of the central difference of c, times dT/dy,
//                  then P^T onto the CTA's nodes (interior columns)
// z-neighbours stay in the thread's registers (three-plane rings),
// x-neighbours come from warp shuffles, y-neighbours through a
// double-buffered shared-memory plane (two barriers per plane).  The P^T
// gather reduces along x with warp shuffles, along z in registers of one lane
// per cell, and along y through shared memory once per node plane; each CTA
// writes its node box once, and boxes of neighbouring CTAs sharing boundary
// nodes are summed by finalize_nodes (gather, no atomics).
//
// MODE selects: the objective only (line search), the stored Gauss-Newton
// linearisation, the gradient, the NGF Gauss-Newton product 2 hbar J^T J v
// (stage W forms dT . P v from the stored dT/dy, stage C forms 2 (a . G w) a
// from the stored a), or the Jacobi diagonal of that product with the
// cross terms of the central-difference adjoint dropped.
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ngf {

template <int MODE>
struct Mode {
    static constexpr bool adj = MODE == MODE_GRAD || MODE == MODE_GRADLIN || MODE == MODE_MATVEC;
    static constexpr bool store = MODE == MODE_LIN || MODE == MODE_GRADLIN;
    static constexpr bool matvec = MODE == MODE_MATVEC;
    static constexpr bool diag = MODE == MODE_DIAG;
    static constexpr bool warp = !matvec && !diag;   // samples T(y), sums 1 - r^2
    static constexpr bool reduce = adj || diag;      // P^T onto nodes
    static constexpr int HZ = adj ? 2 : 1;           // z halo of stage W
    static constexpr int LAG = adj ? 2 : 1;          // planes between W and A
};

// Shared-memory carve-up (floats).  Host and device agree on it.
struct ColSmem {
    int tma, tma_stage, tma_a, ex1, ex2, ex3, nodes, rowA, rowB, total;
};

__host__ __device__ inline ColSmem col_smem(const TileGeom &g, int mode) {
    const bool adj = mode == MODE_GRAD || mode == MODE_GRADLIN || mode == MODE_MATVEC;
    const bool diag = mode == MODE_DIAG, warpm = !(mode == MODE_MATVEC) && !diag, reduce = adj || diag;
    const int NW = g.TY + 4;
    ColSmem s;
    int off = 0;
    // TMA stages first (128-byte aligned): per plane a dT box and an a box,
    // each kTmaBoxX x NW x 3 floats, padded to 128 bytes
    const int box_f = ((kTmaBoxX * NW * 3 * 4 + 127) / 128) * 32;
    const bool tma = g.tma && (mode == MODE_MATVEC || diag);
    s.tma = off;
    s.tma_a = box_f;
    s.tma_stage = 2 * box_f;
    off += tma ? kTmaStages * 2 * box_f + 32 : 0;   // + 128 bytes to align the base
    s.ex1 = off; off += 2 * NW * 32;                       // W value (diag: a_y^2) at plane C (A)
    s.ex2 = off; off += warpm ? 2 * NW * 32 : 0;           // R at plane C
    s.ex3 = off; off += adj ? 2 * NW * 32 : 0;             // c_y at plane A
    s.nodes = off; off += diag ? 0 : (g.nzt > 0 ? g.nzt : 2) * 3 * g.nxt * g.nyt;
    // x- and z-reduced row sums of every node plane of the chunk (y-reduced at the end)
    s.rowA = off; off += reduce ? (g.C[2] + 1) * g.TY * (g.C[0] + 1) * 3 : 0;
    s.rowB = off; off += reduce ? (g.C[2] + 1) * g.TY * (g.C[0] + 1) * 3 : 0;
    s.total = off;
    return s;
}

size_t tile_smem_bytes(const TileGeom &g, int mode) { return sizeof(float) * (size_t)col_smem(g, mode).total; }

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

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// y-reduce the row sums of node planes 0..nplanes-1 and write the CTA's box.
template <int TY, bool SQ>
__device__ __forceinline__ void write_box(const TileGeom &g, const float *rowA, const float *rowB, float *boxes,
                                          int cta, int nplanes, int tid, int nt) {
    const int CX = g.C[0], CY = g.C[1], ry = g.rho[1], lry = g.lrho[1];
    const float iry = g.irho[1];
    const int per = (CX + 1) * (CY + 1);
    for (int e = tid; e < 3 * nplanes * per; e += nt) {
        const int jx = e % (CX + 1), t2 = e / (CX + 1), jy = t2 % (CY + 1), t3 = t2 / (CY + 1);
        const int jz = t3 % nplanes, comp = t3 / nplanes;
        float v = 0.f;
        const int ty_lo = max(0, (jy - 1) * ry), ty_hi = min(TY, (jy + 1) * ry);
        const float *ra = rowA + (long)jz * TY * (CX + 1) * 3, *rb = rowB + (long)jz * TY * (CX + 1) * 3;
        for (int ty = ty_lo; ty < ty_hi; ++ty) {
            float wy = ((ty & (ry - 1)) + 0.5f) * iry;
            if ((ty >> lry) == jy) wy = 1.f - wy;
            if (SQ) wy *= wy;
            v = fmaf(wy, ra[(ty * (CX + 1) + jx) * 3 + comp] + rb[(ty * (CX + 1) + jx) * 3 + comp], v);
        }
        boxes[((long)cta * 3 + comp) * g.box + (jz * (CY + 1) + jy) * (CX + 1) + jx] = v;
    }
}

template <int TY, int MODE, typename TImg>
__global__ void __launch_bounds__(32 * (TY + 4), TY == 8 ? 2 : 1) ngf_tile_kernel(const __grid_constant__ TileArgs<TImg> a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    using M = Mode<MODE>;
    constexpr int NW = TY + 4, NT = 32 * NW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[kTmaStages];
    const TileGeom &g = a.g;
    const ColSmem S = col_smem(g, MODE);
    const bool tma = (M::matvec || M::diag) && g.tma;
    float *ex1 = smem + S.ex1, *ex2 = smem + S.ex2, *ex3 = smem + S.ex3;
    float *s_nodes = smem + S.nodes, *rowA = smem + S.rowA, *rowB = smem + S.rowB;

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long sxy = (long)nx * ny, N = sxy * nz;
    const int TXI = g.TXI;
    const int x0 = blockIdx.x * TXI, y0 = blockIdx.y * TY, z0 = blockIdx.z * g.TZ;
    const int TZc = min(g.TZ, nz - z0);
    const int rx = g.rho[0], rz = g.rho[2];
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const float irx = g.irho[0], iry = g.irho[1], irz = g.irho[2];
    const int gx = x0 - 2 + L, gy = y0 - 2 + w;
    const bool colin = L < TXI + 4 && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const bool inC = L >= 1 && L <= TXI + 2 && w >= 1 && w <= TY + 2;
    const bool inA = L >= 2 && L <= TXI + 1 && w >= 2 && w <= TY + 1;
    const bool intxy = colin && gx >= 1 && gx <= nx - 2 && gy >= 1 && gy <= ny - 2;
    const long col = colin ? (long)gy * nx + gx : 0;
    const int CX = g.C[0];
    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;

    // ---- plane-invariant per-column constants
    const int kx_lo = max(x0 - 2, 0) >> lrx, ky_lo = max(y0 - 2, 0) >> lry;
    int nlx = 0, nly = 0;
    float fxw = 0.f, fyw = 0.f;
    if (colin) {
        const int cxg = gx >> lrx, cyg = gy >> lry;
        fxw = ((gx - (cxg << lrx)) + 0.5f) * irx;
        fyw = ((gy - (cyg << lry)) + 0.5f) * iry;
        nlx = cxg - kx_lo;
        nly = cyg - ky_lo;
    }
    const int nxt = g.nxt, nplane = g.nxt * g.nyt;
    // P^T along x: this column's cell within the tile and its two weights
    const int xl = L - 2;
    const int cxl = inA ? (xl >> lrx) : 0;
    float wx1 = inA ? ((xl & (rx - 1)) + 0.5f) * irx : 0.f, wx0 = inA ? 1.f - wx1 : 0.f;
    if (M::diag) { wx0 *= wx0; wx1 *= wx1; }
    const bool leader = inA && ((xl & (rx - 1)) == 0);

    if (M::reduce)
        for (int i = tid; i < (g.C[2] + 1) * TY * (CX + 1) * 3; i += NT) { rowA[i] = 0.f; rowB[i] = 0.f; }
    // the node planes this CTA interpolates from, loaded once (if they fit)
    const int kz_lo = max(z0 - M::HZ, 0) >> lrz;
    if (!M::diag && g.nzt > 0) {
        const long mxy = (long)g.m[0] * g.m[1], Mn = mxy * g.m[2];
        for (int i = tid; i < g.nzt * 3 * nplane; i += NT) {
            const int pl = i / nplane, r = i - pl * nplane;          // pl = plane * 3 + comp
            const int kz = kz_lo + pl / 3, comp = pl - (pl / 3) * 3;
            const int ly = r / nxt, lx = r - ly * nxt;
            const int ux = kx_lo + lx, uy = ky_lo + ly;
            float v = 0.f;
            if (ux < g.m[0] && uy < g.m[1] && kz < g.m[2]) v = __ldg(a.u + comp * Mn + (long)kz * mxy + (long)uy * g.m[0] + ux);
            s_nodes[i] = v;
        }
    }

    // ---- state carried between planes
    float U0[3] = {0.f, 0.f, 0.f}, U1[3] = {0.f, 0.f, 0.f};   // x-y interpolated node values, planes cz, cz+1
    int cur_cz = -1000;
    float t_m = 0.f, t_0 = 0.f, t_p = 0.f;                     // W value at planes pW-2, pW-1, pW
    float r_m = 0.f, r_0 = 0.f, r_p = 0.f;                     // R at the same planes
    float d_2[3] = {0.f, 0.f, 0.f}, d_1[3] = {0.f, 0.f, 0.f}, d_0[3] = {0.f, 0.f, 0.f};   // dT/dy
    float cx_p = 0.f, cy_p = 0.f, cz_mm = 0.f, cz_m = 0.f;     // adjoint inputs of plane A
    float q0_1 = 0.f, q1_1 = 0.f, q2_2 = 0.f, q2_1 = 0.f;      // diag: a^2 of planes pW-1, pW-2
    float acc[2][2][3] = {};                                    // leader: [x node lo/hi][z plane P0/P1][comp]
    float dsum = 0.f, dcomp = 0.f;
    // matvec / diag prefetch: dT at the next W plane, a at the next C (diag: W) plane
    float dnx[3] = {0.f, 0.f, 0.f}, anx[3] = {0.f, 0.f, 0.f};
    const int nsteps = TZc + 2 * M::HZ;
    constexpr uint32_t kPlaneBytes = 2u * kTmaBoxX * NW * 3 * 4;
    // 128-byte aligned base of the TMA stages
    float *tma_base = smem + S.tma + ((128u - (smem_u32(smem + S.tma) & 127u)) & 127u) / 4;
    // plane j of this CTA's sequence: TMA into stage j % kTmaStages, or (outside
    // the volume) a plain arrive so that the barrier's phase still advances
    auto issue_plane = [&](int j) {
        uint64_t *bar = &bars[j % kTmaStages];
        const int p = z0 - M::HZ + j;
        if (a.no_tma) return;   // test hook: the waits run out instead
        if (p >= 0 && p < nz) {
            float *st = tma_base + (j % kTmaStages) * S.tma_stage;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar, kPlaneBytes);
            tma_load_4d(st, &a.map_dT, bar, x0 - 4, y0 - 2, p, 0);
            tma_load_4d(st + S.tma_a, &a.map_a, bar, x0 - 4, y0 - 2, p, 0);
        } else {
            mbar_arrive(bar);
        }
    };
    if (tma && tid == 0) {
        for (int i = 0; i < kTmaStages; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int j = 0; j < kTmaStages - 2 && j < nsteps; ++j) issue_plane(j);
    }
    if ((M::matvec || M::diag) && !tma) {
        const int p = z0 - M::HZ;
        if (colin && p >= 0 && p < nz) {
            const long v = (long)p * sxy + col;
            dnx[0] = __ldg(a.lin_dT + v); dnx[1] = __ldg(a.lin_dT + N + v); dnx[2] = __ldg(a.lin_dT + 2 * N + v);
            if (M::diag) { anx[0] = __ldg(a.lin_a + v); anx[1] = __ldg(a.lin_a + N + v); anx[2] = __ldg(a.lin_a + 2 * N + v); }
        }
        if (M::matvec && inC && colin && p - 1 >= 0 && p - 1 < nz) {
            const long v = (long)(p - 1) * sxy + col;
            anx[0] = __ldg(a.lin_a + v); anx[1] = __ldg(a.lin_a + N + v); anx[2] = __ldg(a.lin_a + 2 * N + v);
        }
    }
    __syncthreads();

    const int o = w * kTmaBoxX + L + 2;   // this column in a TMA box
    int stage = 0;                         // s % kTmaStages
    uint32_t phase = 0;                    // (s / kTmaStages) & 1
    for (int s = 0; s < nsteps; ++s, stage = stage + 1 == kTmaStages ? 0 : stage + 1, phase ^= (stage == 0)) {
        const int pW = z0 - M::HZ + s, pC = pW - 1, pA = pW - M::LAG;
        const bool zW = pW >= 0 && pW < nz;
        // ------------------------------------------------ node planes for P of plane pW
        if (!M::diag && zW && g.nzt > 0) {
            const int cz = pW >> lrz;
            if (cz != cur_cz && colin) {
                const bool both = cz != cur_cz + 1;
                const float *qa = s_nodes + ((cz - kz_lo) * 3) * nplane + nly * nxt + nlx;
                const float *qb = qa + 3 * nplane;
#pragma unroll
                for (int comp = 0; comp < 3; ++comp) {
                    if (both) {
                        const float *q = qa + comp * nplane;
                        U0[comp] = lerp_fixed(lerp_fixed(q[0], q[1], 1.f - fxw, fxw),
                                              lerp_fixed(q[nxt], q[nxt + 1], 1.f - fxw, fxw), 1.f - fyw, fyw);
                    } else {
                        U0[comp] = U1[comp];
                    }
                    const float *q = qb + comp * nplane;
                    U1[comp] = lerp_fixed(lerp_fixed(q[0], q[1], 1.f - fxw, fxw),
                                          lerp_fixed(q[nxt], q[nxt + 1], 1.f - fxw, fxw), 1.f - fyw, fyw);
                }
            }
            cur_cz = cz;
        } else if (!M::diag && zW) {
            const int cz = pW >> lrz;
            if (cz != cur_cz) {
                const bool both = cz != cur_cz + 1;
                const long mxy = (long)g.m[0] * g.m[1], Mn = mxy * g.m[2];
                for (int kz = both ? cz : cz + 1; kz <= cz + 1; ++kz) {
                    float *dst = s_nodes + (kz & 1) * 3 * nplane;
                    for (int i = tid; i < 3 * nplane; i += NT) {
                        const int comp = i / nplane, r = i - comp * nplane;
                        const int ly = r / nxt, lx = r - ly * nxt;
                        const int ux = kx_lo + lx, uy = ky_lo + ly;
                        float v = 0.f;
                        if (ux < g.m[0] && uy < g.m[1]) v = __ldg(a.u + comp * Mn + (long)kz * mxy + (long)uy * g.m[0] + ux);
                        dst[i] = v;
                    }
                }
                __syncthreads();
                if (colin) {
                    const float *qa = s_nodes + (cz & 1) * 3 * nplane + nly * nxt + nlx;
                    const float *qb = s_nodes + ((cz + 1) & 1) * 3 * nplane + nly * nxt + nlx;
#pragma unroll
                    for (int comp = 0; comp < 3; ++comp) {
                        if (both) {
                            const float *q = qa + comp * nplane;
                            U0[comp] = lerp_fixed(lerp_fixed(q[0], q[1], 1.f - fxw, fxw),
                                                  lerp_fixed(q[nxt], q[nxt + 1], 1.f - fxw, fxw), 1.f - fyw, fyw);
                        } else {
                            U0[comp] = U1[comp];
                        }
                        const float *q = qb + comp * nplane;
                        U1[comp] = lerp_fixed(lerp_fixed(q[0], q[1], 1.f - fxw, fxw),
                                              lerp_fixed(q[nxt], q[nxt + 1], 1.f - fxw, fxw), 1.f - fyw, fyw);
                    }
                }
                cur_cz = cz;
            }
        }
        // ------------------------------------------------ stage W: plane pW
        float val = 0.f, rv = 0.f, dn[3] = {0.f, 0.f, 0.f}, qn[3] = {0.f, 0.f, 0.f};
        float acur[3] = {anx[0], anx[1], anx[2]};   // matvec: a at plane pC
        if (tma) {
            // issue plane s + 3 into the stage of plane s - 2 (free: its last
            // reader, stage C of step s - 1, is behind this step's barriers),
            // then wait for plane s
            if (tid == 0 && s + kTmaStages - 2 < nsteps) issue_plane(s + kTmaStages - 2);
            mbar_wait_bounded(&bars[stage], phase, a.err, a.poll_limit);
            const float *st = tma_base + stage * S.tma_stage;
            if (colin && zW) {
                dn[0] = st[o]; dn[1] = st[NW * kTmaBoxX + o]; dn[2] = st[2 * NW * kTmaBoxX + o];
                if (M::diag) {
                    const float *sa = st + S.tma_a;
                    const float q0 = sa[o], q1 = sa[NW * kTmaBoxX + o], q2 = sa[2 * NW * kTmaBoxX + o];
                    qn[0] = q0 * q0; qn[1] = q1 * q1; qn[2] = q2 * q2;
                }
            }
            if (M::matvec && s >= 1 && colin && pC >= 0 && pC < nz) {
                const float *sa = tma_base + (stage == 0 ? kTmaStages - 1 : stage - 1) * S.tma_stage + S.tma_a;
                acur[0] = sa[o]; acur[1] = sa[NW * kTmaBoxX + o]; acur[2] = sa[2 * NW * kTmaBoxX + o];
            }
        } else if (M::matvec || M::diag) {
            dn[0] = dnx[0]; dn[1] = dnx[1]; dn[2] = dnx[2];
            if (M::diag) { qn[0] = anx[0] * anx[0]; qn[1] = anx[1] * anx[1]; qn[2] = anx[2] * anx[2]; }
            // prefetch the next planes
            const int p = pW + 1;
            dnx[0] = dnx[1] = dnx[2] = 0.f;
            if (colin && p >= 0 && p < nz) {
                const long v = (long)p * sxy + col;
                dnx[0] = __ldg(a.lin_dT + v); dnx[1] = __ldg(a.lin_dT + N + v); dnx[2] = __ldg(a.lin_dT + 2 * N + v);
            }
            anx[0] = anx[1] = anx[2] = 0.f;
            const int pa = M::matvec ? pW : pW + 1;
            if ((M::diag || inC) && colin && pa >= 0 && pa < nz) {
                const long v = (long)pa * sxy + col;
                anx[0] = __ldg(a.lin_a + v); anx[1] = __ldg(a.lin_a + N + v); anx[2] = __ldg(a.lin_a + 2 * N + v);
            }
        }
        if (colin && zW && !M::diag) {
            const float fz = ((pW & (rz - 1)) + 0.5f) * irz;
            float pu[3];
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) pu[comp] = lerp_fixed(U0[comp], U1[comp], 1.f - fz, fz);
            if (M::matvec) {
                val = dn[0] * pu[0] + dn[1] * pu[1] + dn[2] * pu[2];
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
                rv = ldimg(a.R, (long)pW * sxy + col);
                const float dx00 = t100 - t000, dx10 = t110 - t010, dx01 = t101 - t001, dx11 = t111 - t011;
                const float v00 = fmaf(f[0], dx00, t000), v10 = fmaf(f[0], dx10, t010);
                const float v01 = fmaf(f[0], dx01, t001), v11 = fmaf(f[0], dx11, t011);
                const float dy0 = v10 - v00, dy1 = v11 - v01;
                const float w0 = fmaf(f[1], dy0, v00), w1 = fmaf(f[1], dy1, v01);
                const float dz = w1 - w0;
                val = fmaf(f[2], dz, w0);
                const float ax0 = fmaf(f[1], dx10 - dx00, dx00), ax1 = fmaf(f[1], dx11 - dx01, dx01);
                dn[0] = ins[0] ? fmaf(f[2], ax1 - ax0, ax0) * g.invh[0] * (float)stp[0] : 0.f;
                dn[1] = ins[1] ? fmaf(f[2], dy1 - dy0, dy0) * g.invh[1] * (float)stp[1] : 0.f;
                dn[2] = ins[2] ? dz * g.invh[2] * (float)stp[2] : 0.f;
                if (M::store && inA && pW >= z0 && pW < z0 + TZc) {
                    const long v = (long)pW * sxy + col;
                    a.st_dT[v] = dn[0];
                    a.st_dT[N + v] = dn[1];
                    a.st_dT[2 * N + v] = dn[2];
                }
            }
        }
        // rotate the plane rings
        t_m = t_0; t_0 = t_p; t_p = val;
        r_m = r_0; r_0 = r_p; r_p = rv;
#pragma unroll
        for (int k = 0; k < 3; ++k) { d_2[k] = d_1[k]; d_1[k] = d_0[k]; d_0[k] = dn[k]; }

        float zz[3] = {0.f, 0.f, 0.f};
        if (M::diag) {
            // ------------------------------------------ diagonal: A at plane pA = pW - 1
            float *e1 = ex1 + (s & 1) * NW * 32;
            e1[w * 32 + L] = q1_1;                       // a_y^2 of plane pA for the y-neighbours
            __syncthreads();
            const float q0l = __shfl_up_sync(FULL, q0_1, 1), q0r = __shfl_down_sync(FULL, q0_1, 1);
            if (pA >= z0 && pA < z0 + TZc && inA && colin) {
                // the stored a carries the central-difference scale 1 / (2 h) per axis
                const float b = (q0l + q0r) + (e1[(w - 1) * 32 + L] + e1[(w + 1) * 32 + L]) + (q2_2 + qn[2]);
                zz[0] = b * d_1[0] * d_1[0];
                zz[1] = b * d_1[1] * d_1[1];
                zz[2] = b * d_1[2] * d_1[2];
            }
            q2_2 = q2_1; q2_1 = qn[2]; q0_1 = qn[0]; q1_1 = qn[1];
        } else {
            // ------------------------------------------ exchange plane pC for C's y-neighbours
            float *e1 = ex1 + (s & 1) * NW * 32;
            e1[w * 32 + L] = t_0;
            if (M::warp) ex2[(s & 1) * NW * 32 + w * 32 + L] = r_0;
            __syncthreads();
            // ------------------------------------------ stage C: plane pC
            const float tl = __shfl_up_sync(FULL, t_0, 1), tr = __shfl_down_sync(FULL, t_0, 1);
            float rl = 0.f, rr = 0.f;
            if (M::warp) { rl = __shfl_up_sync(FULL, r_0, 1); rr = __shfl_down_sync(FULL, r_0, 1); }
            float cc[3] = {0.f, 0.f, 0.f};
            const bool actC = pC >= z0 - (M::adj ? 1 : 0) && pC < z0 + TZc + (M::adj ? 1 : 0);
            if (actC && inC) {
                const bool interior = intxy && pC >= 1 && pC <= nz - 2;
                const bool own = inA && pC >= z0 && pC < z0 + TZc;
                if (interior) {
                    const float dt0 = tr - tl, dt1 = e1[(w + 1) * 32 + L] - e1[(w - 1) * 32 + L], dt2 = t_p - t_m;
                    if (M::matvec) {
                        // the stored a' = a / (2 h) per axis: a . G t = a' . (plain differences),
                        // and c' = (2 a . G t) a' carries the adjoint's 1 / (2 h)
                        const float dr = 2.f * (acur[0] * dt0 + acur[1] * dt1 + acur[2] * dt2);
                        cc[0] = dr * acur[0]; cc[1] = dr * acur[1]; cc[2] = dr * acur[2];
                    } else {
                        const float g0 = dt0 * g.inv2h[0], g1 = dt1 * g.inv2h[1], g2 = dt2 * g.inv2h[2];
                        const float *e2 = ex2 + (s & 1) * NW * 32;
                        const float f0 = (rr - rl) * g.inv2h[0];
                        const float f1 = (e2[(w + 1) * 32 + L] - e2[(w - 1) * 32 + L]) * g.inv2h[1];
                        const float f2 = (r_p - r_m) * g.inv2h[2];
                        // the same operation order for <f,g>, |f|^2, |g|^2: f = g gives equal values
                        const float fg = __fmaf_rn(f2, g2, __fmaf_rn(f1, g1, __fmaf_rn(f0, g0, g.eta2)));
                        const float ff = __fmaf_rn(f2, f2, __fmaf_rn(f1, f1, __fmaf_rn(f0, f0, g.eta2)));
                        const float gg = __fmaf_rn(g2, g2, __fmaf_rn(g1, g1, __fmaf_rn(g0, g0, g.eta2)));
                        const float rff = __frcp_rn(ff), rgg = __frcp_rn(gg);
                        // 1 - r^2 = (|f x g|^2 + eta^2 |f - g|^2) / (|f|_eta^2 |g|_eta^2); products
                        // rounded separately: exactly zero when f = g
                        const float x0_ = __fmul_rn(f1, g2) - __fmul_rn(f2, g1);
                        const float x1_ = __fmul_rn(f2, g0) - __fmul_rn(f0, g2);
                        const float x2_ = __fmul_rn(f0, g1) - __fmul_rn(f1, g0);
                        const float e0 = f0 - g0, e1_ = f1 - g1, e2_ = f2 - g2;
                        const float num = x0_ * x0_ + x1_ * x1_ + x2_ * x2_ + g.eta2 * (e0 * e0 + e1_ * e1_ + e2_ * e2_);
                        if (own) kahan_add(dsum, dcomp, num * rff * rgg);
                        // a = dr/dg = (f |g|^2 - <f,g> g) / (|f| |g|^3) (norms with eta)
                        const float q0 = __fmul_rn(f0, gg) - __fmul_rn(fg, g0);
                        const float q1 = __fmul_rn(f1, gg) - __fmul_rn(fg, g1);
                        const float q2 = __fmul_rn(f2, gg) - __fmul_rn(fg, g2);
                        if (M::adj) {   // c = d(1 - r^2)/dg = -2 r a = -2 <f,g> q / (|f|^2 |g|^4)
                            const float sc = -2.f * fg * rff * rgg * rgg;
                            cc[0] = sc * q0; cc[1] = sc * q1; cc[2] = sc * q2;
                        }
                        if (M::store && own) {
                            // a = dr/dg, stored with the central-difference scale 1 / (2 h) per axis
                            const float inv = rsqrtf(ff * gg) * rgg;
                            const long v = (long)pC * sxy + col;
                            a.st_a[v] = q0 * inv * g.inv2h[0];
                            a.st_a[N + v] = q1 * inv * g.inv2h[1];
                            a.st_a[2 * N + v] = q2 * inv * g.inv2h[2];
                        }
                    }
                } else if (M::store && own && colin) {
                    const long v = (long)pC * sxy + col;
                    a.st_a[v] = 0.f;
                    a.st_a[N + v] = 0.f;
                    a.st_a[2 * N + v] = 0.f;
                }
            }
            if (!M::adj) continue;
            // ------------------------------------------ exchange c_y of plane pA
            float *e3 = ex3 + (s & 1) * NW * 32;
            e3[w * 32 + L] = cy_p;
            __syncthreads();
            // ------------------------------------------ stage A: plane pA
            const float cxl_ = __shfl_up_sync(FULL, cx_p, 1), cxr_ = __shfl_down_sync(FULL, cx_p, 1);
            if (pA >= z0 && pA < z0 + TZc && inA && colin) {
                // (the GN product's c' already carries 1 / (2 h))
                const float s0 = M::matvec ? 1.f : g.inv2h[0], s1 = M::matvec ? 1.f : g.inv2h[1];
                const float s2 = M::matvec ? 1.f : g.inv2h[2];
                const float b = (cxl_ - cxr_) * s0 + (e3[(w - 1) * 32 + L] - e3[(w + 1) * 32 + L]) * s1 +
                                (cz_mm - cc[2]) * s2;
                zz[0] = b * d_2[0];
                zz[1] = b * d_2[1];
                zz[2] = b * d_2[2];
            }
            cz_mm = cz_m; cz_m = cc[2]; cx_p = cc[0]; cy_p = cc[1];
        }
        if (!(pA >= z0 && pA < z0 + TZc)) continue;
        // ------------------------------------------------ P^T: x by shuffles, z in the leader's registers
        float lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { lo[k] = wx0 * zz[k]; hi[k] = wx1 * zz[k]; }
#pragma unroll
        for (int lg = 0; lg < 3; ++lg) {
            if (lg >= lrx) break;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] += __shfl_down_sync(FULL, lo[k], 1 << lg);
                hi[k] += __shfl_down_sync(FULL, hi[k], 1 << lg);
            }
        }
        const int zl = pA - z0, czl = zl >> lrz;
        float wz1 = ((zl & (rz - 1)) + 0.5f) * irz, wz0 = 1.f - wz1;
        if (M::diag) { wz0 *= wz0; wz1 *= wz1; }
        if (leader)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                acc[0][0][k] = fmaf(wz0, lo[k], acc[0][0][k]);
                acc[0][1][k] = fmaf(wz1, lo[k], acc[0][1][k]);
                acc[1][0][k] = fmaf(wz0, hi[k], acc[1][0][k]);
                acc[1][1][k] = fmaf(wz1, hi[k], acc[1][1][k]);
            }
        if ((zl & (rz - 1)) == rz - 1) {
            // node plane czl is complete for this row: park it, shift the z window
            if (leader) {
                float *ra = rowA + ((long)czl * TY + (w - 2)) * (CX + 1) * 3;
                float *rb = rowB + ((long)czl * TY + (w - 2)) * (CX + 1) * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ra[cxl * 3 + k] = acc[0][0][k];
                    rb[(cxl + 1) * 3 + k] = acc[1][0][k];
                    acc[0][0][k] = acc[0][1][k]; acc[1][0][k] = acc[1][1][k];
                    acc[0][1][k] = 0.f; acc[1][1][k] = 0.f;
                }
            }
        }
    }

    if (M::reduce) {
        // the node plane above the last cell of the chunk, then the y-reduction of all planes
        const int czl = TZc >> lrz;
        if (leader) {
            float *ra = rowA + ((long)czl * TY + (w - 2)) * (CX + 1) * 3;
            float *rb = rowB + ((long)czl * TY + (w - 2)) * (CX + 1) * 3;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ra[cxl * 3 + k] = acc[0][0][k];
                rb[(cxl + 1) * 3 + k] = acc[1][0][k];
            }
        }
        __syncthreads();
        write_box<TY, M::diag>(g, rowA, rowB, a.boxes, cta, czl + 1, tid, NT);
    }
    if (M::warp) {
        double v = (double)dsum - (double)dcomp;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        __shared__ double red[NW];
        __syncthreads();
        if (L == 0) red[w] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < NW; ++i) t += red[i];
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
        cudaError_t e = allow_max_dynamic_smem(k);                                                       \
        if (e != cudaSuccess) return e;                                                                  \
        k<<<grid, 32 * (TYV + 4), smem, st>>>(a);                                                        \
        return cudaGetLastError();                                                                       \
    } while (0)
#define NGF_TY(TYV)                                       \
    switch (mode) {                                       \
        case MODE_OBJ: NGF_LAUNCH(TYV, MODE_OBJ);         \
        case MODE_LIN: NGF_LAUNCH(TYV, MODE_LIN);         \
        case MODE_GRAD: NGF_LAUNCH(TYV, MODE_GRAD);       \
        case MODE_GRADLIN: NGF_LAUNCH(TYV, MODE_GRADLIN); \
        case MODE_MATVEC: NGF_LAUNCH(TYV, MODE_MATVEC);   \
        case MODE_DIAG: NGF_LAUNCH(TYV, MODE_DIAG);       \
        default: return cudaErrorInvalidValue;            \
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
