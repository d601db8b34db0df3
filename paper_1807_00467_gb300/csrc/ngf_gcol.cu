// NGF objective, gradient and Gauss-Newton linearisation (Eq. (1)), the
// column-marching form: the pass of ngf_grad.cu (trilinear warp of the
// template at y = x + P u, central-difference gradients of R and of the warped
// template, the per-voxel residual r and 1 - r^2, the adjoint of the central
// difference and P^T onto the grid nodes) on the column layout of the
// GN-product kernel (gn_product_body.cuh).
//
// A CTA (640 threads, persistent) owns a column of TXI x 16 voxels in x-y and
// marches every z plane from -2 to n3 + 1.  Lane L holds the two adjacent x
// columns x0 - 2 + 2L and x0 - 1 + 2L (one f32x2 instruction serves both),
// warp w the row y0 - 2 + w.  Per plane step, three stages:
//   W (plane pW): y = x + P u by the fixed-order FP32 interpolation (x, then
//                 y, then z, each step fma(w1, b, w0 a)), the FP32 cell
//                 decision, 8 template samples per voxel, T(y) and dT/dy
//                 (stored for the GN product); R(x)
//   C (plane pW - 1): f = grad R, g = grad T(y), 1 - r^2 in cancellation-free
//                 form, a = dr/dg / (2 h) (stored), c = d(1 - r^2)/dg / (2 h)
//   A (plane pW - 2): adjoint of the central difference of c, times dT/dy,
//                 onto the column's two z-node planes in registers
// x neighbours by one shuffle per direction (the pair's other column is
// local), y neighbours through double-buffered exchange rows, z neighbours in
// registers; one barrier per plane.  Each thread keeps the dT/dy of its last
// two planes (read back by stage A) and P u at the two node planes of the
// current cell in shared-memory slots of its own rather than in registers
// (no register spills).  The stored linearisation is
// written once per voxel with 8-byte stores.  P^T: completed node planes are parked per
// lane (hat-weighted lower and upper parts), reduced along x by all threads
// in the next plane and along y in the plane after, into the column's node
// box [3][m3][C1 + 1][C0 + 1] (the GN product's boxes; the node pass sums
// neighbouring columns).  The objective-only mode runs W and C.
#include "common.cuh"
#include "kernels.h"

namespace ngf {

namespace {

constexpr int kTY = 16, kNW = kTY + 4, kNT = 32 * kNW;
constexpr int kEx = kNW * 64;   // floats per exchange buffer (a float2 per lane and warp)
constexpr unsigned FULL = 0xffffffffu;

struct GcSmem {
    int ext, exr, exc, nodes, park, xr, dts, us, total;
};

__host__ __device__ inline GcSmem gc_smem(const ColGeom &g, bool adj) {
    GcSmem s;
    int off = 0;
    s.ext = off; off += 2 * kEx;                                   // T(y) of plane C, double-buffered
    s.exr = off; off += 2 * kEx;                                   // R of plane C
    s.exc = off; off += adj ? 2 * kEx : 0;                         // c_y of plane A
    s.nodes = off; off += 4 * ((g.nyt * g.nxt + 31) & ~31) * 4;    // node planes of u, [slot][y][x][xyz_]
    s.park = off; off += adj ? 2 * kTY * 32 * 6 : 0;               // parked lane parts of 2 node planes
    s.xr = off; off += adj ? 2 * kTY * (g.C0 + 1) * 3 : 0;         // x-reduced rows of 2 node planes
    s.dts = off; off += adj ? 2 * 3 * kNT * 2 : 0;                 // per thread: dT/dy of 2 planes
    s.us = off; off += 2 * 3 * kNT * 2;                             // per thread: P u at 2 node planes
    s.total = off;
    return s;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
// one step of the fixed-order interpolation, fma(w1, b, w0 a), per lane
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 w0, float2 w1) { return fma2(w1, b, mul2(w0, a)); }

// a b - c d and a - b per lane with scalar round-to-nearest operations (each
// product rounded on its own: exactly zero when a b and c d are the same product)
__device__ __forceinline__ float2 xprod(float2 a, float2 b, float2 c, float2 d) {
    return make_float2(__fsub_rn(__fmul_rn(a.x, b.x), __fmul_rn(c.x, d.x)),
                       __fsub_rn(__fmul_rn(a.y, b.y), __fmul_rn(c.y, d.y)));
}
__device__ __forceinline__ float2 diff_rn(float2 a, float2 b) {
    return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <typename T>
__device__ __forceinline__ float2 ld2img(const T *p, long i);
template <>
__device__ __forceinline__ float2 ld2img(const float *p, long i) {
    return __ldg(reinterpret_cast<const float2 *>(p + i));
}
template <>
__device__ __forceinline__ float2 ld2img(const __half *p, long i) {
    return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p + i)));
}

// Per-axis placement of one voxel's template sample from its FP32 cell
// decision (the definition shared with the oracle): cell c (clamped), step
// +-1 to the second sample, fraction f, and whether the derivative along the
// axis is taken (not clamped).
struct Place {
    int c, st;
    float f;
    bool in;
};
__device__ __forceinline__ Place place(float pu, float ih, float ihrel, int i, int n) {
    const float q = __fmul_rn(pu, ih);
    const float fl = floorf(q);
    const float e = __fmaf_rn(pu, ih, -q);
    const float fr = (q - fl) + __fmaf_rn(q, ihrel, e);
    const int k = i + (int)fl;
    const bool lo = k < 0, hi = k >= n - 1;
    Place p;
    p.c = lo ? 0 : (hi ? n - 1 : k);
    p.st = hi ? -1 : 1;
    p.in = !lo && (!hi || (k == n - 1 && q - fl == 0.f));
    p.f = (lo || hi) ? 0.f : fr;
    return p;
}

}  // namespace

template <int MODE, typename TImg, int RZ, int RXY>
__global__ void __launch_bounds__(kNT, 1) ngf_gcol_kernel(const __grid_constant__ GcolArgs<TImg> a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    constexpr bool ADJ = MODE != MODE_OBJ, STORE = MODE == MODE_GRADLIN;
    extern __shared__ __align__(16) float smem[];
    const ColGeom &g = a.g;
    const GcSmem S = gc_smem(g, ADJ);

    const int tid = threadIdx.x, L = tid & 31, w = tid >> 5;
    const int ncols = g.nb[0] * g.nb[1];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], sxy = nx * ny, N = sxy * nz;
    const int lrx = g.lrho[0], lry = g.lrho[1], lrz = g.lrho[2];
    const int rx = g.rho[0], half = rx >> 1, rzm = g.rho[2] - 1;
    const float irz = g.irho[2];
    const int nsteps = nz + 4;
    const int nxt = g.nxt, nplane = nxt * g.nyt, npad = (nplane + 31) & ~31;
    const int C0 = g.C0, C1 = g.C1, XR = (C0 + 1) * 3;
    const long mxy = (long)g.m[0] * g.m[1], Mn = mxy * g.m[2];
    const float ih0 = a.invh[0], ih1 = a.invh[1], ih2 = a.invh[2];
    const float2 i2h0 = bc2(g.inv2h[0]), i2h1 = bc2(g.inv2h[1]), i2h2 = bc2(g.inv2h[2]), eta2 = bc2(a.eta2);

    float4 *s_nodes = reinterpret_cast<float4 *>(smem + S.nodes);
    float2 *park = reinterpret_cast<float2 *>(smem + S.park);   // [2 slots][16 rows][32 lanes][3] (lo, hi)
    float *xr = smem + S.xr;                                     // [2 slots][16 rows][C0 + 1][3]
    float2 *ex_t = reinterpret_cast<float2 *>(smem + S.ext) + w * 32 + L;
    float2 *ex_r = reinterpret_cast<float2 *>(smem + S.exr) + w * 32 + L;
    float2 *ex_c = reinterpret_cast<float2 *>(smem + S.exc) + w * 32 + L;
    const int up = w > 0 ? -32 : 0, dn = w < kNW - 1 ? 32 : 0;   // in float2; the outer rows read themselves
    constexpr int exh = kEx / 2;

    const int i0 = 2 * L - 2;                                    // this lane's pair: local x i0, i0 + 1
    const bool interior_warp = w >= 2 && w < kTY + 2;
    const bool own_pair = interior_warp && i0 >= 0 && i0 < g.TXI;
    const int ph = i0 & (rx - 1);
    float2 *park_lane = park + ((w - 2) * 32 + L) * 3;
    const bool node_warp = (kNW - 1 - w) * 32 < npad;
    const int ntid = tid - (kNT - npad);
    const int lane_major = L * kNW + w;
    const float invXR = 1.f / XR, invNP = 1.f / ((C1 + 1) * (C0 + 1)), invC0 = 1.f / (C0 + 1);
    auto idiv = [](int v, float inv) { return __float2int_rz(((float)v + 0.5f) * inv); };

    for (int t = blockIdx.x; t < ncols; t += gridDim.x) {
        const int x0 = (t % g.nb[0]) * g.TXI, y0 = (t / g.nb[0]) * kTY;
        const int kx_lo = (x0 - 2) >> lrx, ky_lo = (y0 - 2) >> lry;
        float *box = a.boxes + (long)t * 3 * g.box;

        // node planes of u through a 4-slot ring (cp.async, zero outside the grid)
        int ngo = -1;
        if (ntid >= 0 && ntid < nplane) {
            const int ly = ntid / nxt, lx = ntid - ly * nxt;
            const int ux = kx_lo + lx, uy = ky_lo + ly;
            if (ux >= 0 && ux < g.m[0] && uy >= 0 && uy < g.m[1]) ngo = uy * g.m[0] + ux;
        }
        auto node_copy = [&](int kz) {   // node warps only (warp-uniform callers)
            const bool in = ngo >= 0 && kz >= 0 && kz < g.m[2];
            const float *p = in ? a.u + kz * mxy + ngo : a.u;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_nodes + (kz & 3) * npad + ntid);
            const uint32_t n = in ? 4u : 0u;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(p), "r"(n) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 4), "l"(p + Mn), "r"(n) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 8), "l"(p + 2 * Mn), "r"(n) : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        const int cz0 = (-2) >> lrz;
        if (node_warp) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            for (int i = 0; i < 4; ++i) node_copy(cz0 + i);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }

        // this pair's columns: in the volume, interior in x-y, voxel index
        const int gx = x0 + i0, gy = y0 - 2 + w;
        const bool rowin = gy >= 0 && gy < ny, rowint = gy >= 1 && gy <= ny - 2;
        const bool in_e = rowin && gx >= 0 && gx < nx, in_o = rowin && gx + 1 >= 0 && gx + 1 < nx;
        const bool int_e = rowint && gx >= 1 && gx <= nx - 2, int_o = rowint && gx + 1 >= 1 && gx + 1 <= nx - 2;
        const bool own_e = own_pair && in_e, own_o = own_pair && in_o;
        const bool pair_in = in_e && in_o;   // both columns in the volume (nx is even, gx even)
        const int col = pair_in ? gy * nx + gx : 0;
        // fixed-order interpolation weights of the pair (both columns share the cell)
        const int cxg = gx >> lrx, cyg = gy >> lry;
        const float2 fx2 = make_float2(((gx - (cxg << lrx)) + 0.5f) * g.irho[0],
                                       ((gx + 1 - (cxg << lrx)) + 0.5f) * g.irho[0]);
        const float2 wx02 = make_float2(1.f - fx2.x, 1.f - fx2.y);
        const float fy = ((gy - (cyg << lry)) + 0.5f) * g.irho[1];
        const float2 fy2 = bc2(fy), wy02 = bc2(1.f - fy);
        const int qoff = (cyg - ky_lo) * nxt + (cxg - kx_lo);
        auto bilinear = [&](int kz, float2 *U) {
            const float4 *q = s_nodes + (kz & 3) * npad + qoff;
            const float4 n00 = q[0], n10 = q[1], n01 = q[nxt], n11 = q[nxt + 1];
            U[0] = lerp2(lerp2(bc2(n00.x), bc2(n10.x), wx02, fx2), lerp2(bc2(n01.x), bc2(n11.x), wx02, fx2), wy02, fy2);
            U[1] = lerp2(lerp2(bc2(n00.y), bc2(n10.y), wx02, fx2), lerp2(bc2(n01.y), bc2(n11.y), wx02, fx2), wy02, fy2);
            U[2] = lerp2(lerp2(bc2(n00.z), bc2(n10.z), wx02, fx2), lerp2(bc2(n01.z), bc2(n11.z), wx02, fx2), wy02, fy2);
        };
        auto park_plane = [&](const float2 *acc, int kz) {
            if (!interior_warp) return;
            float2 *dst = park_lane + (kz & 1) * (kTY * 32 * 3);
            const float irx = g.irho[0], fe = (ph + 0.5f) * irx;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float ve = own_e ? acc[k].x : 0.f, vo = own_o ? acc[k].y : 0.f;
                const float sum = ve + vo, hi = fmaf(fe, sum, vo * irx);
                dst[k] = make_float2(sum - hi, hi);
            }
        };
        auto x_pass = [&](int kz) {
            const float2 *src = park + (kz & 1) * (kTY * 32 * 3);
            float *dst = xr + (kz & 1) * (kTY * XR);
            if constexpr (RXY > 0) {
                constexpr int H = RXY / 2, C0c = (60 - 60 % RXY) / RXY, XRc = (C0c + 1) * 3, NX = kTY * XRc;
#pragma unroll
                for (int i = 0; i < (NX + kNT - 1) / kNT; ++i) {
                    const int it = tid + i * kNT;
                    if (NX % kNT == 0 || it < NX) {
                        const int row = it / XRc, r = it % XRc, jx = r / 3, k = r % 3;
                        const float2 *p = src + (row * 32 + 1 + jx * H) * 3 + k;
                        const float2 *pl = jx < C0c ? p : p - 3 * H, *ph_ = jx > 0 ? p : p + 3 * H;
                        float lo = 0.f, hi = 0.f;
#pragma unroll
                        for (int q = 0; q < H; ++q) {
                            lo += pl[3 * q].x;
                            hi += ph_[3 * (q - H)].y;
                        }
                        dst[it] = (jx < C0c ? lo : 0.f) + (jx > 0 ? hi : 0.f);
                    }
                }
            } else {
                for (int it = lane_major; it < kTY * XR; it += kNT) {
                    const int row = idiv(it, invXR), r = it - row * XR, jx = (r * 43) >> 7, k = r - jx * 3;
                    const float2 *p = src + (row * 32 + 1 + jx * half) * 3 + k;
                    const float2 *pl = jx < C0 ? p : p - 3 * half, *ph_ = jx > 0 ? p : p + 3 * half;
                    float lo, hi;
                    switch (half) {
                        case 1: lo = pl[0].x; hi = ph_[-3].y; break;
                        case 2: lo = pl[0].x + pl[3].x; hi = ph_[-6].y + ph_[-3].y; break;
                        default: lo = (pl[0].x + pl[3].x) + (pl[6].x + pl[9].x); hi = (ph_[-12].y + ph_[-9].y) + (ph_[-6].y + ph_[-3].y);
                    }
                    dst[it] = (jx < C0 ? lo : 0.f) + (jx > 0 ? hi : 0.f);
                }
            }
        };
        auto y_pass = [&](int kz) {
            const int ry = g.rho[1];
            const int np = (C1 + 1) * (C0 + 1);
            for (int it = (tid + kNT - 64) % kNT; it < 3 * np; it += kNT) {
                const int k = idiv(it, invNP), r = it - k * np;
                const int jy = idiv(r, invC0), jx = r - jy * (C0 + 1);
                const float *src = xr + (kz & 1) * (kTY * XR) + jx * 3 + k;
                float acc = 0.f;
                for (int i = 0; i < ry; ++i) {
                    const float f = (i + 0.5f) * g.irho[1];
                    if (jy < C1) acc = fmaf(1.f - f, src[(jy * ry + i) * XR], acc);
                    if (jy > 0) acc = fmaf(f, src[((jy - 1) * ry + i) * XR], acc);
                }
                box[(long)k * g.box + (long)kz * np + r] = acc;
            }
        };

        {
            float *ex = smem + S.ext;
            for (int i = tid; i < (ADJ ? 6 : 4) * kEx; i += kNT) ex[i] = 0.f;
        }
        __syncthreads();   // node ring filled, exchange rows cleared; the previous column's passes are done

        const float2 z2 = make_float2(0.f, 0.f);
        float2 *usm = reinterpret_cast<float2 *>(smem + S.us) + tid;   // [slot][k], stride kNT
        int u0s = 0;   // slot of the lower node plane
        {
            float2 Ut[3];
            bilinear(cz0, Ut);
            for (int k = 0; k < 3; ++k) usm[k * kNT] = Ut[k];
            bilinear(cz0 + 1, Ut);
            for (int k = 0; k < 3; ++k) usm[(3 + k) * kNT] = Ut[k];
        }
        float2 tm = z2, t0 = z2, rm = z2, r0 = z2;        // T(y) and R at planes pC - 1, pC
        // this thread's dT/dy of planes pW - 2 and pW - 1: [slot = plane parity][component], stride kNT
        float2 *dts = reinterpret_cast<float2 *>(smem + S.dts) + tid;
        if (ADJ)
            for (int i = 0; i < 6; ++i) dts[i * kNT] = z2;
        float2 cxp = z2, czm2 = z2, czm1 = z2;             // c of the adjoint at planes pA, pA - 1
        float2 acc0[3] = {z2, z2, z2}, acc1[3] = {z2, z2, z2};
        float ds_e = 0.f, dc_e = 0.f, ds_o = 0.f, dc_o = 0.f;   // Kahan sums of 1 - r^2
        int xk = -1, yk = -1;

        for (int s0 = 0; s0 < nsteps; s0 += 2) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int s = s0 + j;
                if (s >= nsteps) break;
                const int pW = s - 2, pC = pW - 1;
                const int phW = RZ ? ((j - 2) & (RZ - 1)) : (pW & rzm);
                const float fz = RZ ? (phW + 0.5f) / (float)(RZ ? RZ : 1) : (phW + 0.5f) * irz;
                const bool cell_start = phW == 0 && s > 0;
                if (cell_start && node_warp) asm volatile("cp.async.wait_group 1;" ::: "memory");
                __syncthreads();
                if (ADJ) {
                    if (yk >= 0) y_pass(yk);
                    if (xk >= 0) x_pass(xk);
                    yk = xk;
                    xk = -1;
                }
                if (cell_start) {
                    const int kz = pW >> lrz;
                    float2 Ut[3];
                    bilinear(kz + 1, Ut);
                    for (int k = 0; k < 3; ++k) usm[(u0s * 3 + k) * kNT] = Ut[k];   // over the old lower plane
                    u0s ^= 1;
                    if (node_warp) node_copy(kz + 3);
                }

                // ------------------------------------------------ stage W: plane pW
                float2 val, dw[3];
                {
                    const float2 fz2 = bc2(fz), wz2 = bc2(1.f - fz);
                    const float2 *ul = usm + u0s * 3 * kNT, *uh = usm + (u0s ^ 1) * 3 * kNT;
                    const float2 pu0 = lerp2(ul[0], uh[0], wz2, fz2), pu1 = lerp2(ul[kNT], uh[kNT], wz2, fz2);
                    const float2 pu2 = lerp2(ul[2 * kNT], uh[2 * kNT], wz2, fz2);
                    const Place xe = place(pu0.x, ih0, a.invh_rel[0], gx, nx), xo = place(pu0.y, ih0, a.invh_rel[0], gx + 1, nx);
                    const Place ye = place(pu1.x, ih1, a.invh_rel[1], gy, ny), yo = place(pu1.y, ih1, a.invh_rel[1], gy, ny);
                    const Place ze = place(pu2.x, ih2, a.invh_rel[2], pW, nz), zo = place(pu2.y, ih2, a.invh_rel[2], pW, nz);
                    const TImg *Te = a.T + (ze.c * sxy + ye.c * nx + xe.c), *To = a.T + (zo.c * sxy + yo.c * nx + xo.c);
                    const int sxe = xe.st, sye = ye.st * nx, sze = ze.st * sxy;
                    const int sxo = xo.st, syo = yo.st * nx, szo = zo.st * sxy;
                    const float2 t000 = make_float2(ldimg(Te, 0), ldimg(To, 0));
                    const float2 t100 = make_float2(ldimg(Te, sxe), ldimg(To, sxo));
                    const float2 t010 = make_float2(ldimg(Te, sye), ldimg(To, syo));
                    const float2 t110 = make_float2(ldimg(Te, sye + sxe), ldimg(To, syo + sxo));
                    const float2 t001 = make_float2(ldimg(Te, sze), ldimg(To, szo));
                    const float2 t101 = make_float2(ldimg(Te, sze + sxe), ldimg(To, szo + sxo));
                    const float2 t011 = make_float2(ldimg(Te, sze + sye), ldimg(To, szo + syo));
                    const float2 t111 = make_float2(ldimg(Te, sze + sye + sxe), ldimg(To, szo + syo + sxo));
                    const float2 f0 = make_float2(xe.f, xo.f), f1 = make_float2(ye.f, yo.f), f2 = make_float2(ze.f, zo.f);
                    const float2 dx00 = sub2(t100, t000), dx10 = sub2(t110, t010), dx01 = sub2(t101, t001),
                                 dx11 = sub2(t111, t011);
                    const float2 v00 = fma2(f0, dx00, t000), v10 = fma2(f0, dx10, t010);
                    const float2 v01 = fma2(f0, dx01, t001), v11 = fma2(f0, dx11, t011);
                    const float2 dy0 = sub2(v10, v00), dy1 = sub2(v11, v01);
                    const float2 w0 = fma2(f1, dy0, v00), w1 = fma2(f1, dy1, v01);
                    const float2 dz = sub2(w1, w0);
                    val = fma2(f2, dz, w0);
                    if (ADJ) {
                        const float2 ax0 = fma2(f1, sub2(dx10, dx00), dx00), ax1 = fma2(f1, sub2(dx11, dx01), dx01);
                        // derivative scale 1/h with the step's sign, zero along a clamped axis
                        const float2 sx2 = make_float2(xe.in ? ih0 * (float)xe.st : 0.f, xo.in ? ih0 * (float)xo.st : 0.f);
                        const float2 sy2 = make_float2(ye.in ? ih1 * (float)ye.st : 0.f, yo.in ? ih1 * (float)yo.st : 0.f);
                        const float2 sz2 = make_float2(ze.in ? ih2 * (float)ze.st : 0.f, zo.in ? ih2 * (float)zo.st : 0.f);
                        dw[0] = mul2(fma2(f2, sub2(ax1, ax0), ax0), sx2);
                        dw[1] = mul2(fma2(f2, sub2(dy1, dy0), dy0), sy2);
                        dw[2] = mul2(dz, sz2);
                        if (STORE && own_pair && pair_in && pW >= 0 && pW < nz) {
                            const long v = (long)pW * sxy + col;
                            *reinterpret_cast<float2 *>(a.st_dT + v) = dw[0];
                            *reinterpret_cast<float2 *>(a.st_dT + N + v) = dw[1];
                            *reinterpret_cast<float2 *>(a.st_dT + 2 * (long)N + v) = dw[2];
                        }
                    }
                }
                const float2 rv = (pair_in && pW >= 0 && pW < nz) ? ld2img(a.R, (long)pW * sxy + col) : z2;

                // ------------------------------------------------ stage C: plane pC
                const int bo = (j & 1) * exh;
                float2 c0 = z2, c1 = z2, c2 = z2;
                {
                    const float tl = __shfl_up_sync(FULL, t0.y, 1), tr = __shfl_down_sync(FULL, t0.x, 1);
                    const float rl = __shfl_up_sync(FULL, r0.y, 1), rr = __shfl_down_sync(FULL, r0.x, 1);
                    const float2 g0 = mul2(make_float2(t0.y - tl, tr - t0.x), i2h0);
                    const float2 g1 = mul2(sub2(ex_t[bo + dn], ex_t[bo + up]), i2h1);
                    const float2 g2 = mul2(sub2(val, tm), i2h2);
                    const float2 f0 = mul2(make_float2(r0.y - rl, rr - r0.x), i2h0);
                    const float2 f1 = mul2(sub2(ex_r[bo + dn], ex_r[bo + up]), i2h1);
                    const float2 f2 = mul2(sub2(rv, rm), i2h2);
                    // the same operation order for <f,g>, |f|^2, |g|^2: f = g gives equal values
                    const float2 fg = fma2(f2, g2, fma2(f1, g1, fma2(f0, g0, eta2)));
                    const float2 ff = fma2(f2, f2, fma2(f1, f1, fma2(f0, f0, eta2)));
                    const float2 gg = fma2(g2, g2, fma2(g1, g1, fma2(g0, g0, eta2)));
                    const float2 rff = make_float2(__frcp_rn(ff.x), __frcp_rn(ff.y));
                    const float2 rgg = make_float2(__frcp_rn(gg.x), __frcp_rn(gg.y));
                    const bool zin = pC >= 1 && pC <= nz - 2;
                    const bool ie = int_e && zin, io = int_o && zin;
                    // 1 - r^2 = (|f x g|^2 + eta^2 |f - g|^2) / (|f|_eta^2 |g|_eta^2); the
                    // products rounded separately (scalar round-to-nearest operations: a
                    // packed product next to a packed difference need not round the same
                    // way), so the value is exactly zero when f = g
                    const float2 x0_ = xprod(f1, g2, f2, g1), x1_ = xprod(f2, g0, f0, g2), x2_ = xprod(f0, g1, f1, g0);
                    const float2 e0 = diff_rn(f0, g0), e1 = diff_rn(f1, g1), e2 = diff_rn(f2, g2);
                    const float2 num = fma2(eta2, fma2(e2, e2, fma2(e1, e1, mul2(e0, e0))),
                                            fma2(x2_, x2_, fma2(x1_, x1_, mul2(x0_, x0_))));
                    const float2 dv = mul2(mul2(num, rff), rgg);
                    const bool oz = pC >= 0 && pC < nz;
                    kahan_add(ds_e, dc_e, (own_e && oz && ie) ? dv.x : 0.f);
                    kahan_add(ds_o, dc_o, (own_o && oz && io) ? dv.y : 0.f);
                    if (ADJ) {
                        // a = dr/dg = (f |g|^2 - <f,g> g) / (|f| |g|^3); c = d(1 - r^2)/dg =
                        // -2 <f,g> q / (|f|^2 |g|^4); both times 1/(2h) per axis
                        const float2 q0 = xprod(f0, gg, fg, g0), q1 = xprod(f1, gg, fg, g1);
                        const float2 q2 = xprod(f2, gg, fg, g2);   // zero when f = g
                        const float2 scv = mul2(mul2(mul2(mul2(bc2(-2.f), fg), rff), rgg), rgg);
                        const float2 sc = make_float2(ie ? scv.x : 0.f, io ? scv.y : 0.f);
                        c0 = mul2(mul2(sc, q0), i2h0);
                        c1 = mul2(mul2(sc, q1), i2h1);
                        c2 = mul2(mul2(sc, q2), i2h2);
                        if (STORE && own_pair && pair_in && oz) {
                            const float2 inv = make_float2(ie ? rsqrtf(ff.x * gg.x) * rgg.x : 0.f,
                                                           io ? rsqrtf(ff.y * gg.y) * rgg.y : 0.f);
                            const long v = (long)pC * sxy + col;
                            *reinterpret_cast<float2 *>(a.st_a + v) = mul2(mul2(q0, inv), i2h0);
                            *reinterpret_cast<float2 *>(a.st_a + N + v) = mul2(mul2(q1, inv), i2h1);
                            *reinterpret_cast<float2 *>(a.st_a + 2 * (long)N + v) = mul2(mul2(q2, inv), i2h2);
                        }
                    }
                }

                // ------------------------------------------------ stage A: plane pA = pW - 2
                if (ADJ) {
                    const float cxl = __shfl_up_sync(FULL, cxp.y, 1), cxr = __shfl_down_sync(FULL, cxp.x, 1);
                    const int phA = RZ ? (j & (RZ - 1)) : ((pW - 2) & rzm);
                    const float wz1 = RZ ? (phA + 0.5f) / (float)(RZ ? RZ : 1) : (phA + 0.5f) * irz;
                    const float2 bx = make_float2(cxl - cxp.y, cxp.x - cxr);
                    const float2 bsum = add2(add2(bx, sub2(ex_c[bo + up], ex_c[bo + dn])), sub2(czm2, c2));
                    const float2 b1 = mul2(bc2(wz1), bsum), b0 = sub2(bsum, b1);
                    for (int k = 0; k < 3; ++k) {
                        const float2 d2k = dts[((j & 1) * 3 + k) * kNT];   // dT/dy of plane pA (this slot)
                        acc0[k] = fma2(b0, d2k, acc0[k]);
                        acc1[k] = fma2(b1, d2k, acc1[k]);
                    }
                    if (phA == (RZ ? RZ - 1 : rzm) && s >= 4) {
                        const int kz = (s - 4) >> lrz;   // node plane (pA >> lrz) is complete
                        park_plane(acc0, kz);
                        xk = kz;
                        for (int k = 0; k < 3; ++k) {
                            acc0[k] = acc1[k];
                            acc1[k] = z2;
                        }
                    }
                    ex_c[exh - bo] = c1;
                    czm2 = czm1; czm1 = c2;
                    cxp = c0;
                    for (int k = 0; k < 3; ++k) dts[((j & 1) * 3 + k) * kNT] = dw[k];
                }
                // ------------------------------------------------ hand over to the next plane
                ex_t[exh - bo] = val;
                ex_r[exh - bo] = rv;
                tm = t0; t0 = val;
                rm = r0; r0 = rv;
            }
        }
        if (ADJ) {   // the pending passes and the top node plane (above the last cell)
            __syncthreads();
            if (yk >= 0) y_pass(yk);
            if (xk >= 0) x_pass(xk);
            park_plane(acc0, g.m[2] - 1);
            __syncthreads();
            if (xk >= 0) y_pass(xk);
            x_pass(g.m[2] - 1);
            __syncthreads();
            y_pass(g.m[2] - 1);
        }
        // the column's sum of 1 - r^2 (FP64 across the threads)
        {
            double v = ((double)ds_e - (double)dc_e) + ((double)ds_o - (double)dc_o);
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
            __shared__ double red[kNW];
            if (L == 0) red[w] = v;
            __syncthreads();
            if (tid == 0) {
                double sum = 0.0;
                for (int i = 0; i < kNW; ++i) sum += red[i];
                a.dpart[t] = sum;
            }
        }
    }
}

bool ngf_gcol_supported(const ColGeom &g) {
    if (g.rho[0] < 2 || g.n[0] % 2 || g.n[0] < 64 || g.n[1] < 20 || g.m[2] > 256 || g.nxt * g.nyt > kNT) return false;
    return (size_t)gc_smem(g, true).total * sizeof(float) <= 227u * 1024u;
}

template <typename TImg>
static cudaError_t launch_gcol(int mode, const GcolArgs<TImg> &a, cudaStream_t st) {
    if (!ngf_gcol_supported(a.g)) return cudaErrorInvalidValue;
    const bool adj = mode != MODE_OBJ;
    const size_t smem = sizeof(float) * (size_t)gc_smem(a.g, adj).total;
    const int ncols = a.g.nb[0] * a.g.nb[1];
    const int sms = device_sm_count();
    const int grid = ncols < sms ? ncols : sms;
    auto run = [&](auto kernel) {
        cudaError_t e = allow_max_dynamic_smem(kernel);
        if (e != cudaSuccess) return e;
        kernel<<<grid, kNT, smem, st>>>(a);
        return cudaGetLastError();
    };
    const bool r44 = a.g.rho[0] == 4 && a.g.rho[1] == 4, r2 = a.g.rho[2] == 2;
#define NGF_GC(M) (r44 ? (r2 ? run(ngf_gcol_kernel<M, TImg, 2, 4>) : run(ngf_gcol_kernel<M, TImg, 0, 4>)) \
                       : (r2 ? run(ngf_gcol_kernel<M, TImg, 2, 0>) : run(ngf_gcol_kernel<M, TImg, 0, 0>)))
    switch (mode) {
        case MODE_OBJ: return NGF_GC(MODE_OBJ);
        case MODE_GRAD: return NGF_GC(MODE_GRAD);
        case MODE_GRADLIN:
        case MODE_LIN: return NGF_GC(MODE_GRADLIN);
        default: return cudaErrorInvalidValue;
    }
#undef NGF_GC
}

cudaError_t launch_ngf_gcol(int mode, const GcolArgs<float> &a, cudaStream_t st) { return launch_gcol(mode, a, st); }
cudaError_t launch_ngf_gcol(int mode, const GcolArgs<__half> &a, cudaStream_t st) { return launch_gcol(mode, a, st); }

}  // namespace ngf
