// Shared device helpers and launch descriptors of the ngfreg kernels.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ngf {

// Host-side launch helpers, safe to call from several host threads at once
// (function-local statics are initialised exactly once).  The device is the
// one current at the first call; the library drives one GPU per process.
inline int device_sm_count() {
    static const int sms = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || v <= 0)
            v = 1;
        return v;
    }();
    return sms;
}

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum less the kernel's static shared memory.  That value is fixed per
// kernel, so launches of one kernel with different sizes from concurrent host
// threads cannot lower the limit under one another; a launch asking for more
// than the limit still fails.
template <typename K>
inline cudaError_t allow_max_dynamic_smem(K kernel) {
    static const int optin = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 48 * 1024;
        return v;
    }();
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}


// Image element loads: float32, or IEEE half storing (HU + 1024).  The NGF
// distance only sees differences, so the offset cancels (Eq. (1)).
__device__ __forceinline__ float ldimg(const float *p, long i) { return __ldg(p + i); }
__device__ __forceinline__ float ldimg(const __half *p, long i) { return __half2float(__ldg(p + i)); }

// One interpolation step of the fixed-order FP32 prolongation: w0 * a, then
// fma(w1, b, .), one rounding each (no contraction of the product).
__device__ __forceinline__ float lerp_fixed(float a, float b, float w0, float w1) {
    return __fmaf_rn(w1, b, __fmul_rn(w0, a));
}

// Voxel-tile kernel geometry (host fills, passed by value).
struct TileGeom {
    int n[3];          // voxels
    int m[3];          // nodes
    int rho[3];        // n / (m - 1), a power of two
    int lrho[3];       // log2(rho)
    float irho[3];     // 1 / rho
    float invh[3];     // float(1 / h), used for the FP32 cell decision
    float invh_rel[3]; // 1 - h * float(1 / h): relative error of invh
    float inv2h[3];    // 1 / (2 h) for central differences
    float eta2;        // eta^2
    int TXI;           // voxels per tile along x (multiple of rho[0]; tile + 2-voxel halo <= 32 lanes)
    int TY;            // voxels per tile along y (one warp per row, plus 4 halo rows)
    int TZ;            // voxels per z chunk (multiple of rho[2])
    int nb[3];         // tiles per axis
    int C[3];          // cells per tile per axis (box = C + 1 nodes)
    int nxt, nyt;      // node-tile extent loaded for the prolongation
    int nzt;           // node planes preloaded per CTA (0: two planes streamed as needed)
    int box;           // floats per box per component: (C0+1)(C1+1)(C2+1)
    int tma;           // 1: stream the stored linearisation with TMA (tensor maps valid)
};

template <typename TImg>
struct TileArgs {
    TileGeom g;
    const TImg *R;          // reference image
    const TImg *T;          // template image
    const float *u;         // node field interpolated per voxel (u, or v for the matvec)
    const float *lin_dT;    // stored dT/dy [3][N] (matvec input)
    const float *lin_a;     // stored dr/dg [3][N], component a scaled by 1 / (2 h_a) (matvec input)
    float *st_dT;           // linearisation output dT/dy [3][N]
    float *st_a;            // linearisation output dr/dg [3][N], component a scaled by 1 / (2 h_a)
    float *boxes;           // per-CTA node partials [cta][3][C2+1][C1+1][C0+1]
    double *dpart;          // per-CTA partial sums of (1 - r^2)
    // Stored linearisation streamed by TMA (GN product and diagonal): tensor
    // maps over lin_dT and lin_a as 4-D {x, y, z, component}, box
    // {kTmaBoxX, TY + 4, 1, 3} starting at (x0 - 4, y0 - 2, plane, 0).
    CUtensorMap map_dT, map_a;
    int *err;               // set to 1 if a bounded wait on a TMA barrier gave up
    const int *skip = nullptr;   // nonzero: the launch does nothing (a line-search try after acceptance)
    int poll_limit = 1 << 20;    // polls of a TMA barrier before a wait gives up
    int no_tma = 0;         // test hook: issue no TMA copy (every wait runs out)
};

constexpr int kTmaBoxX = 36;      // floats per TMA box row: tile columns x0-4 .. x0+31
constexpr int kTmaStages = 5;     // planes in flight: 3 ahead of the one being used

// Column geometry of the column-marching GN-product kernel (gn_product.cu):
// a CTA owns TXI x 16 voxel columns in x-y and marches every z plane; lane L
// holds the x columns x0 - 2 + 2L and x0 - 1 + 2L.
constexpr int kColBoxX = 68;      // floats per TMA box row: columns x0-4 .. x0+63
struct ColGeom {
    int n[3];          // voxels
    int m[3];          // nodes
    int rho[3];        // n / (m - 1)
    int lrho[3];       // log2(rho)
    float irho[3];     // 1 / rho
    float inv2h[3];    // 1 / (2 h)
    int TXI;           // owned voxel columns per tile along x (60 - 60 % rho_x)
    int nb[2];         // tiles along x, y
    int C0, C1;        // cells per tile along x, y
    int nxt, nyt;      // node-plane extent read by a tile's prolongation
    int box;           // floats per component of a column's node box: (C0 + 1)(C1 + 1) m3
    int tma;           // 1: tensor maps valid
};

struct ColArgs {
    ColGeom g;
    const float *v;         // node field to prolongate (GN product)
    float *boxes;           // per-column node boxes [column][3][m3][C1 + 1][C0 + 1]
    CUtensorMap map_dT, map_a;   // stored dT/dy, a as {x, y, z, component}, box {68, 20, 1, 3}
    int *err;               // set to 1 if a bounded wait on a TMA barrier gave up
    const int *skip = nullptr;
    int chain = 0;          // set by the launcher: CTAs walk several columns
    int poll_limit = 1 << 20;    // polls of a TMA barrier before a wait gives up
    int no_tma = 0;         // test hook: issue no TMA copy (every wait runs out)
};

// Node-box finaliser: out[c][k] = scale * sum over the CTA boxes holding k.
struct BoxGeom {
    int m[3];
    int nb[3];
    int C[3];
    int box;
};

}  // namespace ngf
