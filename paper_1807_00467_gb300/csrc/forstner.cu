// Keypoint extraction of Sec. II-C1 (Foerstner operator): the distinctiveness
// F_D = 1 / trace((G_sigma * grad F grad F^T)^-1), its maximum over a cubic
// window, and the voxels of the mask where F_D equals that maximum.
//
// The keep-or-drop decision compares floating-point values, so the response
// is computed in FP64 (the gradient of FP32 image values is exact in FP64):
// the work is a few hundred FP64 operations per voxel, small even at
// GB300's FP64 rate.  Conventions: central differences and Gaussian taps
// read the nearest voxel outside the volume; the Gaussian has taps -5..5
// with weights exp(-i^2 / (2 sigma^2)) normalised to sum 1; the window of the
// maximum filter spans offsets -3..2 per axis; keypoints are listed in linear
// index order (z, then y, then x).
#include <stdint.h>

#include "../../include/ngfreg.h"
#include "common.cuh"

namespace ngf {
namespace {

constexpr int kRad = 5;            // Gaussian taps -5..5
constexpr int kLo = 3, kHi = 2;    // window offsets -3..2 (6 voxels)
constexpr int kChunk = 4096;       // voxels per block of the compaction

struct Taps {
    double w[2 * kRad + 1];
};

__device__ __forceinline__ int clampi(int v, int hi) { return v < 0 ? 0 : (v > hi ? hi : v); }

// the six products g_a g_b (a <= b) of the central-difference gradient, [6][N]
__global__ void st_products_kernel(int nx, int ny, int nz, const float *img, double *S) {
    const long N = (long)nx * ny * nz;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        auto at = [&](int xx, int yy, int zz) {
            return (double)__ldg(img + ((long)clampi(zz, nz - 1) * ny + clampi(yy, ny - 1)) * nx + clampi(xx, nx - 1));
        };
        const double gx = 0.5 * (at(x + 1, y, z) - at(x - 1, y, z));
        const double gy = 0.5 * (at(x, y + 1, z) - at(x, y - 1, z));
        const double gz = 0.5 * (at(x, y, z + 1) - at(x, y, z - 1));
        S[i] = gx * gx;
        S[N + i] = gx * gy;
        S[2 * N + i] = gx * gz;
        S[3 * N + i] = gy * gy;
        S[4 * N + i] = gy * gz;
        S[5 * N + i] = gz * gz;
    }
}

// one axis of the separable Gaussian over the six channels
__global__ void gauss_pass_kernel(int axis, int nx, int ny, int nz, const double *in, double *out, const Taps t) {
    const long N = (long)nx * ny * nz;
    const int ext = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long)nx * ny);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const int c = axis == 0 ? (int)(i % nx) : (axis == 1 ? (int)((i / nx) % ny) : (int)(i / ((long)nx * ny)));
        const long base = i - (long)c * stride;
        for (int ch = 0; ch < 6; ++ch) {
            const double *p = in + ch * N + base;
            double s = 0.0;
#pragma unroll
            for (int k = -kRad; k <= kRad; ++k) s = fma(t.w[k + kRad], p[(long)clampi(c + k, ext - 1) * stride], s);
            out[ch * N + i] = s;
        }
    }
}

// F_D = det S / (sum of the principal 2 x 2 minors), 0 where that sum is 0
__global__ void response_kernel(long N, const double *S, double *R) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double xx = S[i], xy = S[N + i], xz = S[2 * N + i], yy = S[3 * N + i], yz = S[4 * N + i],
                     zz = S[5 * N + i];
        const double c0 = yy * zz - yz * yz, c1 = xx * zz - xz * xz, c2 = xx * yy - xy * xy;
        const double det = xx * c0 - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
        const double m = c0 + c1 + c2;
        R[i] = m > 0.0 ? det / m : 0.0;
    }
}

// one axis of the window maximum (offsets -3..2, nearest voxel outside)
__global__ void max_pass_kernel(int axis, int nx, int ny, int nz, const double *in, double *out) {
    const long N = (long)nx * ny * nz;
    const int ext = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long)nx * ny);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const int c = axis == 0 ? (int)(i % nx) : (axis == 1 ? (int)((i / nx) % ny) : (int)(i / ((long)nx * ny)));
        const long base = i - (long)c * stride;
        double m = in[base + (long)clampi(c - kLo, ext - 1) * stride];
        for (int k = -kLo + 1; k <= kHi; ++k) m = fmax(m, in[base + (long)clampi(c + k, ext - 1) * stride]);
        out[i] = m;
    }
}

__device__ __forceinline__ bool is_key(long i, const double *R, const double *Rm, const uint8_t *mask) {
    return (!mask || mask[i]) && R[i] > 0.0 && R[i] == Rm[i];
}

// keypoints per block of kChunk voxels
__global__ void __launch_bounds__(256) count_kernel(long N, const double *R, const double *Rm, const uint8_t *mask,
                                                    int *counts) {
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const long b0 = (long)blockIdx.x * kChunk;
    int c = 0;
    for (long i = b0 + threadIdx.x; i < min(N, b0 + kChunk); i += blockDim.x) c += is_key(i, R, Rm, mask);
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// exclusive scan of the block counts (one block), total in offs[nb]
__global__ void __launch_bounds__(1024) scan_kernel(int nb, const int *counts, int *offs) {
    __shared__ int part[1025];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (nb + nt - 1) / nt, a0 = min(nb, tid * chunk), a1 = min(nb, a0 + chunk);
    int s = 0;
    for (int i = a0; i < a1; ++i) s += counts[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int i = 0; i < nt; ++i) {
            const int x = part[i];
            part[i] = t;
            t += x;
        }
        part[nt] = t;
    }
    __syncthreads();
    s = part[tid];
    for (int i = a0; i < a1; ++i) {
        offs[i] = s;
        s += counts[i];
    }
    if (tid == 0) offs[nb] = part[nt];
}

// each block writes its keypoints in index order: 256 consecutive voxels per
// round, ranks from warp ballots and the warps' prefix
__global__ void __launch_bounds__(256) emit_kernel(int nx, int ny, long N, const double *R, const double *Rm,
                                                   const uint8_t *mask, const int *offs, int max_kp, int *kps) {
    __shared__ int wsum[8];
    __shared__ int base;
    if (threadIdx.x == 0) base = offs[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long b0 = (long)blockIdx.x * kChunk;
    for (long r = b0; r < min(N, b0 + kChunk); r += 256) {
        const long i = r + threadIdx.x;
        const bool k = i < N && i < b0 + kChunk && is_key(i, R, Rm, mask);
        const unsigned bal = __ballot_sync(0xffffffffu, k);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int q = 0; q < 8; ++q) {
            pre += q < w ? wsum[q] : 0;
            tot += wsum[q];
        }
        if (k) {
            const int slot = base + pre + __popc(bal & ((1u << lane) - 1u));
            if (slot < max_kp) {
                kps[3 * slot] = (int)(i % nx);
                kps[3 * slot + 1] = (int)((i / nx) % ny);
                kps[3 * slot + 2] = (int)(i / ((long)nx * ny));
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
}

int fgrid(long n) { return (int)((n + 255) / 256 < 152L * 32 ? (n + 255) / 256 : 152L * 32); }

}  // namespace

// workspace: S and its smoothing buffer [6][N] doubles each, R and Rm [N]
// doubles, block counts and offsets
size_t forstner_layout(long N, char *base, double **S, double **T, double **R, double **Rm, int **counts,
                       int **offs) {
    size_t off = 0;
    auto take = [&](size_t b) {
        off = (off + 255) & ~(size_t)255;
        char *p = base ? base + off : nullptr;
        off += b;
        return p;
    };
    const long nb = (N + kChunk - 1) / kChunk;
    *S = (double *)take(sizeof(double) * 6 * N);
    *T = (double *)take(sizeof(double) * 6 * N);
    *R = (double *)take(sizeof(double) * N);
    *Rm = (double *)take(sizeof(double) * N);
    *counts = (int *)take(sizeof(int) * nb);
    *offs = (int *)take(sizeof(int) * (nb + 1));
    return (off + 255) & ~(size_t)255;
}

}  // namespace ngf

using namespace ngf;

extern "C" int kp_forstner_workspace_size(const int32_t *n, size_t *bytes) {
    if (!n || !bytes || n[0] <= 0 || n[1] <= 0 || n[2] <= 0) return RG_EINVAL;
    double *S, *T, *R, *Rm;
    int *c, *o;
    *bytes = forstner_layout((long)n[0] * n[1] * n[2], nullptr, &S, &T, &R, &Rm, &c, &o);
    return RG_OK;
}

extern "C" int kp_forstner(const int32_t *n, const float *F, const uint8_t *mask, double sigma, int32_t max_kp,
                           int32_t *kps, int32_t *count, double *response, void *ws, size_t ws_bytes, void *stream) {
    size_t need;
    if (!n || !F || !kps || !count || max_kp < 0 || !(sigma > 0.0) || kp_forstner_workspace_size(n, &need) != RG_OK ||
        !ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return RG_EINVAL;
    const long N = (long)n[0] * n[1] * n[2];
    const int nb = (int)((N + kChunk - 1) / kChunk);
    double *S, *T, *R, *Rm;
    int *counts, *offs;
    forstner_layout(N, (char *)ws, &S, &T, &R, &Rm, &counts, &offs);
    cudaStream_t st = (cudaStream_t)stream;
    Taps t;
    double sum = 0.0;
    for (int k = -kRad; k <= kRad; ++k) sum += (t.w[k + kRad] = exp(-(double)(k * k) / (2.0 * sigma * sigma)));
    for (int k = 0; k <= 2 * kRad; ++k) t.w[k] /= sum;
    const int g = fgrid(N);
    st_products_kernel<<<g, 256, 0, st>>>(n[0], n[1], n[2], F, S);
    gauss_pass_kernel<<<g, 256, 0, st>>>(0, n[0], n[1], n[2], S, T, t);
    gauss_pass_kernel<<<g, 256, 0, st>>>(1, n[0], n[1], n[2], T, S, t);
    gauss_pass_kernel<<<g, 256, 0, st>>>(2, n[0], n[1], n[2], S, T, t);
    response_kernel<<<g, 256, 0, st>>>(N, T, R);
    max_pass_kernel<<<g, 256, 0, st>>>(0, n[0], n[1], n[2], R, Rm);
    max_pass_kernel<<<g, 256, 0, st>>>(1, n[0], n[1], n[2], Rm, S);
    max_pass_kernel<<<g, 256, 0, st>>>(2, n[0], n[1], n[2], S, Rm);
    count_kernel<<<nb, 256, 0, st>>>(N, R, Rm, mask, counts);
    scan_kernel<<<1, 1024, 0, st>>>(nb, counts, offs);
    emit_kernel<<<nb, 256, 0, st>>>(n[0], n[1], N, R, Rm, mask, offs, max_kp, kps);
    if (cudaGetLastError() != cudaSuccess) return RG_ECUDA;
    int total = 0;
    if (response && cudaMemcpyAsync(response, R, sizeof(double) * N, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RG_ECUDA;
    if (cudaMemcpyAsync(&total, offs + nb, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RG_ECUDA;
    *count = total;
    return RG_OK;
}
