// NGF distance without any device allocation by the library or the caller.
//
// Some callers cannot allocate device memory when they need the distance:
// code running while a stream is being captured into a CUDA graph (where
// cudaMalloc is not allowed), plug-ins inside a host application that owns
// every device buffer and hands out only the images, or services with a fixed
// memory budget that must not grow after start-up.  They cannot size and
// provide the workspace that rg_ctx_create needs, so this entry point keeps
// the only scratch it uses, one partial sum per CTA of the tile kernel, in a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
#include <mutex>

#include "../../include/ngfreg.h"
#include "kernels.h"

using namespace ngf;

int ngf_host_tile_geom(const rg_image_geom *img, const rg_grid_geom *grid, double eta, TileGeom *t);

// One FP64 partial sum of (1 - r^2) per CTA; each call overwrites the first
// ncta entries before reading them, so nothing has to start at zero.  In host
// code the name g_partials is only a host-side handle: its device address is
// obtained with cudaGetSymbolAddress (scratch_address below).
static __device__ __align__(256) double g_partials[RG_NOALLOC_MAX_CTAS];

namespace {

constexpr int kMaxCtas = RG_NOALLOC_MAX_CTAS;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
double *g_addr[kMaxDevices] = {};   // device address of g_partials, per device

// Sum the partials in a fixed order and scale by the voxel volume.
__global__ void noalloc_sum_kernel(int n, double hbar, double *D) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += g_partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *D = hbar * red[0];
}

// Device address of g_partials on the current device (looked up once per device).
int scratch_address(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RG_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return RG_ECUDA;
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return RG_OK;
}

}  // namespace

extern "C" int ngf_distance_noalloc(const rg_image_geom *img, const rg_grid_geom *grid, const float *R_dev,
                                    const float *T_dev, const float *u_dev, double eta, double *D_dev,
                                    void *cuda_stream) {
    if (!img || !grid || !R_dev || !T_dev || !u_dev || !D_dev || !(eta > 0.0)) return RG_EINVAL;
    TileGeom t;
    if (ngf_host_tile_geom(img, grid, eta, &t) != RG_OK) return RG_EINVAL;
    const long ncta = (long)t.nb[0] * t.nb[1] * t.nb[2];
    if (ncta > kMaxCtas) return RG_ESCRATCH;
    double *partials = nullptr;
    int st = scratch_address(&partials);
    if (st != RG_OK) return st;
    TileArgs<float> a;
    a.g = t;
    a.R = R_dev;
    a.T = T_dev;
    a.u = u_dev;
    a.lin_dT = a.lin_a = nullptr;
    a.st_dT = a.st_a = nullptr;
    a.boxes = nullptr;
    a.dpart = partials;
    a.err = nullptr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (launch_ngf_tile(MODE_OBJ, a, s) != cudaSuccess) return RG_ECUDA;
    const double hbar = img->h[0] * img->h[1] * img->h[2];
    noalloc_sum_kernel<<<1, 256, 0, s>>>((int)ncta, hbar, D_dev);
    return cudaGetLastError() == cudaSuccess ? RG_OK : RG_ECUDA;
}
