// Thread-block view shared by the kernels and the persistent batched PCG
// kernel (pcg_batch.cu): the code of a kernel runs either as its own launch
// (one block = one CUDA block) or as a "virtual block" of a persistent CTA,
// a group of whole warps of the CTA with a named barrier of its own.
#pragma once

#include <cuda_runtime.h>

namespace ngf {

struct VBlock {
    int tid;    // thread index within the block
    int bid;    // block index within the launch (linear)
    int nblk;   // blocks in the launch
    int bar;    // 0: the CUDA block (__syncthreads), else a named barrier id
    int nt;     // threads of the block (a multiple of 32)
    int x, y, z;   // block coordinates of a three-dimensional launch (bid = (z ny + y) nx + x)
    __device__ __forceinline__ void sync() const {
        if (bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};

// The block view of a plain launch.
__device__ __forceinline__ VBlock cuda_block() {
    VBlock b;
    b.tid = threadIdx.x;
    b.bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    b.nblk = gridDim.x * gridDim.y * gridDim.z;
    b.bar = 0;
    b.nt = blockDim.x;
    b.x = blockIdx.x;
    b.y = blockIdx.y;
    b.z = blockIdx.z;
    return b;
}

// A block of a persistent CTA: warps [w0, w0 + nt / 32), named barrier bar,
// block bid of a launch of nx x ny x nz blocks.
__device__ __forceinline__ VBlock warp_block(int tid, int bid, int nx, int ny, int nz, int bar, int nt) {
    VBlock b;
    b.tid = tid;
    b.bid = bid;
    b.nblk = nx * ny * nz;
    b.bar = bar;
    b.nt = nt;
    b.x = bid % nx;
    b.y = (bid / nx) % ny;
    b.z = bid / (nx * ny);
    return b;
}

// The block view of a plain launch on a one-dimensional grid.
__device__ __forceinline__ VBlock cuda_block_1d() {
    VBlock b;
    b.tid = threadIdx.x;
    b.bid = blockIdx.x;
    b.nblk = gridDim.x;
    b.bar = 0;
    b.nt = blockDim.x;
    b.x = blockIdx.x;
    b.y = b.z = 0;
    return b;
}

}  // namespace ngf
