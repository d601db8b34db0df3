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
    return b;
}

}  // namespace ngf
