// Deterministic grid reductions without waiting: every block publishes an FP64
// partial, and the block that finishes last (atomic ticket) sums all partials
// in a fixed order.  Used by the PCG vector kernels.
#pragma once

#include "kernels.h"

namespace ngf {

__device__ __forceinline__ double lb_warp_sum(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// FP32 warp sum (fixed shuffle tree); FP64 is ~1/64 of the FP32 rate on this
// part, so only the per-warp partials are widened
__device__ __forceinline__ float lb_warp_sum_f(float v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum of part[0..n) in a fixed order (lane-strided, then a fixed shuffle
// tree) by one warp; valid in every lane.
__device__ __forceinline__ double lb_sum_parts(const double *part, int n) {
    double s = 0.0;
    for (int i = threadIdx.x & 31; i < n; i += 32) s += __ldcg(part + i);
    return lb_warp_sum(s);
}

// True in the block that arrives last (after every block has published its
// partials); that block resets the ticket for the next launch.
__device__ __forceinline__ bool lb_last_block(unsigned *ticket, unsigned nblocks) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        is_last = t == nblocks - 1;
        if (is_last) *ticket = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

// PCG step length from p.q: alpha = r.z / p.q; the solve stops on a
// non-positive curvature p.q or a vanishing r.z (one thread).
__device__ __forceinline__ void pcg_set_alpha(PcgScalars *sc, double pq) {
    sc->pq = pq;
    if (sc->stop || !(sc->rz != 0.0) || !(pq > 0.0)) {
        sc->stop = 1;
        sc->alpha = 0.0;
    } else {
        sc->alpha = sc->rz / pq;
    }
}

}  // namespace ngf
