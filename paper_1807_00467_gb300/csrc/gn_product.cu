// Column-marching Gauss-Newton product of the NGF term and its Jacobi
// diagonal: the launches of the body in gn_product_body.cuh (the design is
// described there).
#include "gn_product_body.cuh"

namespace ngf {

namespace {

using namespace gnpk;

template <int RZ, bool DG, bool CHAIN, int RXY>
__global__ void __launch_bounds__(kNT, 1) gn_product_kernel(const __grid_constant__ ColArgs a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    uint32_t pbits = 0;
    gn_product_body<RZ, DG, CHAIN, RXY>(a, smem, bars, blockIdx.x, gridDim.x, true, pbits);
}

}  // namespace

bool gn_product_supported(const ColGeom &g) {
    if (!g.tma || g.rho[0] < 2 || g.m[2] > 256 || g.nxt * g.nyt > kNT) return false;
    return (size_t)pc_smem(g).total * sizeof(float) <= 227u * 1024u;
}

cudaError_t launch_gn_product(const ColArgs &a0, bool diag, cudaStream_t st) {
    if (!gn_product_supported(a0.g)) return cudaErrorInvalidValue;
    ColArgs a = a0;
    const size_t smem = sizeof(float) * (size_t)pc_smem(a.g).total;
    const int ncols = a.g.nb[0] * a.g.nb[1];
    // persistent CTAs (one per SM, columns strided by the grid) when a column's
    // plane sequence is a whole number of ring cycles, else one column per CTA
    const bool chain = (a.g.n[2] + 4) % kStages == 0;
    a.chain = chain;
    const int sms = device_sm_count();
    const int grid = chain ? (ncols < sms ? ncols : sms) : ncols;
    auto run = [&](auto kernel) {
        cudaError_t e = allow_max_dynamic_smem(kernel);
        if (e != cudaSuccess) return e;
        kernel<<<grid, kNT, smem, st>>>(a);
        return cudaGetLastError();
    };
    const bool r44 = a.g.rho[0] == 4 && a.g.rho[1] == 4;
#define NGF_PC(RZ, DG)                                                                                      \
    (chain ? (r44 ? run(gn_product_kernel<RZ, DG, true, 4>) : run(gn_product_kernel<RZ, DG, true, 0>)) \
           : run(gn_product_kernel<RZ, DG, false, 0>))
    switch (a.g.rho[2] * 2 + (diag ? 1 : 0)) {
        case 2: return NGF_PC(1, false);
        case 3: return NGF_PC(1, true);
        case 4: return NGF_PC(2, false);
        case 5: return NGF_PC(2, true);
        case 8: return NGF_PC(4, false);
        case 9: return NGF_PC(4, true);
        case 17: return NGF_PC(0, true);   // rho_z = 8: phases from the plane index
        default: return NGF_PC(0, false);
    }
#undef NGF_PC
}

}  // namespace ngf
