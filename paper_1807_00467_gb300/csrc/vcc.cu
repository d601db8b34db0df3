// Volume change control, Eqs. (7)-(9): the launches of the per-cell body of
// vcc_body.cuh (gradient and energy, Gauss-Newton product, its diagonal).
#include "vcc_body.cuh"

namespace ngf {

namespace {

using vcck::NC;

template <int VM>
__global__ void __launch_bounds__(NC, VM == 0 ? 5 : 4) vcc_cell_kernel(const VccArgs a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    __shared__ vcck::VccSmem sm;
    vcck::vcc_cell_body<VM>(a, cuda_block(), sm);
}

}  // namespace

cudaError_t launch_vcc_cells(const VccArgs &a, cudaStream_t st) {
    dim3 grid(a.nb[0], a.nb[1], a.nb[2]);
    if (a.diag) vcc_cell_kernel<2><<<grid, NC, 0, st>>>(a);
    else if (a.v) vcc_cell_kernel<1><<<grid, NC, 0, st>>>(a);
    else vcc_cell_kernel<0><<<grid, NC, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ngf
