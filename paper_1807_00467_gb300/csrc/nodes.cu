// Node passes of the gradient and the GN product: the launches of the bodies
// in nodes_body.cuh (curvature L v with its energy partials; the node-box
// gather with the curvature adjoint and the PCG's d . q partials).
#include "nodes_body.cuh"

namespace ngf {

namespace {

using nodek::NT;

__global__ void __launch_bounds__(NT) curv_kernel(const NodeArgs a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    __shared__ nodek::NodeSmem sm;
    nodek::curv_body<true>(a, cuda_block(), sm);
}

__global__ void __launch_bounds__(NT, 5) node_kernel(const NodeArgs a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    __shared__ nodek::NodeSmem sm;
    nodek::node_body<true>(a, cuda_block(), sm);
}

}  // namespace

int node_blocks(const int *m) {
    int gx, gy, gz;
    nodek::node_grid(m, gx, gy, gz);
    return gx * gy * gz;
}

cudaError_t launch_curv(const NodeArgs &a, cudaStream_t st) {
    int gx, gy, gz;
    nodek::node_grid(a.m, gx, gy, gz);
    curv_kernel<<<dim3(gx, gy, gz), NT, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nodes(const NodeArgs &a, cudaStream_t st) {
    int gx, gy, gz;
    nodek::node_grid(a.m, gx, gy, gz);
    node_kernel<<<dim3(gx, gy, gz), NT, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ngf
