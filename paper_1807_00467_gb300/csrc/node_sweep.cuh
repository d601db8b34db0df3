// P^T of the trilinear prolongation onto a tile's node box, shared by the
// tile kernels: column sums parked per node plane are reduced along x, then
// along y, with the hat weights of the grid ratio.
#pragma once

namespace ngf {

// P^T along one axis by a sweep over a row of n = C R source values
// (stride `ss`): node c receives (1 - f_i) v from its own cell and f_i v from
// the cell below, f_i = (i + 1/2) / R the trilinear weights of the ratio R
// (squared weights for the Jacobi diagonal, SQ); writes the C + 1 node values
// (stride `ds`) times `scale`.
template <int R, int C, bool SQ>
__device__ __forceinline__ void hat_sweep(const float *src, int ss, float *dst, int ds, float scale) {
    float below = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float own = 0.f, up = 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const float v = src[(c * R + i) * ss];
            own = fmaf(SQ ? (1.f - (i + 0.5f) / R) * (1.f - (i + 0.5f) / R) : 1.f - (i + 0.5f) / R, v, own);
            up = fmaf(SQ ? ((i + 0.5f) / R) * ((i + 0.5f) / R) : (i + 0.5f) / R, v, up);
        }
        dst[c * ds] = scale * (below + own);
        below = up;
    }
    dst[C * ds] = scale * below;
}

// x then y reduction of the parked column sums rows[plane][ty][tx][comp] of a
// TY-row tile onto its node box [comp][plane][jy][jx] (times `scale`), through
// xr[plane][ty][jx][comp]; NT threads take part.
template <int TY, int NT, int RX, int RY, bool SQ>
__device__ __forceinline__ void node_reduce(const float *rows, float *xr, float *box, int boxsz, int nplanes,
                                            float scale, int tid) {
    constexpr int TXI = 28 - 28 % RX, CX = TXI / RX, CY = TY / RY;
    for (int r = tid; r < nplanes * TY * 3; r += NT) {
        const int k = r % 3, pr = r / 3;   // pr = plane * TY + ty
        hat_sweep<RX, CX, SQ>(rows + pr * TXI * 3 + k, 3, xr + pr * (CX + 1) * 3 + k, 3, 1.f);
    }
    __syncthreads();
    for (int r = tid; r < nplanes * (CX + 1) * 3; r += NT) {
        const int k = r % 3, q = r / 3, jx = q % (CX + 1), pl = q / (CX + 1);
        hat_sweep<RY, CY, SQ>(xr + (pl * TY * (CX + 1) + jx) * 3 + k, (CX + 1) * 3,
                              box + (long)k * boxsz + pl * (CY + 1) * (CX + 1) + jx, CX + 1, scale);
    }
}

// the same with the ratios chosen at run time (rx in {2, 4, 8}, ry in {1, 2, 4, 8})
template <int TY, int NT, bool SQ>
__device__ __forceinline__ void node_reduce_any(int rx, int ry, const float *rows, float *xr, float *box, int boxsz,
                                                int nplanes, float scale, int tid) {
#define NGF_NR(RX, RY) node_reduce<TY, NT, RX, RY, SQ>(rows, xr, box, boxsz, nplanes, scale, tid)
    switch (rx * 16 + ry) {
        case 2 * 16 + 1: NGF_NR(2, 1); break;
        case 2 * 16 + 2: NGF_NR(2, 2); break;
        case 2 * 16 + 4: NGF_NR(2, 4); break;
        case 2 * 16 + 8: NGF_NR(2, 8); break;
        case 4 * 16 + 1: NGF_NR(4, 1); break;
        case 4 * 16 + 2: NGF_NR(4, 2); break;
        case 4 * 16 + 4: NGF_NR(4, 4); break;
        case 4 * 16 + 8: NGF_NR(4, 8); break;
        case 8 * 16 + 1: NGF_NR(8, 1); break;
        case 8 * 16 + 2: NGF_NR(8, 2); break;
        case 8 * 16 + 4: NGF_NR(8, 4); break;
        default: NGF_NR(8, 8); break;
    }
#undef NGF_NR
}

}  // namespace ngf
