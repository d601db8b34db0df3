// Node-grid kernels: curvature (Eq. (5)), volume change control (Eqs. (7)-(9)),
// keypoint penalty (Eq. (10)), the node-box finaliser, objective terms,
// PCG vector operations with FP64 reductions, and pyramid transfers.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace ngf {

// ------------------------------------------------------------------ reductions
// Block sum of one double per thread; thread 0 receives the total.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (blockDim.x + 31) / 32; ++i) t += red[i];
    return t;
}

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ------------------------------------------------------------------ VCC
// gradient, GN product and GN diagonal: one thread per cell (vcc.cu)
cudaError_t launch_vcc(const VccArgs &a, cudaStream_t st) { return launch_vcc_cells(a, st); }

// ------------------------------------------------------------------ keypoints
// A keypoint's trilinear weights are fixed by its position x_i: cell c_i =
// floor(x_i / g) clamped to the grid, fractions f_i = x_i / g - c_i.  The
// index built once per set of keypoints sorts them by (cell, i); the node
// sums 2 P^T src (gradient: src_i = x_i + (P u)(x_i) - y_i; GN product: src_i =
// (P v)(x_i); diagonal: 2 delta w^2) are then gathered without atomics: node
// n receives from the cells n - o of its corner offsets o = 0..7 in the order
// (o, i), summed by one thread (the one of the smallest o whose cell holds
// keypoints), so repeated calls give the same bits.
int kp_blocks(int nk) { return nk <= 0 ? 1 : (nk + 255) / 256; }

// corner o = ox + 2 oy + 4 oz of a cell: trilinear weight from the fractions
__device__ __forceinline__ float kp_weight(int o, const float *f) {
    return ((o & 1) ? f[0] : 1.f - f[0]) * ((o & 2) ? f[1] : 1.f - f[1]) * ((o & 4) ? f[2] : 1.f - f[2]);
}

// index, step 1: cell and fractions of every keypoint
__global__ void kp_cells_kernel(const KpArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nk) return;
    const int mm[3] = {a.m[0], a.m[1], a.m[2]};
    int c[3];
    for (int ax = 0; ax < 3; ++ax) {
        const float t = a.kx[3 * i + ax] * a.ig[ax];
        const int ci = max(0, min((int)floorf(t), mm[ax] - 2));
        c[ax] = ci;
        a.ix.frac[3 * i + ax] = t - ci;
    }
    a.ix.cell[i] = (c[2] * mm[1] + c[1]) * mm[0] + c[0];
}

// index, step 2: the rank of (cell_i, i) among all keypoints (a permutation:
// the pairs are distinct), keypoints in 256-wide shared-memory tiles
__global__ void __launch_bounds__(256) kp_rank_kernel(const KpArgs a) {
    __shared__ int tile[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ci = i < a.nk ? a.ix.cell[i] : 0;
    int rank = 0;
    for (int j0 = 0; j0 < a.nk; j0 += 256) {
        __syncthreads();
        if (j0 + (int)threadIdx.x < a.nk) tile[threadIdx.x] = a.ix.cell[j0 + threadIdx.x];
        __syncthreads();
        const int nj = min(256, a.nk - j0);
        for (int t = 0; t < nj; ++t) {
            const int cj = tile[t];
            rank += (cj < ci || (cj == ci && j0 + t < i)) ? 1 : 0;
        }
    }
    if (i < a.nk) {
        a.ix.perm[rank] = i;
        a.ix.sb[rank] = ci;
    }
}

// index, step 3: the first sorted position of every cell that holds keypoints
// (soc is -1 everywhere before)
__global__ void kp_heads_kernel(const KpArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.nk) return;
    if (r == 0 || a.ix.sb[r] != a.ix.sb[r - 1]) a.ix.soc[a.ix.sb[r]] = r;
}

cudaError_t launch_kp_index(const KpArgs &a, int step, cudaStream_t st) {
    if (a.nk <= 0) return cudaSuccess;
    const int nb = kp_blocks(a.nk);
    if (step == 0) {
        const long M = (long)a.m[0] * a.m[1] * a.m[2];
        const cudaError_t e = cudaMemsetAsync(a.ix.soc, 0xff, sizeof(int) * M, st);
        if (e != cudaSuccess) return e;
        kp_cells_kernel<<<nb, 256, 0, st>>>(a);
    } else if (step == 1) {
        kp_rank_kernel<<<nb, 256, 0, st>>>(a);
    } else {
        kp_heads_kernel<<<nb, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// per keypoint: residual (energy) and the source of its node contributions
__global__ void kp_kernel(const KpArgs a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int mx = a.m[0], my = a.m[1], mz = a.m[2];
    const long mxy = (long)mx * my, M = mxy * mz;
    float e = 0.f;
    if (i < a.nk) {
        const float f[3] = {a.ix.frac[3 * i], a.ix.frac[3 * i + 1], a.ix.frac[3 * i + 2]};
        const long base = a.ix.cell[i];
        float w[8];
        long nd[8];
        for (int o = 0; o < 8; ++o) {
            w[o] = kp_weight(o, f);
            nd[o] = base + (o & 1) + ((o >> 1) & 1) * mx + (o >> 2) * mxy;
        }
        for (int k = 0; k < 3; ++k) {
            float pu = 0.f, pv = 0.f;
            for (int o = 0; o < 8; ++o) {
                pu = fmaf(w[o], a.u[k * M + nd[o]], pu);
                if (a.v) pv = fmaf(w[o], a.v[k * M + nd[o]], pv);
            }
            const float res = a.kx[3 * i + k] + pu - a.ky[3 * i + k];
            e = fmaf(res, res, e);
            if (a.out) a.ix.src[3 * i + k] = a.v ? pv : res;
        }
    }
    if (a.part) {
        double t = block_sum((double)e);
        if (threadIdx.x == 0) a.part[blockIdx.x] = t;
    }
}

// node sums: thread (r, o) for the first sorted keypoint r of a cell and a
// corner o of that cell owns node n = cell + o unless a cell n - o' with o' < o
// holds keypoints; the owner adds, in the order (o'', i), the contributions
// of every keypoint in the cells n - o'' to out[n] (diag: 2 delta w^2 to all
// three components; else 2 scale w src_i)
template <bool DIAG>
__global__ void kp_gather_kernel(const KpArgs a, double two_delta, float *out) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = t >> 3, o = t & 7;
    if (r >= a.nk) return;
    const int *sb = a.ix.sb;
    if (r > 0 && sb[r] == sb[r - 1]) return;
    const int mx = a.m[0], my = a.m[1];
    const long mxy = (long)mx * my, M = mxy * a.m[2];
    const int b = sb[r];
    const int cz = b / (int)mxy, cy = (b - cz * (int)mxy) / mx, cx = b - cz * (int)mxy - cy * mx;
    const int nx = cx + (o & 1), ny = cy + ((o >> 1) & 1), nz = cz + (o >> 2);
    // the cell n - o' of corner offset o', or -1 outside the cell grid
    auto cell_at = [&](int op) {
        const int x = nx - (op & 1), y = ny - ((op >> 1) & 1), z = nz - (op >> 2);
        if (x < 0 || y < 0 || z < 0 || x > mx - 2 || y > my - 2 || z > a.m[2] - 2) return -1;
        return (z * my + y) * mx + x;
    };
    for (int op = 0; op < o; ++op) {
        const int c = cell_at(op);
        if (c >= 0 && a.ix.soc[c] >= 0) return;
    }
    float acc[3] = {0.f, 0.f, 0.f};
    for (int op = 0; op < 8; ++op) {
        const int c = cell_at(op);
        const int s = c >= 0 ? a.ix.soc[c] : -1;
        if (s < 0) continue;
        for (int q = s; q < a.nk && sb[q] == c; ++q) {
            const int i = a.ix.perm[q];
            const float f[3] = {a.ix.frac[3 * i], a.ix.frac[3 * i + 1], a.ix.frac[3 * i + 2]};
            const float w = kp_weight(op, f);
            if (DIAG) {
                const float add = (float)(two_delta * w * w);
                acc[0] += add; acc[1] += add; acc[2] += add;
            } else {
                for (int k = 0; k < 3; ++k) acc[k] += 2.f * a.scale * w * a.ix.src[3 * i + k];
            }
        }
    }
    const long n = (long)nz * mxy + (long)ny * mx + nx;
    for (int k = 0; k < 3; ++k) out[k * M + n] += acc[k];
}

cudaError_t launch_kp(const KpArgs &a, cudaStream_t st) {
    kp_kernel<<<kp_blocks(a.nk), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_kp_gather(const KpArgs &a, cudaStream_t st) {
    if (!a.out || a.nk <= 0) return cudaSuccess;
    kp_gather_kernel<false><<<(8 * a.nk + 255) / 256, 256, 0, st>>>(a, 0.0, a.out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ terms
__device__ double sum_parts(const double *p, int n) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    return block_sum(s);
}

__global__ void terms_kernel(const TermsArgs a) {
    if (a.skip && *a.skip) return;   // uniform: every block reads the same flag
    double D = a.dpart ? sum_parts(a.dpart, a.nd) * a.dscale : 0.0;
    __syncthreads();
    double R = a.rpart ? sum_parts(a.rpart, a.nr) * a.rscale : 0.0;
    __syncthreads();
    double V = a.vpart ? sum_parts(a.vpart, a.nv) * a.vscale : 0.0;
    __syncthreads();
    double K = a.kpart ? sum_parts(a.kpart, a.nkp) : 0.0;
    __syncthreads();
    __shared__ int sfold;
    __shared__ float smn, smx;
    if (threadIdx.x == 0) { sfold = 0; smn = 3.4e38f; smx = -3.4e38f; }
    __syncthreads();
    if (a.vpart) {
        int f = 0;
        float mn = 3.4e38f, mx = -3.4e38f;
        for (int i = threadIdx.x; i < a.nv; i += blockDim.x) {
            f += a.fold[i];
            mn = fminf(mn, a.dmin[i]);
            mx = fmaxf(mx, a.dmax[i]);
        }
        if (f) atomicAdd(&sfold, f);
        // min/max via shared atomics on the float bit patterns is avoided: serialise per warp
        for (int off = 16; off > 0; off >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        }
        __shared__ float wmn[32], wmx[32];
        if ((threadIdx.x & 31) == 0) { wmn[threadIdx.x >> 5] = mn; wmx[threadIdx.x >> 5] = mx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { smn = fminf(smn, wmn[i]); smx = fmaxf(smx, wmx[i]); }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double J = D + a.alpha * R + a.gamma * V + a.delta * K;
        if (sfold) { J = INFINITY; V = INFINITY; }
        else if (a.nonfinite && !isfinite(J)) atomicExch(a.nonfinite, 1);
        a.terms[0] = D; a.terms[1] = R; a.terms[2] = V; a.terms[3] = K; a.terms[4] = J;
        if (a.dminmax) { a.dminmax[0] = a.vpart ? smn : 1.0; a.dminmax[1] = a.vpart ? smx : 1.0; }
    }
}

cudaError_t launch_terms(const TermsArgs &a, cudaStream_t st) {
    terms_kernel<<<1, 512, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ PCG vectors
int vec_blocks(long n) {
    long b = (n + 256 * 8 - 1) / (256 * 8);
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

#define GRID_STRIDE(i, n) for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

// diag += alpha ghat diag(L^T L) + tau (the curvature part of the
// preconditioner; L^T L column k: own row and the rows of its neighbours)
__global__ void jacobi_diag_kernel(int alpha_on, int mx, int my, int mz, float ig2x, float ig2y, float ig2z,
                                   double alpha_ghat, double tau, float *diag) {
    const long mxy = (long)mx * my, M = mxy * mz;
    GRID_STRIDE(k, M) {
        const int kz = (int)(k / mxy), rem = (int)(k - kz * mxy), ky = rem / mx, kx = rem - ky * mx;
        const int kk[3] = {kx, ky, kz}, mm[3] = {mx, my, mz};
        const double ig2[3] = {ig2x, ig2y, ig2z};
        double own = 0.0, nb = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            if (kk[ax] >= 1 && kk[ax] <= mm[ax] - 2) own -= 2.0 * ig2[ax];
            if (kk[ax] - 1 >= 1) nb += ig2[ax] * ig2[ax];
            if (kk[ax] + 1 <= mm[ax] - 2) nb += ig2[ax] * ig2[ax];
        }
        const float d = (float)((alpha_on ? alpha_ghat * (own * own + nb) : 0.0) + tau);
        diag[k] += d; diag[M + k] += d; diag[2 * M + k] += d;
    }
}

cudaError_t launch_jacobi_diag(int alpha_on, const int *m, const float *ig2, double alpha_ghat, double tau,
                               float *diag, cudaStream_t st) {
    long M = (long)m[0] * m[1] * m[2];
    jacobi_diag_kernel<<<vec_blocks(M), 256, 0, st>>>(alpha_on, m[0], m[1], m[2], ig2[0], ig2[1], ig2[2], alpha_ghat,
                                                     tau, diag);
    return cudaGetLastError();
}

cudaError_t launch_kp_diag(const KpArgs &a, double two_delta, float *diag, cudaStream_t st) {
    if (a.nk <= 0) return cudaSuccess;
    kp_gather_kernel<true><<<(8 * a.nk + 255) / 256, 256, 0, st>>>(a, two_delta, diag);
    return cudaGetLastError();
}

// reciprocal of the preconditioner diagonal; entries that are not positive
// (rows without any term) use 1
__global__ void invert_kernel(long n, float *d) {
    GRID_STRIDE(i, n) d[i] = d[i] > 0.f ? 1.f / d[i] : 1.f;
}

cudaError_t launch_invert(long n, float *d, cudaStream_t st) {
    invert_kernel<<<vec_blocks(n), 256, 0, st>>>(n, d);
    return cudaGetLastError();
}

__global__ void dot_kernel(long n, const float *x, const float *y, double *part) {
    Kahan acc;
    GRID_STRIDE(i, n) acc.add(x[i] * y[i]);
    double t = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

cudaError_t launch_dot(long n, const float *x, const float *y, double *part, cudaStream_t st) {
    dot_kernel<<<vec_blocks(n), 256, 0, st>>>(n, x, y, part);
    return cudaGetLastError();
}

// which: 0 rz = sum (start); 1 pq = sum -> alpha; 2 rz_new = sum -> beta;
//        3 r0 = sqrt(sum); 4 rend = sqrt(sum); 5 reset (no sum)
__global__ void pcg_scalar_kernel(int which, const double *part, int nparts, PcgScalars *sc, double *rzh) {
    double v = 0.0;
    if (which != 5) v = sum_parts(part, nparts);
    if (threadIdx.x != 0) return;
    switch (which) {
        case 0:
            sc->rz = v;
            if (rzh) rzh[0] = v;
            break;
        case 1:
            sc->pq = v;
            if (sc->stop || !(sc->rz != 0.0) || !(v > 0.0)) { sc->stop = 1; sc->alpha = 0.0; }
            else sc->alpha = sc->rz / v;
            break;
        case 2:
            sc->rz_new = v;
            if (sc->stop) { sc->beta = 0.0; }
            else {
                sc->beta = v / sc->rz;
                sc->rz = v;
                sc->steps += 1;
                if (rzh) rzh[sc->steps] = v;
            }
            break;
        case 3: sc->r0 = sqrt(v); break;
        case 4: sc->rend = sqrt(v); break;
        case 5:
            sc->rz = sc->rz_new = sc->pq = sc->alpha = sc->beta = sc->r0 = sc->rend = 0.0;
            sc->stop = 0; sc->steps = 0;
            break;
    }
}

cudaError_t launch_pcg_scalar(int which, const double *part, int nparts, PcgScalars *sc, cudaStream_t st,
                              double *rzh) {
    pcg_scalar_kernel<<<1, 256, 0, st>>>(which, part, nparts, sc, rzh);
    return cudaGetLastError();
}

// |r_steps|^2 partials, the residual of the last completed step
__global__ void dot_slot_kernel(long n, const float *Rh, long stride, const PcgScalars *sc, double *part) {
    const float *r = Rh + (long)sc->steps * stride;
    Kahan acc;
    GRID_STRIDE(i, n) acc.add(r[i] * r[i]);
    double t = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

cudaError_t launch_dot_slot(long n, const float *Rh, long stride, const PcgScalars *sc, double *part,
                            cudaStream_t st) {
    dot_slot_kernel<<<vec_blocks(n), 256, 0, st>>>(n, Rh, stride, sc, part);
    return cudaGetLastError();
}

__global__ void axpy_copy_kernel(long n, float t, const float *x, const float *p, float *y, const int *skip) {
    if (skip && *skip) return;
    GRID_STRIDE(i, n) y[i] = fmaf(t, p[i], x[i]);
}

cudaError_t launch_axpy_copy(long n, float t, const float *x, const float *p, float *y, cudaStream_t st,
                             const int *skip) {
    axpy_copy_kernel<<<vec_blocks(n), 256, 0, st>>>(n, t, x, p, y, skip);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pyramid
template <typename TImg>
__global__ void restrict_kernel(int nx, int ny, int nz, const TImg *in, TImg *out) {
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const long N = (long)cx * cy * cz;
    GRID_STRIDE(i, N) {
        const int jz = (int)(i / ((long)cx * cy)), rem = (int)(i - (long)jz * cx * cy), jy = rem / cx, jx = rem - jy * cx;
        float s = 0.f;
        for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            s += ldimg(in, ((long)(2 * jz + oz) * ny + (2 * jy + oy)) * nx + 2 * jx + ox);
        }
        s *= 0.125f;
        if constexpr (sizeof(TImg) == 2) out[i] = __float2half_rn(s);
        else out[i] = s;
    }
}

cudaError_t launch_restrict(const int *n, bool half, const void *in, void *out, cudaStream_t st) {
    long N = (long)(n[0] / 2) * (n[1] / 2) * (n[2] / 2);
    if (half)
        restrict_kernel<__half><<<vec_blocks(N), 256, 0, st>>>(n[0], n[1], n[2], (const __half *)in, (__half *)out);
    else
        restrict_kernel<float><<<vec_blocks(N), 256, 0, st>>>(n[0], n[1], n[2], (const float *)in, (float *)out);
    return cudaGetLastError();
}

__global__ void prolong_grid_kernel(int cx, int cy, int cz, const float *uc, float *uf) {
    const int fx = 2 * cx - 1, fy = 2 * cy - 1, fz = 2 * cz - 1;
    const long Mf = (long)fx * fy * fz, Mc = (long)cx * cy * cz;
    GRID_STRIDE(k, Mf) {
        const int kz = (int)(k / ((long)fx * fy)), rem = (int)(k - (long)kz * fx * fy), ky = rem / fx, kx = rem - ky * fx;
        const int lo[3] = {kx / 2, ky / 2, kz / 2}, hi[3] = {(kx + 1) / 2, (ky + 1) / 2, (kz + 1) / 2};
        for (int c = 0; c < 3; ++c) {
            float s = 0.f;
            for (int o = 0; o < 8; ++o) {
                const int x = (o & 1) ? hi[0] : lo[0], y = ((o >> 1) & 1) ? hi[1] : lo[1], z = (o >> 2) ? hi[2] : lo[2];
                s += uc[c * Mc + ((long)z * cy + y) * cx + x];
            }
            uf[c * Mf + k] = 0.125f * s;
        }
    }
}

cudaError_t launch_prolong_grid(const int *mc, const float *uc, float *uf, cudaStream_t st) {
    long Mf = (long)(2 * mc[0] - 1) * (2 * mc[1] - 1) * (2 * mc[2] - 1);
    prolong_grid_kernel<<<vec_blocks(Mf), 256, 0, st>>>(mc[0], mc[1], mc[2], uc, uf);
    return cudaGetLastError();
}

__global__ void inject_grid_kernel(int fx, int fy, int fz, int step, const float *uf, int cx, int cy, int cz, float *uc) {
    const long Mc = (long)cx * cy * cz, Mf = (long)fx * fy * fz;
    GRID_STRIDE(k, Mc) {
        const int kz = (int)(k / ((long)cx * cy)), rem = (int)(k - (long)kz * cx * cy), ky = rem / cx, kx = rem - ky * cx;
        for (int c = 0; c < 3; ++c)
            uc[c * Mc + k] = uf[c * Mf + ((long)(step * kz) * fy + step * ky) * fx + step * kx];
    }
}

cudaError_t launch_inject_grid(const int *mf, int step, const float *uf, const int *mc, float *uc, cudaStream_t st) {
    long Mc = (long)mc[0] * mc[1] * mc[2];
    inject_grid_kernel<<<vec_blocks(Mc), 256, 0, st>>>(mf[0], mf[1], mf[2], step, uf, mc[0], mc[1], mc[2], uc);
    return cudaGetLastError();
}

}  // namespace ngf
