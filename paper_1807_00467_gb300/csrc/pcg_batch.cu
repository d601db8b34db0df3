// Persistent batched PCG: the reorthogonalised PCG steps of the Gauss-Newton
// systems of several volumes (image pairs, pyramid levels of uneven sizes) in
// one cooperative launch (the Gauss-Newton solve of Sec. II-D3 on the
// objective of Eq. (11)).
//
// One CTA per SM (640 threads, the GN-product kernel's shape) runs every PCG
// step k of every volume as five grid-wide phases:
//   A  H d pieces: the NGF GN product of every column (gn_product_body), the
//      VCC product of every cell block (vcc_cell_body, five 128-thread blocks
//      per item) and the curvature L d of every node tile (curv_body, two
//      256-thread blocks per item);
//   B  node pass: q = H d and the partials of d . q (node_body);
//   C  step:   alpha, r' = r - alpha q, Gram-Schmidt coefficient partials;
//   D  reorth: r_{k+1} = r' - sum_j c_j r_j and the partials of r . z;
//   E  dir:    beta, s += alpha d, d = z + beta d    (pcg_body.cuh).
// Within a phase the CTAs take (volume, unit) items from an atomic work
// counter, largest units first; the phases are separated by grid barriers.
// Every item runs the same code with the same partition and reduction order
// as the per-volume kernels, so each volume's iterates equal those of its
// own launches bit for bit.  Each volume keeps its own FP64 device scalars.
//
// Grid barrier: one arrival per CTA (release), then thread 0 polls the count
// (acquire) with a bounded number of polls; a CTA whose wait runs out raises
// the launch's abort flag and every volume's error flag (the caller reports
// RG_ETIMEOUT), and every CTA leaves at its next barrier.  The launch is
// cooperative, so all CTAs are resident and a barrier only runs out when a
// test hook withholds an arrival.
#include "gn_product_body.cuh"
#include "nodes_body.cuh"
#include "pcg_body.cuh"
#include "vcc_body.cuh"

#include <algorithm>
#include <mutex>

namespace ngf {

namespace {

using gnpk::kNT;
constexpr int kVccPer = kNT / vcck::NC;        // VCC cell blocks per item (5 x 128 threads)
constexpr int kNodePer = kNT / nodek::NT;      // node tiles per item (2 x 256 threads, 128 idle)
static_assert(pcgk::kVT <= kNT, "a PCG vector block fits in a CTA");

struct KPair {
    BatchPair b;
    pcgk::Part part;       // vector partition (pcg_body.cuh)
    int nvec;              // vector blocks
    int ncols, nvcc, nnode;
    int rz, rxy;           // GN-product specialisation: rho_z ring phases (0: generic), rho 4 x 4
};

struct KArgs {
    KPair p[kBatchMax];
    int npairs, iters;
    // first item of each volume in phase A (columns, then VCC groups, then
    // curvature groups), phase B and the vector phases; [npairs] = totals
    int colOff[kBatchMax + 1], vccOff[kBatchMax + 1], curvOff[kBatchMax + 1];
    int nodeOff[kBatchMax + 1], vecOff[kBatchMax + 1];
    unsigned *ctl;
    int poll_limit;
    int hook_skip;
};
static_assert(sizeof(KArgs) <= 32000, "the descriptors travel as kernel parameters");

__device__ __forceinline__ int find_pair(const int *off, int n, int item) {
    int p = 0;
    while (p + 1 < n && off[p + 1] <= item) ++p;
    return p;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `nbar` (1, 2, ...).  False: the launch was aborted.
__device__ __forceinline__ bool grid_barrier(const KArgs &A, unsigned nbar, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = nbar * gridDim.x;
        __threadfence();
        if (!(A.hook_skip && nbar == 1 && blockIdx.x == 0)) atomicAdd(&A.ctl[0], 1u);
        int ok = 1;
        for (int it = 0; ld_acquire(&A.ctl[0]) < target; ++it) {
            if (*(volatile unsigned *)&A.ctl[1]) {
                ok = 0;
                break;
            }
            if (it > A.poll_limit) {
                atomicExch(&A.ctl[1], 1u);
                for (int q = 0; q < A.npairs; ++q) atomicExch(A.p[q].b.col.err, 1);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The next item of a phase's work counter (the same value in every thread).
__device__ __forceinline__ int next_item(unsigned *ctr, int *s_item) {
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    return it;
}

__device__ __forceinline__ void gn_column(const KPair &P, float *smem, uint64_t *bars, int t, uint32_t &pbits) {
    const ColArgs &a = P.b.col;
    if (P.rxy == 4) {
        switch (P.rz) {
            case 2: gnpk::gn_product_body<2, false, false, 4, true>(a, smem, bars, t, 1, false, pbits); return;
            case 4: gnpk::gn_product_body<4, false, false, 4, true>(a, smem, bars, t, 1, false, pbits); return;
            default: gnpk::gn_product_body<0, false, false, 4, true>(a, smem, bars, t, 1, false, pbits); return;
        }
    }
    gnpk::gn_product_body<0, false, false, 0, true>(a, smem, bars, t, 1, false, pbits);
}

__global__ void __launch_bounds__(kNT, 1) pcg_batch_kernel(const __grid_constant__ KArgs A) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[gnpk::kStages];
    __shared__ int s_item, s_ok;
    const int tid = threadIdx.x;
    if (tid == kNT - 32) {
        for (int i = 0; i < gnpk::kStages; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t pbits = 0;
    unsigned nbar = 0;
    const int np = A.npairs;
    const int nA = A.curvOff[np], nB = A.nodeOff[np], nV = A.vecOff[np];
    for (int k = 0; k < A.iters; ++k) {
        unsigned *ctr = A.ctl + 2 + 5 * k;
        // ---------------------------------------------------------------- A: H d pieces
        for (int it; (it = next_item(ctr, &s_item)) < nA;) {
            if (it < A.colOff[np]) {
                const int p = find_pair(A.colOff, np, it);
                gn_column(A.p[p], smem, bars, it - A.colOff[p], pbits);
            } else if (it < A.vccOff[np]) {
                const int p = find_pair(A.vccOff, np, it);
                const KPair &P = A.p[p];
                const int v = tid / vcck::NC, bid = (it - A.vccOff[p]) * kVccPer + v;
                if (bid < P.nvcc) {
                    VBlock b{tid % vcck::NC, bid, P.nvcc, 1 + v, vcck::NC};
                    vcck::vcc_cell_body<1>(P.b.vcc, b, reinterpret_cast<vcck::VccSmem *>(smem)[v]);
                }
            } else {
                const int p = find_pair(A.curvOff, np, it);
                const KPair &P = A.p[p];
                const int v = tid / nodek::NT, bid = (it - A.curvOff[p]) * kNodePer + v;
                if (v < kNodePer && bid < P.nnode) {
                    VBlock b{tid % nodek::NT, bid, P.nnode, 1 + v, nodek::NT};
                    nodek::curv_body<false>(P.b.nodes, b, reinterpret_cast<nodek::NodeSmem *>(smem)[v]);
                }
            }
        }
        if (!grid_barrier(A, ++nbar, &s_ok)) return;
        // ---------------------------------------------------------------- B: node pass, d . q partials
        for (int it; (it = next_item(ctr + 1, &s_item)) < nB;) {
            const int p = find_pair(A.nodeOff, np, it);
            const KPair &P = A.p[p];
            const int v = tid / nodek::NT, bid = (it - A.nodeOff[p]) * kNodePer + v;
            if (v < kNodePer && bid < P.nnode) {
                VBlock b{tid % nodek::NT, bid, P.nnode, 1 + v, nodek::NT};
                nodek::node_body<false>(P.b.nodes, b, reinterpret_cast<nodek::NodeSmem *>(smem)[v]);
            }
        }
        if (!grid_barrier(A, ++nbar, &s_ok)) return;
        // ---------------------------------------------------------------- C, D, E: the vector phases
        for (int ph = 0; ph < 3; ++ph) {
            for (int it; (it = next_item(ctr + 2 + ph, &s_item)) < nV;) {
                const int p = find_pair(A.vecOff, np, it);
                const KPair &P = A.p[p];
                if (tid >= pcgk::kVT) continue;
                const VBlock b{tid, it - A.vecOff[p], P.nvec, 1, pcgk::kVT};
                const PcgArgs &g = P.b.pcg;
                pcgk::PcgSmem &sm = *reinterpret_cast<pcgk::PcgSmem *>(smem);
                if (ph == 0)
                    pcgk::pcg_step_body(P.part, g.sc, g.apart, P.nnode, P.b.nodes.out, g.minv, g.Rh, g.stride, k,
                                        g.part, b, sm);
                else if (ph == 1)
                    pcgk::pcg_reorth_body(P.part, g.sc, g.minv, g.Rh, g.stride, k, g.rzh, g.part, g.rzpart, b, sm);
                else
                    pcgk::pcg_dir_body(P.part, g.sc, g.minv, g.Rh + (long)(k + 1) * g.stride, g.d, P.b.s, k, g.rzh,
                                       g.rzpart, b, sm);
            }
            if ((k + 1 < A.iters || ph < 2) && !grid_barrier(A, ++nbar, &s_ok)) return;
        }
    }
}

size_t batch_smem(const KArgs &A) {
    size_t s = std::max(sizeof(pcgk::PcgSmem),
                        std::max(kVccPer * sizeof(vcck::VccSmem), kNodePer * sizeof(nodek::NodeSmem)));
    for (int p = 0; p < A.npairs; ++p) s = std::max(s, sizeof(float) * (size_t)gnpk::pc_smem(A.p[p].b.col.g).total);
    return s;
}

}  // namespace

bool pcg_batch_supported(const ColGeom &g) { return gn_product_supported(g); }

cudaError_t launch_pcg_batch(const BatchPair *pairs, int npairs, int iters, unsigned *ctl, int poll_limit,
                             int hook_skip, cudaStream_t st) {
    if (npairs < 1 || npairs > kBatchMax || iters < 1 || iters > RG_PCG_MAX || !ctl) return cudaErrorInvalidValue;
    static KArgs A;   // large: built in static storage (callers serialise on the host)
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    A.npairs = npairs;
    A.iters = iters;
    A.ctl = ctl;
    A.poll_limit = poll_limit;
    A.hook_skip = hook_skip;
    // deeper volumes first: their columns are the longest items of phase A
    int order[kBatchMax];
    for (int p = 0; p < npairs; ++p) order[p] = p;
    std::stable_sort(order, order + npairs,
                     [&](int x, int y) { return pairs[x].col.g.n[2] > pairs[y].col.g.n[2]; });
    for (int p = 0; p < npairs; ++p) {
        KPair &P = A.p[p];
        P.b = pairs[order[p]];
        const ColGeom &g = P.b.col.g;
        if (!pcg_batch_supported(g) || !P.b.s || P.b.pcg.n != 3L * g.m[0] * g.m[1] * g.m[2])
            return cudaErrorInvalidValue;
        P.part = pcgk::make_part(P.b.pcg.n, &P.nvec);
        P.ncols = g.nb[0] * g.nb[1];
        P.nvcc = P.b.vcc_on ? P.b.vcc.nb[0] * P.b.vcc.nb[1] * P.b.vcc.nb[2] : 0;
        P.nnode = node_blocks(g.m);
        P.rz = (g.rho[2] == 2 || g.rho[2] == 4) ? g.rho[2] : 0;
        P.rxy = (g.rho[0] == 4 && g.rho[1] == 4) ? 4 : 0;
    }
    // item offsets: phase A holds every column, then every VCC group, then
    // every curvature group
    int n = 0;
    for (int p = 0; p < npairs; ++p) { A.colOff[p] = n; n += A.p[p].ncols; }
    A.colOff[npairs] = n;
    for (int p = 0; p < npairs; ++p) { A.vccOff[p] = n; n += (A.p[p].nvcc + kVccPer - 1) / kVccPer; }
    A.vccOff[npairs] = n;
    for (int p = 0; p < npairs; ++p) { A.curvOff[p] = n; n += (A.p[p].nnode + kNodePer - 1) / kNodePer; }
    A.curvOff[npairs] = n;
    n = 0;
    for (int p = 0; p < npairs; ++p) { A.nodeOff[p] = n; n += (A.p[p].nnode + kNodePer - 1) / kNodePer; }
    A.nodeOff[npairs] = n;
    n = 0;
    for (int p = 0; p < npairs; ++p) { A.vecOff[p] = n; n += A.p[p].nvec; }
    A.vecOff[npairs] = n;

    const size_t smem = batch_smem(A);
    cudaError_t e = allow_max_dynamic_smem(pcg_batch_kernel);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_batch_kernel, kNT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(device_sm_count());
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, pcg_batch_kernel, A);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace ngf
