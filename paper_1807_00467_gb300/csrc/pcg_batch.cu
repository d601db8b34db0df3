// Persistent batched PCG: the reorthogonalised PCG steps of the Gauss-Newton
// systems of several volumes (image pairs, pyramid levels of uneven sizes) in
// one cooperative launch (the Gauss-Newton solve of Sec. II-D3 on the
// objective of Eq. (11)).
//
// One CTA per SM (640 threads, the GN-product kernel's shape) runs every PCG
// step k of every volume as five phases:
//   A  H d pieces: the NGF GN product of every column (gn_product_body), the
//      VCC product of every cell block (vcc_cell_body, five 128-thread blocks
//      per item) and the curvature L d of every node tile (curv_body, two
//      256-thread blocks per item);
//   B  node pass: q = H d and the partials of d . q (node_body);
//   C  step:   alpha, r' = r - alpha q, Gram-Schmidt coefficient partials;
//   D  reorth: r_{k+1} = r' - sum_j c_j r_j and the partials of r . z;
//   E  dir:    beta, s += alpha d, d = z + beta d    (pcg_body.cuh).
// The CTAs take (volume, unit) items from one atomic work counter in the
// order (step, phase, volume, unit).  An item waits only for the previous
// phase of its own volume (per-volume completion counters), whose items all
// come earlier in that order and are held by running CTAs, so phases of
// different volumes overlap and nothing waits for a CTA that is not running.
// Every item runs the same code with the same partition and reduction order
// as the per-volume kernels, so each volume's iterates equal those of its
// own launches bit for bit.  Each volume keeps its own FP64 device scalars.
//
// Waits: thread 0 polls the counter with a growing pause, for a bounded
// number of polls and at most two seconds; a CTA whose wait runs out raises
// the launch's abort flag and every volume's error flag (the caller reports
// RG_ETIMEOUT), and the other CTAs leave at their next wait.  The launch is
// cooperative, so all CTAs are resident and a wait only runs out when a test
// hook withholds a completion.
#include "gn_product_body.cuh"
#include "nodes_body.cuh"
#include "pcg_body.cuh"
#include "vcc_body.cuh"

#include <algorithm>
#include <mutex>

namespace ngf {

namespace {

using gnpk::kNT;
constexpr int kVccRun = kNT / vcck::NC;        // VCC cell blocks at once (5 x 128 threads)
constexpr int kNodeRun = kNT / nodek::NT;      // node tiles at once (2 x 256 threads, 128 idle)
// units per work item: the light phases take several rounds per item, so the
// per-item cost (work counter, completion record) stays small
constexpr int kVccPer = 4 * kVccRun, kNodePer = 8 * kNodeRun, kVecPer = 2;
static_assert(pcgk::kVT <= kNT, "a PCG vector block fits in a CTA");

struct KPair {
    BatchPair b;
    pcgk::Part part;       // vector partition (pcg_body.cuh)
    int nvec;              // vector blocks
    int ncols, nvcc, nnode;
    int nA, nB, nV;        // items of phase A (columns, VCC groups, curvature groups), B and each vector phase
    int rz, rxy;           // GN-product specialisation: rho_z ring phases (0: generic), rho 4 x 4
};

struct KArgs {
    KPair p[kBatchMax];
    int npairs, iters;
    // first item of each volume in phase A (columns, then VCC groups, then
    // curvature groups), phase B and the vector phases; [npairs] = totals
    int colOff[kBatchMax + 1], vccOff[kBatchMax + 1], curvOff[kBatchMax + 1];
    int nodeOff[kBatchMax + 1], vecOff[kBatchMax + 1];
    unsigned *ctl;         // control words (kCtlAbort, done_ctr)
    int poll_limit;
    int hook_skip;
};
static_assert(sizeof(KArgs) <= 32000, "the descriptors travel as kernel parameters");

__device__ __forceinline__ int find_pair(const int *off, int n, int item) {
    int p = 0;
    while (p + 1 < n && off[p + 1] <= item) ++p;
    return p;
}

// Control words (kBatchCtlWords): the work counter and the abort flag on
// lines of their own, then one 128-byte line per volume holding its five
// completion counters, so that polls of one volume's counters do not contend
// with the atomics of the others.
constexpr int kCtlAbort = 32, kCtlDone = 64, kCtlLine = 32;
__device__ __forceinline__ unsigned *done_ctr(const KArgs &A, int p, int ph) {
    return A.ctl + kCtlDone + kCtlLine * p + ph;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait until pair p's phase ph has completed `need` items: thread 0 polls
// with relaxed loads and a growing pause (up to ~4 us) for at most
// poll_limit polls or two seconds, then one acquire fence; the CTA then
// proceeds.  False: the launch was aborted (this wait or another CTA's ran out).
__device__ __forceinline__ bool wait_done(const KArgs &A, int p, int ph, unsigned need, int *s_ok) {
    if (threadIdx.x == 0) {
        const volatile unsigned *ctr = done_ctr(A, p, ph);
        const volatile unsigned *abort_flag = A.ctl + kCtlAbort;
        int ok = 1;
        if (*ctr < need) {
            const unsigned long long t0 = global_ns();
            unsigned pause = 32;
            for (int it = 0; *ctr < need; ++it) {
                if (*abort_flag) {
                    ok = 0;
                    break;
                }
                if (it > A.poll_limit || global_ns() - t0 > 2000000000ull) {
                    atomicExch(A.ctl + kCtlAbort, 1u);
                    for (int q = 0; q < A.npairs; ++q) atomicExch(A.p[q].b.col.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(pause);
                if (pause < 4096) pause *= 2;
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Record one completed item of pair p's phase ph (after every thread's
// writes).  Test hook: the launch's first item is never recorded, so the
// waits of its pair's next phase run out.
__device__ __forceinline__ void item_done(const KArgs &A, int p, int ph, int it) {
    __syncthreads();
    if (threadIdx.x == 0 && !(A.hook_skip && it == 0)) {
        __threadfence();
        atomicAdd(done_ctr(A, p, ph), 1u);
    }
}

// The next item of a phase's work counter (the same value in every thread).
__device__ __forceinline__ int next_item(unsigned *ctr, int *s_item) {
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    return it;
}

// Node tile bid of a volume as block v (256 threads, named barrier 1 + v) of a CTA.
__device__ __forceinline__ VBlock node_block(const KPair &P, int tid, int bid, int v) {
    int gx, gy, gz;
    nodek::node_grid(P.b.nodes.m, gx, gy, gz);
    return warp_block(tid % nodek::NT, bid, gx, gy, gz, 1 + v, nodek::NT);
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
    const int np = A.npairs;
    const int nA = A.curvOff[np], nB = A.nodeOff[np], nV = A.vecOff[np];
    const int per_step = nA + nB + 3 * nV;
    // items in the order (step, phase, pair, unit); an item waits only for the
    // previous phase of its own pair, whose items all come earlier in the order
    for (int it; (it = next_item(A.ctl, &s_item)) < A.iters * per_step;) {
        const int k = it / per_step;
        int r = it - k * per_step;
        if (r < nA) {
            // ---------------------------------------------------------------- A: H d pieces
            int p;
            if (r < A.colOff[np]) p = find_pair(A.colOff, np, r);
            else if (r < A.vccOff[np]) p = find_pair(A.vccOff, np, r);
            else p = find_pair(A.curvOff, np, r);
            const KPair &P = A.p[p];
            if (k > 0 && !wait_done(A, p, 4, (unsigned)k * P.nV, &s_ok)) return;
            if (r < A.colOff[np]) {
                gn_column(P, smem, bars, r - A.colOff[p], pbits);
            } else if (r < A.vccOff[np]) {
                const int v = tid / vcck::NC;
                const int *nb = P.b.vcc.nb;
                for (int bid = (r - A.vccOff[p]) * kVccPer + v, e = min(bid - v + kVccPer, P.nvcc); bid < e;
                     bid += kVccRun) {
                    const VBlock b = warp_block(tid % vcck::NC, bid, nb[0], nb[1], nb[2], 1 + v, vcck::NC);
                    vcck::vcc_cell_body<1>(P.b.vcc, b, reinterpret_cast<vcck::VccSmem *>(smem)[v]);
                }
            } else {
                const int v = tid / nodek::NT;
                if (v < kNodeRun)
                    for (int bid = (r - A.curvOff[p]) * kNodePer + v, e = min(bid - v + kNodePer, P.nnode); bid < e;
                         bid += kNodeRun)
                        nodek::curv_body<false>(P.b.nodes, node_block(P, tid, bid, v),
                                                reinterpret_cast<nodek::NodeSmem *>(smem)[v]);
            }
            item_done(A, p, 0, it);
            continue;
        }
        r -= nA;
        if (r < nB) {
            // ---------------------------------------------------------------- B: node pass, d . q partials
            const int p = find_pair(A.nodeOff, np, r);
            const KPair &P = A.p[p];
            if (!wait_done(A, p, 0, (unsigned)(k + 1) * P.nA, &s_ok)) return;
            const int v = tid / nodek::NT;
            if (v < kNodeRun)
                for (int bid = (r - A.nodeOff[p]) * kNodePer + v, e = min(bid - v + kNodePer, P.nnode); bid < e;
                     bid += kNodeRun)
                    nodek::node_body<false>(P.b.nodes, node_block(P, tid, bid, v),
                                            reinterpret_cast<nodek::NodeSmem *>(smem)[v]);
            item_done(A, p, 1, it);
            continue;
        }
        // -------------------------------------------------------------------- C, D, E: the vector phases
        r -= nB;
        const int ph = r / nV;
        r -= ph * nV;
        const int p = find_pair(A.vecOff, np, r);
        const KPair &P = A.p[p];
        const unsigned need = (unsigned)(k + 1) * (ph == 0 ? P.nB : P.nV);
        if (!wait_done(A, p, 1 + ph, need, &s_ok)) return;
        const int b0 = (r - A.vecOff[p]) * kVecPer;
        for (int vb = b0; tid < pcgk::kVT && vb < min(b0 + kVecPer, P.nvec); ++vb) {
            const VBlock b = warp_block(tid, vb, P.nvec, 1, 1, 1, pcgk::kVT);
            const PcgArgs &g = P.b.pcg;
            pcgk::PcgSmem &sm = *reinterpret_cast<pcgk::PcgSmem *>(smem);
            if (vb > b0) b.sync();   // the last block's reads of the shared scratch are done
            if (ph == 0)
                pcgk::pcg_step_body(P.part, g.sc, g.apart, P.nnode, P.b.nodes.out, g.minv, g.Rh, g.stride, k, g.part,
                                    b, sm);
            else if (ph == 1)
                pcgk::pcg_reorth_body(P.part, g.sc, g.minv, g.Rh, g.stride, k, g.rzh, g.part, g.rzpart, b, sm);
            else
                pcgk::pcg_dir_body(P.part, g.sc, g.minv, g.Rh + (long)(k + 1) * g.stride, g.d, P.b.s, k, g.rzh,
                                   g.rzpart, b, sm);
        }
        item_done(A, p, 2 + ph, it);
    }
}

size_t batch_smem(const KArgs &A) {
    size_t s = std::max(sizeof(pcgk::PcgSmem),
                        std::max(kVccRun * sizeof(vcck::VccSmem), kNodeRun * sizeof(nodek::NodeSmem)));
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
        P.nB = (P.nnode + kNodePer - 1) / kNodePer;
        P.nA = P.ncols + (P.nvcc + kVccPer - 1) / kVccPer + P.nB;
        P.nV = (P.nvec + kVecPer - 1) / kVecPer;
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
    for (int p = 0; p < npairs; ++p) { A.vecOff[p] = n; n += A.p[p].nV; }
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
