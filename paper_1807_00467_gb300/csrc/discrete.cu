// Discrete keypoint stage, Sec. II-C: NGF features, the patch cost volume of
// Eq. 2 over 33^3 displacement labels, the minimum spanning tree of the edge
// weights of Eq. 3, exact min-marginals by two passes of min-sum belief
// propagation (Eq. 4), and the symmetric refinement of Sec. II-C4.
//
// Layouts.  Images and features are [z][y][x] at 1 mm spacing; a feature is
// the float4 (grad I, eta) / ||(grad I, eta)||.  Keypoints are int32 (x, y, z)
// voxel positions.  Labels: d = 2 (i - 16) per axis, l = (i_z 33 + i_y) 33 + i_x;
// cost volumes, messages and marginals are float [k][l].
//
// Decisions that produce integers are taken in FP32 by rules both sides of
// the parity tests share: the MST edge weight is rounded after each operation
// (sqrt, difference, division, sum) and edges are ordered by (weight, smaller
// index, larger index); the label argmin takes the lowest index among equal
// energies.
#include <cooperative_groups.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "../../include/ngfreg.h"
#include "common.cuh"

namespace cg = cooperative_groups;

namespace ngf {
namespace {

constexpr int kS = 33;              // labels per axis
constexpr int kL = kS * kS * kS;    // 35937 labels
constexpr int kPlane = kS * kS;     // labels per z plane
constexpr int kW = kS + 3;          // window points per axis: patch (4) + labels (33) - 1
constexpr int kCvG = 2;             // z labels per cost-volume CTA
constexpr int kCvT = 224;           // cost-volume threads (2 x 33 rows x 3 runs of 11 labels = 198 busy)
constexpr int kRun = 11;            // labels per thread along x
constexpr int kCl = 8;              // CTAs per message (one thread-block cluster)
constexpr int kBpT = 256;           // threads per message CTA

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------------------ features
__global__ void features_kernel(int nx, int ny, int nz, const float *img, float eta, float4 *feat) {
    const long N = (long)nx * ny * nz;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        auto at = [&](int xx, int yy, int zz) {
            return __ldg(img + ((long)clampi(zz, 0, nz - 1) * ny + clampi(yy, 0, ny - 1)) * nx + clampi(xx, 0, nx - 1));
        };
        const float gx = 0.5f * (at(x + 1, y, z) - at(x - 1, y, z));
        const float gy = 0.5f * (at(x, y + 1, z) - at(x, y - 1, z));
        const float gz = 0.5f * (at(x, y, z + 1) - at(x, y, z - 1));
        const float s = __frsqrt_rn(fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, eta * eta))));
        feat[i] = make_float4(gx * s, gy * s, gz * s, eta * s);
    }
}

// ------------------------------------------------------------ cost volume
// CTA (keypoint k, z labels 2g, 2g + 1): the moving features at the window
// points k + 2 w - 35 (w = 0..35 per axis) of the kCvG + 3 planes it needs are
// staged in shared memory; thread (dz, dy, run) accumulates 11 labels along x,
// reusing each loaded window row for 11 labels x 4 patch columns.
__global__ void __launch_bounds__(kCvT) cost_volume_kernel(int nx, int ny, int nz, const float4 *__restrict__ ffix,
                                                           const float4 *__restrict__ fmov, const int *__restrict__ kps,
                                                           float *__restrict__ D) {
    extern __shared__ float4 sm4[];
    float4 *win = sm4;                          // [kCvG + 3][kW][kW]
    float4 *pf = sm4 + (kCvG + 3) * kW * kW;    // [4][4][4] fixed patch
    const int ng = (kS + kCvG - 1) / kCvG;
    const int k = blockIdx.x / ng, g = blockIdx.x - k * ng;
    const int kx = kps[3 * k], ky = kps[3 * k + 1], kz = kps[3 * k + 2];
    const int dz0 = g * kCvG;
    const int tid = threadIdx.x;
    for (int i = tid; i < (kCvG + 3) * kW * kW; i += kCvT) {
        const int pz = i / (kW * kW), r = i - pz * kW * kW, wy = r / kW, wx = r - wy * kW;
        const int z = clampi(kz + 2 * (dz0 + pz) - 35, 0, nz - 1);
        const int y = clampi(ky + 2 * wy - 35, 0, ny - 1), x = clampi(kx + 2 * wx - 35, 0, nx - 1);
        win[i] = __ldg(fmov + ((long)z * ny + y) * nx + x);
    }
    if (tid < 64) {
        const int px = tid & 3, py = (tid >> 2) & 3, pz = tid >> 4;
        const int z = clampi(kz + 2 * pz - 3, 0, nz - 1), y = clampi(ky + 2 * py - 3, 0, ny - 1);
        const int x = clampi(kx + 2 * px - 3, 0, nx - 1);
        pf[tid] = __ldg(ffix + ((long)z * ny + y) * nx + x);
    }
    __syncthreads();
    const int run = tid % 3, dy = (tid / 3) % kS, dzl = tid / (3 * kS);
    const int dz = dz0 + dzl;
    if (dzl >= kCvG || dz >= kS) return;
    const int dx0 = run * kRun;
    float acc[kRun];
#pragma unroll
    for (int j = 0; j < kRun; ++j) acc[j] = 0.f;
#pragma unroll 1
    for (int pz = 0; pz < 4; ++pz) {
#pragma unroll 1
        for (int py = 0; py < 4; ++py) {
            const float4 *row = win + ((dzl + pz) * kW + (dy + py)) * kW + dx0;
            float4 m[kRun + 3];
#pragma unroll
            for (int j = 0; j < kRun + 3; ++j) m[j] = row[j];
            const float4 *f = pf + (pz * 4 + py) * 4;
#pragma unroll
            for (int px = 0; px < 4; ++px) {
                const float4 q = f[px];
#pragma unroll
                for (int j = 0; j < kRun; ++j) {
                    const float4 a = m[j + px];
                    const float r = fmaf(a.w, q.w, fmaf(a.z, q.z, fmaf(a.y, q.y, a.x * q.x)));
                    acc[j] = fmaf(r, r, acc[j]);
                }
            }
        }
    }
    float *out = D + (long)k * kL + ((long)dz * kS + dy) * kS + dx0;
#pragma unroll
    for (int j = 0; j < kRun; ++j) out[j] = fmaf(-acc[j], 1.f / 64.f, 1.f);
}

// ------------------------------------------------------------ MST (Boruvka)
__device__ __forceinline__ float edge_w(const int *kps, const float *inten, float sig, int a, int b) {
    const int dx = kps[3 * a] - kps[3 * b], dy = kps[3 * a + 1] - kps[3 * b + 1], dz = kps[3 * a + 2] - kps[3 * b + 2];
    const float dist = __fsqrt_rn((float)(dx * dx + dy * dy + dz * dz));
    return __fadd_rn(dist, __fdiv_rn(fabsf(__fsub_rn(inten[a], inten[b])), sig));
}
// weight bits (non-negative floats order as their bit patterns), then the
// smaller and the larger index: a strict total order on the edges
__device__ __forceinline__ unsigned long long edge_key(float w, int a, int b) {
    const unsigned lo = a < b ? a : b, hi = a < b ? b : a;
    return ((unsigned long long)__float_as_uint(w) << 32) | (lo << 16) | hi;
}

__global__ void mst_init_kernel(int n, int *comp, int *hook, unsigned long long *best, int *nedges) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        comp[v] = v;
        hook[v] = v;
        best[v] = ~0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *nedges = 0;
}

// per vertex (one warp): the lightest edge to another component, then the
// minimum per component
__global__ void mst_min_edge_kernel(int n, const int *kps, const float *inten, float sig, const int *comp,
                                    unsigned long long *best) {
    const int lane = threadIdx.x & 31;
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= n) return;
    const int cv = comp[v];
    unsigned long long b = ~0ull;
    for (int u = lane; u < n; u += 32)
        if (comp[u] != cv) {
            const unsigned long long key = edge_key(edge_w(kps, inten, sig, v, u), v, u);
            b = key < b ? key : b;
        }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t < b ? t : b;
    }
    if (lane == 0 && b != ~0ull) atomicMin(best + cv, b);
}

// each component adds its lightest edge and hooks onto the component at the
// other end; of a mutual pair (both chose the same edge) the smaller adds the
// edge and the larger hooks
__global__ void mst_hook_kernel(int n, const int *comp, const unsigned long long *best, int *hook, int *edges,
                                int *nedges) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        if (comp[c] != c || best[c] == ~0ull) continue;
        const int lo = (int)((best[c] >> 16) & 0xffff), hi = (int)(best[c] & 0xffff);
        const int d = comp[lo] == c ? comp[hi] : comp[lo];
        const bool mutual = best[d] == best[c];
        if (!mutual || c < d) {
            const int s = atomicAdd(nedges, 1);
            if (s < n - 1) {
                edges[2 * s] = lo;
                edges[2 * s + 1] = hi;
            }
        }
        if (!mutual || c > d) hook[c] = d;
    }
}

// components = roots of the hook forest (chains end after < n steps)
__global__ void mst_jump_kernel(int n, const int *hook, int *comp) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int r = comp[v];
        for (int s = 0; s < n && hook[r] != r; ++s) r = hook[r];
        comp[v] = r;
    }
}

__global__ void mst_reset_kernel(int n, int *hook, unsigned long long *best) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        hook[v] = v;
        best[v] = ~0ull;
    }
}

// edges sorted by (lo, hi): each edge's rank counted over all edges
__global__ void mst_sort_kernel(int m, const int *edges, const int *nedges, int *out, int *err) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && *nedges != m) atomicExch(err, 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const long ki = ((long)edges[2 * i] << 16) | edges[2 * i + 1];
        int r = 0;
        for (int j = 0; j < m; ++j) {
            const long kj = ((long)edges[2 * j] << 16) | edges[2 * j + 1];
            r += kj < ki;
        }
        out[2 * r] = edges[2 * i];
        out[2 * r + 1] = edges[2 * i + 1];
    }
}

// ------------------------------------------------------------ tree
// One CTA: adjacency lists (sorted), breadth-first levels from the centre of
// a longest path (found by two sweeps from `root`), parents and sorted child
// lists; order[0] is the root the messages run to.  Edges with an index outside [0, n) or
// equal ends are ignored and each vertex is claimed once, so a list that is
// not a spanning tree cannot write out of bounds (vertices it does not reach
// are left out of the levels).  Scratch: deg/off [n + 1] each, adj [2 n].
__device__ __forceinline__ bool edge_ok(int n, int a, int b) { return a >= 0 && a < n && b >= 0 && b < n && a != b; }

// exclusive scan of cnt[0..n) into out[0..n], one CTA (chunks per thread)
__device__ void cta_scan(int n, const int *cnt, int *out, int *s_part) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (n + nt - 1) / nt, a0 = min(n, tid * chunk), a1 = min(n, a0 + chunk);
    int s = 0;
    for (int v = a0; v < a1; ++v) s += cnt[v];
    s_part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int i = 0; i < nt; ++i) {
            const int x = s_part[i];
            s_part[i] = t;
            t += x;
        }
        s_part[nt] = t;
    }
    __syncthreads();
    s = s_part[tid];
    for (int v = a0; v < a1; ++v) {
        const int c = cnt[v];
        out[v] = s;
        s += c;
    }
    if (tid == 0) out[n] = s_part[nt];
    __syncthreads();
}

__global__ void __launch_bounds__(1024) tree_kernel(int n, int root, const int *edges, int *deg, int *off, int *adj,
                                                    int *order, int *level_off, int *nlevels, int *parent,
                                                    int *child_off, int *child) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_count, s_lvl, s_far, s_root;
    __shared__ int s_part[1025];
    for (int v = tid; v <= n; v += nt) deg[v] = 0;
    __syncthreads();
    for (int e = tid; e < n - 1; e += nt) {
        const int a = edges[2 * e], b = edges[2 * e + 1];
        if (!edge_ok(n, a, b)) continue;
        atomicAdd(deg + a, 1);
        atomicAdd(deg + b, 1);
    }
    __syncthreads();
    cta_scan(n, deg, off, s_part);
    for (int v = tid; v < n; v += nt) deg[v] = off[v];   // fill cursors
    __syncthreads();
    for (int e = tid; e < n - 1; e += nt) {
        const int a = edges[2 * e], b = edges[2 * e + 1];
        if (!edge_ok(n, a, b)) continue;
        adj[atomicAdd(deg + a, 1)] = b;
        adj[atomicAdd(deg + b, 1)] = a;
    }
    __syncthreads();
    for (int v = tid; v < n; v += nt)   // insertion sort of each (short) list
        for (int i = off[v] + 1; i < off[v + 1]; ++i) {
            const int x = adj[i];
            int j = i - 1;
            while (j >= off[v] && adj[j] > x) {
                adj[j + 1] = adj[j];
                --j;
            }
            adj[j + 1] = x;
        }
    __syncthreads();
    // breadth-first levels from r: order[], level_off[], parent[]; returns the
    // number of levels and (in s_far) the smallest index on the deepest level
    auto bfs = [&](int r) {
        for (int v = tid; v < n; v += nt) parent[v] = -2;   // unvisited
        __syncthreads();
        if (tid == 0) {
            order[0] = r;
            parent[r] = -1;
            level_off[0] = 0;
            level_off[1] = 1;
            s_count = 1;
            s_lvl = 0;
        }
        __syncthreads();
        for (int lv = 0; lv < n; ++lv) {   // at most n levels
            const int b0 = level_off[lv], b1 = level_off[lv + 1];
            if (b0 == b1) break;
            for (int i = b0 + tid; i < b1; i += nt) {
                const int v = order[i];
                for (int j = off[v]; j < off[v + 1]; ++j) {
                    const int u = adj[j];
                    if (atomicCAS(parent + u, -2, v) == -2) order[atomicAdd(&s_count, 1)] = u;
                }
            }
            __syncthreads();
            if (tid == 0) {
                level_off[lv + 2] = s_count;
                s_lvl = lv + 1;
            }
            __syncthreads();
        }
        if (tid == 0) {
            int far = n;
            for (int i = level_off[s_lvl - 1]; i < level_off[s_lvl]; ++i) far = min(far, order[i]);
            s_far = far;
        }
        __syncthreads();
    };
    // root = centre of a longest path (two sweeps), so the levels are fewest
    bfs(root);
    bfs(s_far);
    if (tid == 0) {
        int c = s_far;
        for (int st = 0; st < (s_lvl - 1) / 2; ++st) c = parent[c];
        s_root = c;
    }
    __syncthreads();
    bfs(s_root);
    if (tid == 0) *nlevels = s_lvl;   // levels 0 .. s_lvl - 1 are non-empty
    // child lists: the neighbours claimed by v, in sorted order
    for (int v = tid; v < n; v += nt) {
        int c = 0;
        for (int j = off[v]; j < off[v + 1]; ++j) c += parent[adj[j]] == v;
        deg[v] = c;
    }
    __syncthreads();
    cta_scan(n, deg, child_off, s_part);
    for (int v = tid; v < n; v += nt) {
        int c = child_off[v];
        for (int j = off[v]; j < off[v + 1]; ++j)
            if (parent[adj[j]] == v) child[c++] = adj[j];
    }
}

// ------------------------------------------------------------ belief propagation
// One 33-point line of the min-convolution: out[j] = min_i v[i] + C[|i - j|].
__device__ __forceinline__ void min_conv_line(float (&v)[kS], const float (&C)[kS]) {
    float o[kS];
#pragma unroll
    for (int j = 0; j < kS; ++j) {
        float m = v[j];   // C[0] = 0
#pragma unroll
        for (int i = 0; i < kS; ++i)
            if (i != j) m = fminf(m, v[i] + C[i > j ? i - j : j - i]);
        o[j] = m;
    }
#pragma unroll
    for (int j = 0; j < kS; ++j) v[j] = o[j];
}

struct BpArgs {
    const float *D;        // [n][L] unary costs
    float *up;             // [n][L] message to the parent
    float *marg;           // [n][L] marginals
    const int *order, *parent, *child_off, *child;
    const int *kps;
    const float *inten;
    float sig, alpha;
    int base;              // first vertex of the level in order[]
};

// Message of vertex k (DOWN: message of its parent q to k, then k's marginal),
// spread over a cluster of 8 CTAs: CTA r owns z planes [4 r, 4 r + 4) (the
// last one also plane 32), runs the x and y passes on them, and after a
// cluster barrier the z pass on its share of the 1089 (y, x) columns, reading
// the planes of the other CTAs through distributed shared memory.  The UP
// pass leaves h_k = D_k + sum of the children's messages in marg[k]; the DOWN
// pass adds the parent's message to it, which completes k's marginal.
template <bool DOWN>
__global__ void __launch_bounds__(kBpT) bp_message_kernel(const BpArgs a) {
    constexpr int kPer = (5 * kPlane + kBpT - 1) / kBpT;   // slab values per thread
    __shared__ float s[5 * kPlane];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int k = a.order[a.base + blockIdx.x / kCl];
    const int q = a.parent[k];
    const int z0 = 4 * r, nzp = r == kCl - 1 ? 5 : 4, nown = nzp * kPlane;
    const int tid = threadIdx.x;
    const float lam = __fdiv_rn(a.alpha, edge_w(a.kps, a.inten, a.sig, k, q));
    float C[kS];
#pragma unroll
    for (int d = 0; d < kS; ++d) C[d] = d == 0 ? 0.f : lam * (float)(4 * d * d);
    // h over the own planes (all loads of one array issued together): UP:
    // D_k + the children's messages; DOWN: the parent's marginal without k's message
    const long pb = (long)z0 * kPlane;
    {
        float h[kPer];
        const float *src = DOWN ? a.marg + (long)q * kL + pb : a.D + (long)k * kL + pb;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int i = tid + t * kBpT;
            h[t] = i < nown ? __ldg(src + i) : 0.f;
        }
        if (DOWN) {
            const float *u = a.up + (long)k * kL + pb;
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int i = tid + t * kBpT;
                if (i < nown) h[t] -= __ldg(u + i);
            }
        } else {
            for (int c = a.child_off[k]; c < a.child_off[k + 1]; ++c) {
                const float *u = a.up + (long)a.child[c] * kL + pb;
#pragma unroll
                for (int t = 0; t < kPer; ++t) {
                    const int i = tid + t * kBpT;
                    if (i < nown) h[t] += __ldg(u + i);
                }
            }
            float *mk = a.marg + (long)k * kL + pb;
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int i = tid + t * kBpT;
                if (i < nown) mk[i] = h[t];
            }
        }
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int i = tid + t * kBpT;
            if (i < nown) s[i] = h[t];
        }
    }
    __syncthreads();
    // x pass, y pass (own planes, one line per thread), then the z pass over
    // columns [j0, j1) of all planes; one copy of the line code for all three
    const int per = (kPlane + kCl - 1) / kCl, j0 = r * per, j1 = min(kPlane, j0 + per);
    const int zl = tid / kS, w = tid - zl * kS, j = j0 + tid;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
        if (pass == 2) cl.sync();   // every CTA's planes are complete
        const bool act = pass < 2 ? tid < nzp * kS : j < j1;
        float v[kS];
        if (act) {
            if (pass < 2) {
                const int base = zl * kPlane + (pass == 0 ? w * kS : w), step = pass == 0 ? 1 : kS;
#pragma unroll
                for (int i = 0; i < kS; ++i) v[i] = s[base + i * step];
            } else {
#pragma unroll
                for (int z = 0; z < kS; ++z) {
                    const int owner = z / 4 < kCl - 1 ? z / 4 : kCl - 1;
                    const float *rs = cl.map_shared_rank(s, owner);
                    v[z] = rs[(z - 4 * owner) * kPlane + j];
                }
            }
            min_conv_line(v, C);
            if (pass < 2) {
                const int base = zl * kPlane + (pass == 0 ? w * kS : w), step = pass == 0 ? 1 : kS;
#pragma unroll
                for (int i = 0; i < kS; ++i) s[base + i * step] = v[i];
            } else if (DOWN) {
                float *mk = a.marg + (long)k * kL + j;
#pragma unroll
                for (int z = 0; z < kS; ++z) mk[(long)z * kPlane] += v[z];
            } else {
                float *uk = a.up + (long)k * kL + j;
#pragma unroll
                for (int z = 0; z < kS; ++z) uk[(long)z * kPlane] = v[z];
            }
        }
        if (pass < 2) __syncthreads();
    }
    cl.sync();   // no CTA leaves while another may still read its planes
}

// marginal of the root (order[0]): D + the children's messages
__global__ void bp_root_kernel(const BpArgs a) {
    const int root = a.order[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kL; i += gridDim.x * blockDim.x) {
        float m = a.D[(long)root * kL + i];
        for (int c = a.child_off[root]; c < a.child_off[root + 1]; ++c) m += a.up[(long)a.child[c] * kL + i];
        a.marg[(long)root * kL + i] = m;
    }
}

// ------------------------------------------------------------ argmin, refinement
// per keypoint: the label of least energy (lowest index among equal values);
// with Eb: energy (E + Eb(mirrored label)) / 2.  Writes the displacement and,
// when kps_out is given, the moved keypoint.
__global__ void __launch_bounds__(256) argmin_kernel(int n, const float *E, const float *Eb, const int *kps,
                                                     int *disp, int *kps_out) {
    const int k = blockIdx.x;
    float bv = __int_as_float(0x7f800000);
    int bl = kL;
    for (int l = threadIdx.x; l < kL; l += blockDim.x) {
        float e = E[(long)k * kL + l];
        if (Eb) {
            const int ix = l % kS, iy = (l / kS) % kS, iz = l / kPlane;
            const int m = ((kS - 1 - iz) * kS + (kS - 1 - iy)) * kS + (kS - 1 - ix);
            e = 0.5f * (e + Eb[(long)k * kL + m]);
        }
        if (e < bv || (e == bv && l < bl)) {
            bv = e;
            bl = l;
        }
    }
    __shared__ float sv[256];
    __shared__ int sl[256];
    sv[threadIdx.x] = bv;
    sl[threadIdx.x] = bl;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const float v2 = sv[threadIdx.x + o];
            const int l2 = sl[threadIdx.x + o];
            if (v2 < sv[threadIdx.x] || (v2 == sv[threadIdx.x] && l2 < sl[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                sl[threadIdx.x] = l2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int l = sl[0] < kL ? sl[0] : kL / 2;   // all NaN: label 0
        const int d[3] = {2 * (l % kS - 16), 2 * ((l / kS) % kS - 16), 2 * (l / kPlane - 16)};
        for (int c = 0; c < 3; ++c) {
            disp[3 * k + c] = d[c];
            if (kps_out) kps_out[3 * k + c] = kps[3 * k + c] + d[c];
        }
    }
}

__global__ void gather_intensity_kernel(int nx, int ny, int nz, const float *img, int n, const int *kps, float *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int x = clampi(kps[3 * k], 0, nx - 1), y = clampi(kps[3 * k + 1], 0, ny - 1);
        const int z = clampi(kps[3 * k + 2], 0, nz - 1);
        out[k] = img[((long)z * ny + y) * nx + x];
    }
}

__global__ void flag_kernel(int *err) { *err = 0; }

// ------------------------------------------------------------ host side
struct KpWs {
    float4 *fF, *fM;
    float *D, *up, *E1, *E2;
    float *inten;
    int *kps2, *disp1;
    int *comp, *hook, *edges_raw, *edges, *nedges, *err;
    unsigned long long *best;
    int *deg, *off, *adj, *order, *level_off, *nlevels, *parent, *child_off, *child;
};

struct Carve {
    char *base;
    size_t off;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// match == 0: scratch of kp_mst / kp_bp_marginals only (no features or volumes)
size_t kp_layout(Carve &cv, KpWs &w, long N, int n, bool match) {
    w.fF = match ? cv.take<float4>(N) : nullptr;
    w.fM = match ? cv.take<float4>(N) : nullptr;
    w.D = match ? cv.take<float>((size_t)n * kL) : nullptr;
    w.up = cv.take<float>((size_t)n * kL);
    w.E1 = match ? cv.take<float>((size_t)n * kL) : nullptr;
    w.E2 = match ? cv.take<float>((size_t)n * kL) : nullptr;
    w.inten = cv.take<float>(n);
    w.kps2 = cv.take<int>(3 * (size_t)n);
    w.disp1 = cv.take<int>(3 * (size_t)n);
    w.comp = cv.take<int>(n);
    w.hook = cv.take<int>(n);
    w.edges_raw = cv.take<int>(2 * (size_t)n);
    w.edges = cv.take<int>(2 * (size_t)n);
    w.nedges = cv.take<int>(1);
    w.err = cv.take<int>(1);
    w.best = cv.take<unsigned long long>(n);
    w.deg = cv.take<int>(n + 1);
    w.off = cv.take<int>(n + 1);
    w.adj = cv.take<int>(2 * (size_t)n);
    w.order = cv.take<int>(n);
    w.level_off = cv.take<int>(n + 2);
    w.nlevels = cv.take<int>(1);
    w.parent = cv.take<int>(n);
    w.child_off = cv.take<int>(n + 1);
    w.child = cv.take<int>(n);
    return (cv.off + 255) & ~(size_t)255;
}

std::atomic<long long> g_kp_launches{0};   // kernels launched by the entry points of this file
inline void counted(long long n = 1) { g_kp_launches.fetch_add(n, std::memory_order_relaxed); }

int grid_for(long n, int t) { return (int)std::min<long>((n + t - 1) / t, 152L * 16); }

cudaError_t run_features(const int *n, const float *img, float eta, float4 *feat, cudaStream_t st) {
    const long N = (long)n[0] * n[1] * n[2];
    features_kernel<<<grid_for(N, 256), 256, 0, st>>>(n[0], n[1], n[2], img, eta, feat);
    counted();
    return cudaGetLastError();
}

cudaError_t run_cost(const int *n, const float4 *ffix, const float4 *fmov, int nk, const int *kps, float *D,
                     cudaStream_t st) {
    if (nk <= 0) return cudaSuccess;
    const size_t smem = sizeof(float4) * ((kCvG + 3) * kW * kW + 64);
    cudaError_t e = allow_max_dynamic_smem(cost_volume_kernel);
    if (e != cudaSuccess) return e;
    const int ng = (kS + kCvG - 1) / kCvG;
    cost_volume_kernel<<<nk * ng, kCvT, smem, st>>>(n[0], n[1], n[2], ffix, fmov, kps, D);
    counted();
    return cudaGetLastError();
}

cudaError_t run_mst(int n, const int *kps, const float *inten, float sig, KpWs &w, cudaStream_t st) {
    const int gb = grid_for(n, 256);
    mst_init_kernel<<<gb, 256, 0, st>>>(n, w.comp, w.hook, w.best, w.nedges);
    int rounds = 1;
    while ((1 << (rounds - 1)) < n) ++rounds;   // components at least halve per round
    for (int it = 0; it < rounds; ++it) {
        mst_min_edge_kernel<<<(n * 32 + 255) / 256, 256, 0, st>>>(n, kps, inten, sig, w.comp, w.best);
        mst_hook_kernel<<<gb, 256, 0, st>>>(n, w.comp, w.best, w.hook, w.edges_raw, w.nedges);
        mst_jump_kernel<<<gb, 256, 0, st>>>(n, w.hook, w.comp);
        mst_reset_kernel<<<gb, 256, 0, st>>>(n, w.hook, w.best);
    }
    mst_sort_kernel<<<grid_for(n - 1, 128), 128, 0, st>>>(n - 1, w.edges_raw, w.nedges, w.edges, w.err);
    counted(2 + 4L * rounds);
    return cudaGetLastError();
}

cudaError_t launch_cluster(void (*kernel)(const BpArgs), int nverts, const BpArgs &a, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl * nverts);
    cfg.blockDim = dim3(kBpT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// Tree from the sorted MST edges, then the two passes; the level sizes are
// read back once (one synchronisation) to size the per-level launches.
int run_bp(int n, const float *D, const int *kps, const float *inten, float sig, float alpha, KpWs &w, float *marg,
           cudaStream_t st) {
    const int root = 0;   // start of the sweeps that find the tree's centre
    tree_kernel<<<1, 1024, 0, st>>>(n, root, w.edges, w.deg, w.off, w.adj, w.order, w.level_off, w.nlevels, w.parent,
                                    w.child_off, w.child);
    if (cudaGetLastError() != cudaSuccess) return RG_ECUDA;
    // the level count and offsets, read on the caller's stream in one synchronisation
    int nl = 0;
    std::vector<int> lo(n + 2);
    if (cudaMemcpyAsync(&nl, w.nlevels, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(lo.data(), w.level_off, sizeof(int) * (n + 2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RG_ECUDA;
    if (nl < 1 || nl > n) return RG_ECUDA;
    BpArgs a;
    a.D = D;
    a.up = w.up;
    a.marg = marg;
    a.order = w.order;
    a.parent = w.parent;
    a.child_off = w.child_off;
    a.child = w.child;
    a.kps = kps;
    a.inten = inten;
    a.sig = sig;
    a.alpha = alpha;
    long long cnt = 1;
    for (int lv = nl - 1; lv >= 1; --lv) {
        a.base = lo[lv];
        if (launch_cluster(bp_message_kernel<false>, lo[lv + 1] - lo[lv], a, st) != cudaSuccess) return RG_ECUDA;
        ++cnt;
    }
    bp_root_kernel<<<grid_for(kL, 256), 256, 0, st>>>(a);
    ++cnt;
    for (int lv = 1; lv < nl; ++lv) {
        a.base = lo[lv];
        if (launch_cluster(bp_message_kernel<true>, lo[lv + 1] - lo[lv], a, st) != cudaSuccess) return RG_ECUDA;
        ++cnt;
    }
    counted(cnt);
    return cudaGetLastError() == cudaSuccess ? RG_OK : RG_ECUDA;
}

}  // namespace
}  // namespace ngf

using namespace ngf;

static bool kp_ok(const int32_t *n, int32_t nk) {
    return n && n[0] > 0 && n[1] > 0 && n[2] > 0 && nk >= 2 && nk <= 65535;
}

extern "C" int kp_workspace_size(const int32_t *n, int32_t nk, size_t *bytes) {
    if (!kp_ok(n, nk) || !bytes) return RG_EINVAL;
    Carve cv{nullptr, 0};
    KpWs w;
    *bytes = kp_layout(cv, w, (long)n[0] * n[1] * n[2], nk, true);
    return RG_OK;
}

extern "C" int kp_scratch_size(int32_t nk, size_t *bytes) {
    if (nk < 2 || nk > 65535 || !bytes) return RG_EINVAL;
    Carve cv{nullptr, 0};
    KpWs w;
    *bytes = kp_layout(cv, w, 0, nk, false);
    return RG_OK;
}

extern "C" int kp_ngf_features(const int32_t *n, const float *img, double eta, float *feat, void *stream) {
    if (!n || !img || !feat || n[0] <= 0 || n[1] <= 0 || n[2] <= 0 || ((uintptr_t)feat & 15)) return RG_EINVAL;
    return run_features(n, img, (float)eta, (float4 *)feat, (cudaStream_t)stream) == cudaSuccess ? RG_OK : RG_ECUDA;
}

extern "C" int kp_cost_volume(const int32_t *n, const float *feat_fixed, const float *feat_moving, int32_t nk,
                              const int32_t *kps, float *D, void *stream) {
    if (!n || !feat_fixed || !feat_moving || !kps || !D || nk < 0 || ((uintptr_t)feat_fixed & 15) ||
        ((uintptr_t)feat_moving & 15))
        return RG_EINVAL;
    return run_cost(n, (const float4 *)feat_fixed, (const float4 *)feat_moving, nk, kps, D, (cudaStream_t)stream) ==
                   cudaSuccess
               ? RG_OK
               : RG_ECUDA;
}

static int kp_scratch(int32_t nk, void *ws, size_t ws_bytes, KpWs &w) {
    size_t need;
    if (kp_scratch_size(nk, &need) != RG_OK || !ws || ws_bytes < need || ((uintptr_t)ws & 255)) return RG_EINVAL;
    Carve cv{(char *)ws, 0};
    kp_layout(cv, w, 0, nk, false);
    return RG_OK;
}

extern "C" int kp_mst(int32_t nk, const int32_t *kps, const float *intensity, double sigma_i, int32_t *edges,
                      void *ws, size_t ws_bytes, void *stream) {
    KpWs w;
    if (!kps || !intensity || !edges || kp_scratch(nk, ws, ws_bytes, w) != RG_OK) return RG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    flag_kernel<<<1, 1, 0, st>>>(w.err);
    counted();
    if (run_mst(nk, kps, intensity, (float)sigma_i, w, st) != cudaSuccess) return RG_ECUDA;
    int err = 0;
    if (cudaMemcpyAsync(edges, w.edges, sizeof(int) * 2 * (nk - 1), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RG_ECUDA;
    return err ? RG_ECUDA : RG_OK;
}

extern "C" int kp_bp_marginals(int32_t nk, const float *D, const int32_t *kps, const float *intensity,
                               const int32_t *edges, double sigma_i, double alpha, float *marginals, void *ws,
                               size_t ws_bytes, void *stream) {
    KpWs w;
    if (!D || !kps || !intensity || !edges || !marginals || kp_scratch(nk, ws, ws_bytes, w) != RG_OK)
        return RG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(w.edges, edges, sizeof(int) * 2 * (nk - 1), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RG_ECUDA;
    return run_bp(nk, D, kps, intensity, (float)sigma_i, (float)alpha, w, marginals, st);
}

extern "C" int kp_match(const int32_t *n, const float *F, const float *M, int32_t nk, const int32_t *kps,
                        const kp_params *p, int32_t symmetric, int32_t *disp, float *marginals, void *ws,
                        size_t ws_bytes, void *stream) {
    size_t need;
    if (!kp_ok(n, nk) || !F || !M || !kps || !p || !disp || kp_workspace_size(n, nk, &need) != RG_OK || !ws ||
        ws_bytes < need || ((uintptr_t)ws & 255))
        return RG_EINVAL;
    Carve cv{(char *)ws, 0};
    KpWs w;
    kp_layout(cv, w, (long)n[0] * n[1] * n[2], nk, true);
    cudaStream_t st = (cudaStream_t)stream;
    const float sig = (float)p->sigma_i, alpha = (float)p->alpha;
    flag_kernel<<<1, 1, 0, st>>>(w.err);
    counted();
    if (run_features(n, F, (float)p->eta, w.fF, st) != cudaSuccess ||
        run_features(n, M, (float)p->eta, w.fM, st) != cudaSuccess)
        return RG_ECUDA;
    // forward: F fixed, M moving
    if (run_cost(n, w.fF, w.fM, nk, kps, w.D, st) != cudaSuccess) return RG_ECUDA;
    gather_intensity_kernel<<<grid_for(nk, 256), 256, 0, st>>>(n[0], n[1], n[2], F, nk, kps, w.inten);
    counted();
    if (run_mst(nk, kps, w.inten, sig, w, st) != cudaSuccess) return RG_ECUDA;
    int s = run_bp(nk, w.D, kps, w.inten, sig, alpha, w, w.E1, st);
    if (s) return s;
    float *E = w.E1, *Eb = nullptr;
    if (symmetric) {
        // backward from the forward match: M fixed, F moving
        argmin_kernel<<<nk, 256, 0, st>>>(nk, w.E1, nullptr, kps, w.disp1, w.kps2);
        if (run_cost(n, w.fM, w.fF, nk, w.kps2, w.D, st) != cudaSuccess) return RG_ECUDA;
        gather_intensity_kernel<<<grid_for(nk, 256), 256, 0, st>>>(n[0], n[1], n[2], M, nk, w.kps2, w.inten);
        counted(2);
        if (run_mst(nk, w.kps2, w.inten, sig, w, st) != cudaSuccess) return RG_ECUDA;
        if ((s = run_bp(nk, w.D, w.kps2, w.inten, sig, alpha, w, w.E2, st))) return s;
        Eb = w.E2;
    }
    argmin_kernel<<<nk, 256, 0, st>>>(nk, E, Eb, kps, disp, nullptr);
    counted();
    // marginals: forward [nk][L], then (symmetric) backward [nk][L]
    if (marginals) {
        if (cudaMemcpyAsync(marginals, E, sizeof(float) * (size_t)nk * kL, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return RG_ECUDA;
        if (Eb && cudaMemcpyAsync(marginals + (size_t)nk * kL, Eb, sizeof(float) * (size_t)nk * kL,
                                  cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return RG_ECUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RG_ECUDA;
    return err ? RG_ECUDA : RG_OK;
}

extern "C" int64_t kp_launch_count(void) { return g_kp_launches.load(); }
