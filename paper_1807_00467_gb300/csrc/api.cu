// C ABI of the ngfreg library: contexts over a caller-provided workspace,
// objective / gradient / Gauss-Newton products, PCG, the fixed Gauss-Newton
// schedule and the multilevel driver (Sec. II-D of arXiv 1807.00467).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/ngfreg.h"
#include "kernels.h"

using namespace ngf;

struct rg_ctx {
    rg_image_geom img;
    rg_grid_geom grid;
    rg_dtype dtype;
    rg_params P;
    int nk_max;
    int pcg_max;
    cudaStream_t st;
    const void *R, *T;
    int nk;
    const float *kx, *ky;
    long N, M;
    double g[3], hbar, ghat;
    TileGeom tg;
    BoxGeom bA, bB;
    int nA, nB, nR, nKb, nV;
    int nD;                   // D partials written by the last objective / gradient pass (tiles or columns)
    long nA_cap, boxA_cap;      // NGF tile scratch sized for every supported tile height
    float *lin_dT, *lin_a, *lin_u;
    float *boxA, *boxB, *curv_w;
    double *dpart, *rpart, *vpart, *kpart, *vecpart, *terms_tmp, *dminmax;
    int *fold;
    float *dmin, *dmax;
    float *minv, *d, *q, *tg_, *tu, *ts;
    float *Rh;                // PCG residual history, pcg_max + 1 slots of pcg_stride(3 M) floats
    int *tma_err;             // [0]: set by the kernels if a bounded TMA wait gave up; [1]: PCG ticket;
                              // [2]: set by the terms kernel when an objective came out NaN (or +inf without a fold)
    bool err_zeroed;
    CUtensorMap map_dT, map_a;
    ColGeom cg;               // column-marching GN-product kernel: geometry, tensor maps, node boxes
    CUtensorMap map_col_dT, map_col_a;
    BoxGeom bM;
    const BoxGeom *bcur;      // node-box geometry of the last NGF tile launch (read by the node pass)
    int hook_no_tma, hook_poll;   // test hooks (rg_debug_hook)
    int pass_sel;                 // objective / gradient pass: 0 by size, 1 column-marching, 2 tile
                                  // (autotuner choice, or the RG_HOOK_PASS test hook)
    double *rzh, *pcgpart, *rzpart, *apart;   // PCG: r_j.z_j, coefficient / r.z / d.q partials
    KpIndex kpix;             // keypoint index (rebuilt by rg_set_keypoints)
    PcgScalars *sc;
    bool has_lin, minv_valid;
    char err[512];
    GnState *gn;              // device side of a Gauss-Newton iteration
    double *gnrep;            // its report rows [kGnRows][RG_REPORT_COLS]
    double *range_terms;      // terms output of a d-range pass (volume term only)
    unsigned *bctl;           // control words of a persistent batched PCG launch led by this context
    const int *skip;          // set while a line-search try is launched: the try's kernels skip when *skip
    cudaStream_t gst;         // private stream of device-driven schedules (created on first use)
    cudaEvent_t gev[2];
    long long launches;       // library kernels launched (or replayed) for this context
    bool general_only;        // tile kernels: the general column kernel only (autotuner choice)
    // optional per-kernel CUDA-event timing (rg_profile)
    bool prof;
    std::vector<cudaEvent_t> *ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> *ev_used;
};

static std::atomic<long long> g_launches{0};
struct ProfScope;

// Record events around one library kernel launch when profiling is on.
struct ProfScope {
    rg_ctx *c;
    int id;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(rg_ctx *c_, int id_) : c(c_), id(id_) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (c) ++c->launches;
        if (!c || !c->prof) return;
        a = take();
        b = take();
        if (a && b) cudaEventRecord(a, c->st);
    }
    cudaEvent_t take() {
        cudaEvent_t e = nullptr;
        if (!c->ev_pool->empty()) {
            e = c->ev_pool->back();
            c->ev_pool->pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    }
    ~ProfScope() {
        if (!c || !c->prof || !a || !b) return;
        cudaEventRecord(b, c->st);
        c->ev_used->push_back({id, {a, b}});
    }
};

#define LAUNCH(id, expr)           \
    do {                           \
        ProfScope ps_(c, (id));    \
        CK(expr);                  \
    } while (0)

static int set_err(rg_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(expr)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return set_err(c, RG_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

static bool pow2_le8(int r) { return r == 1 || r == 2 || r == 4 || r == 8; }

static int check_geom(const rg_image_geom *img, const rg_grid_geom *grid) {
    if (!img || !grid) return RG_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (img->n[a] < 4 || grid->m[a] < 2 || !(img->h[a] > 0.0)) return RG_EINVAL;
        if (img->n[a] % (grid->m[a] - 1) != 0) return RG_EINVAL;
        if (!pow2_le8(img->n[a] / (grid->m[a] - 1))) return RG_EINVAL;
    }
    if ((long)img->n[0] * img->n[1] * img->n[2] >= (1L << 31) * 3L / 4) return RG_EINVAL;
    return RG_OK;
}

// Tile shape: TXI x TY voxel columns in x-y (one thread per column, plus a
// 2-voxel halo: TXI + 4 <= 32 lanes), TZ voxel planes per z chunk.
static void tile_geom(const rg_image_geom *img, const rg_grid_geom *grid, TileGeom &t, int TY = 16) {
    for (int a = 0; a < 3; ++a) {
        t.n[a] = img->n[a];
        t.m[a] = grid->m[a];
        t.rho[a] = img->n[a] / (grid->m[a] - 1);
        t.lrho[a] = t.rho[a] == 8 ? 3 : t.rho[a] == 4 ? 2 : t.rho[a] == 2 ? 1 : 0;
        t.irho[a] = 1.0f / (float)t.rho[a];
        t.invh[a] = (float)(1.0 / img->h[a]);
        t.invh_rel[a] = (float)(1.0 - img->h[a] * (double)t.invh[a]);
        t.inv2h[a] = (float)(1.0 / (2.0 * img->h[a]));
    }
    t.TXI = 28 - 28 % t.rho[0];
    t.TY = TY;
    // z chunk: 32 voxels, fewer (whole cells) while the per-CTA row sums of all
    // node planes ((TZ / rho_z + 1) x TY x (TXI / rho_x + 1) x 3 floats, twice) exceed 64 KB
    t.TZ = 32 - 32 % t.rho[2];
    while (t.TZ > t.rho[2] &&
           2L * (t.TZ / t.rho[2] + 1) * t.TY * (t.TXI / t.rho[0] + 1) * 3 * 4 > 64 * 1024)
        t.TZ -= t.rho[2];
    t.nxt = (t.TXI + 3) / t.rho[0] + 3;
    t.nyt = (t.TY + 3) / t.rho[1] + 3;
    t.C[0] = t.TXI / t.rho[0];
    t.C[1] = t.TY / t.rho[1];
    t.C[2] = t.TZ / t.rho[2];
    t.box = (t.C[0] + 1) * (t.C[1] + 1) * (t.C[2] + 1);
    t.nb[0] = (t.n[0] + t.TXI - 1) / t.TXI;
    t.nb[1] = (t.n[1] + t.TY - 1) / t.TY;
    t.nb[2] = (t.n[2] + t.TZ - 1) / t.TZ;
    t.tma = 0;
    // node planes of the chunk and its 2-plane halo, preloaded once per CTA if they fit in 48 KB
    t.nzt = (t.TZ + 3) / t.rho[2] + 3;
    if ((long)t.nzt * 3 * t.nxt * t.nyt > 12 * 1024) t.nzt = 0;
}

// Column geometry of the column-marching GN-product kernel: TXI x 16 voxel
// columns in x-y (TXI = 60 less a remainder so that it is whole cells), every z
// plane; node boxes [3][m3][C1 + 1][C0 + 1] per column.
static void col_geom(const rg_image_geom *img, const rg_grid_geom *grid, ColGeom &c) {
    for (int a = 0; a < 3; ++a) {
        c.n[a] = img->n[a];
        c.m[a] = grid->m[a];
        c.rho[a] = img->n[a] / (grid->m[a] - 1);
        c.lrho[a] = c.rho[a] == 8 ? 3 : c.rho[a] == 4 ? 2 : c.rho[a] == 2 ? 1 : 0;
        c.irho[a] = 1.0f / (float)c.rho[a];
        c.inv2h[a] = (float)(1.0 / (2.0 * img->h[a]));
    }
    c.TXI = 60 - 60 % c.rho[0];
    c.nb[0] = (c.n[0] + c.TXI - 1) / c.TXI;
    c.nb[1] = (c.n[1] + 15) / 16;
    c.C0 = c.TXI / c.rho[0];
    c.C1 = 16 / c.rho[1];
    // node columns of voxel columns x0 - 2 .. x0 + 61 (rows y0 - 2 .. y0 + 17) and the next node
    c.nxt = ((61 >> c.lrho[0]) + 1) - ((-2) >> c.lrho[0]) + 1;
    c.nyt = ((17 >> c.lrho[1]) + 1) - ((-2) >> c.lrho[1]) + 1;
    c.box = (c.C0 + 1) * (c.C1 + 1) * c.m[2];
    c.tma = 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA maps over a stored [3][n3][n2][n1] float field as the 4-D tensor
// {x, y, z, component}; box {box_x, TY + 4, 1, 3}.  Returns false (and the
// kernels read with plain loads) when the driver entry point is unavailable or
// the row pitch is not a multiple of 16 bytes.
static bool encode_field_map(CUtensorMap *map, const int *n, int TY, float *base, int box_x = kTmaBoxX) {
    if (n[0] % 4 != 0 || n[0] < box_x || n[1] < TY + 4) return false;
    static const EncodeTiledFn fn = [] {   // looked up once, also under concurrent callers
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return (EncodeTiledFn)f;
    }();
    if (!fn) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2], 3};
    const cuuint64_t strides[3] = {(cuuint64_t)n[0] * 4, (cuuint64_t)n[0] * n[1] * 4,
                                   (cuuint64_t)n[0] * n[1] * n[2] * 4};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)(TY + 4), 1, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Tile geometry for callers outside this file (the no-allocation entry point).
int ngf_host_tile_geom(const rg_image_geom *img, const rg_grid_geom *grid, double eta, TileGeom *t) {
    if (check_geom(img, grid) != RG_OK || !t) return RG_EINVAL;
    tile_geom(img, grid, *t);
    t->eta2 = (float)(eta * eta);
    return RG_OK;
}

struct Carver {
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

static void layout(rg_ctx *c, Carver &cv) {
    const long N = c->N, M = c->M;
    c->lin_dT = cv.take<float>(3 * N);
    c->lin_a = cv.take<float>(3 * N);
    c->lin_u = cv.take<float>(3 * M);
    c->boxA = cv.take<float>((size_t)c->boxA_cap);
    c->boxB = cv.take<float>((size_t)c->nB * 3 * c->bB.box);
    c->curv_w = cv.take<float>(3 * M);
    c->dpart = cv.take<double>(c->nA_cap);
    c->rpart = cv.take<double>(c->nR);
    c->vpart = cv.take<double>(c->nB);
    c->kpart = cv.take<double>(c->nKb);
    c->vecpart = cv.take<double>(c->nV);
    c->terms_tmp = cv.take<double>(8);
    c->dminmax = cv.take<double>(2);
    c->fold = cv.take<int>(c->nB);
    c->dmin = cv.take<float>(c->nB);
    c->dmax = cv.take<float>(c->nB);
    c->minv = cv.take<float>(3 * M);
    c->Rh = cv.take<float>(pcg_stride(3 * M) * (size_t)(c->pcg_max + 1));
    c->rzh = cv.take<double>(c->pcg_max + 1);
    c->pcgpart = cv.take<double>((size_t)pcg_blocks(3 * M) * (c->pcg_max + 2));
    c->rzpart = cv.take<double>(pcg_blocks(3 * M));
    c->apart = cv.take<double>(std::max(pcg_blocks(3 * M), c->nR));
    c->d = cv.take<float>(3 * M);
    c->q = cv.take<float>(3 * M);
    c->tg_ = cv.take<float>(3 * M);
    c->tu = cv.take<float>(3 * M);
    c->ts = cv.take<float>(3 * M);
    c->sc = cv.take<PcgScalars>(1);
    c->tma_err = cv.take<int>(4);
    c->gn = cv.take<GnState>(1);
    c->gnrep = cv.take<double>(RG_REPORT_COLS * kGnRows);
    c->range_terms = cv.take<double>(8);
    c->bctl = cv.take<unsigned>(kBatchCtlWords);
    const long nkx = c->nk_max > 0 ? c->nk_max : 0;
    c->kpix.cell = cv.take<int>(nkx);
    c->kpix.frac = cv.take<float>(3 * nkx);
    c->kpix.sb = cv.take<int>(nkx);
    c->kpix.perm = cv.take<int>(nkx);
    c->kpix.src = cv.take<float>(3 * nkx);
    c->kpix.soc = cv.take<int>(nkx > 0 ? M : 0);
}

static void derive(rg_ctx *c) {
    c->N = (long)c->img.n[0] * c->img.n[1] * c->img.n[2];
    c->M = (long)c->grid.m[0] * c->grid.m[1] * c->grid.m[2];
    for (int a = 0; a < 3; ++a) c->g[a] = c->img.n[a] * c->img.h[a] / (c->grid.m[a] - 1);
    c->hbar = c->img.h[0] * c->img.h[1] * c->img.h[2];
    c->ghat = c->g[0] * c->g[1] * c->g[2];
    c->nA_cap = 0;
    c->boxA_cap = 0;
    for (int ty : {8, 16}) {
        TileGeom t;
        tile_geom(&c->img, &c->grid, t, ty);
        const long n = (long)t.nb[0] * t.nb[1] * t.nb[2];
        if (n > c->nA_cap) c->nA_cap = n;
        if (n * 3 * t.box > c->boxA_cap) c->boxA_cap = n * 3 * t.box;
    }
    col_geom(&c->img, &c->grid, c->cg);
    {
        const long n = (long)c->cg.nb[0] * c->cg.nb[1] * 3 * c->cg.box;
        if (n > c->boxA_cap) c->boxA_cap = n;
    }
    c->bM.m[0] = c->grid.m[0];
    c->bM.m[1] = c->grid.m[1];
    c->bM.m[2] = c->grid.m[2];
    c->bM.nb[0] = c->cg.nb[0];
    c->bM.nb[1] = c->cg.nb[1];
    c->bM.nb[2] = 1;
    c->bM.C[0] = c->cg.C0;
    c->bM.C[1] = c->cg.C1;
    c->bM.C[2] = c->grid.m[2] - 1;
    c->bM.box = c->cg.box;
    tile_geom(&c->img, &c->grid, c->tg, 16);
    c->nA = c->tg.nb[0] * c->tg.nb[1] * c->tg.nb[2];
    c->nD = c->nA;
    for (int a = 0; a < 3; ++a) {
        c->bA.m[a] = c->grid.m[a];
        c->bA.nb[a] = c->tg.nb[a];
        c->bA.C[a] = c->tg.C[a];
        c->bB.m[a] = c->grid.m[a];
        c->bB.C[a] = kVccTile[a];
        c->bB.nb[a] = (c->grid.m[a] - 1 + kVccTile[a] - 1) / kVccTile[a];
    }
    c->bA.box = c->tg.box;
    c->bB.box = (kVccTile[0] + 1) * (kVccTile[1] + 1) * (kVccTile[2] + 1);
    c->nB = c->bB.nb[0] * c->bB.nb[1] * c->bB.nb[2];
    c->nR = node_blocks(c->grid.m);
    c->nKb = kp_blocks(c->nk_max > 0 ? c->nk_max : 1);
    c->nV = vec_blocks(3 * c->M);
}

extern "C" int rg_workspace_size(const rg_image_geom *img, const rg_grid_geom *grid, rg_dtype dtype, int32_t nk_max,
                                 int32_t pcg_max, size_t *bytes) {
    if (check_geom(img, grid) != RG_OK || !bytes || (dtype != RG_F32 && dtype != RG_F16) || nk_max < 0 ||
        pcg_max < 0 || pcg_max > RG_PCG_MAX)
        return RG_EINVAL;
    // the keypoint index holds cell indices and 8 nk gather threads in int
    if (nk_max > (1 << 27) || (nk_max > 0 && (long)grid->m[0] * grid->m[1] * grid->m[2] > INT_MAX)) return RG_EINVAL;
    rg_ctx tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.img = *img;
    tmp.grid = *grid;
    tmp.nk_max = nk_max;
    tmp.pcg_max = pcg_max;
    derive(&tmp);
    Carver cv{nullptr, 0};
    layout(&tmp, cv);
    *bytes = (cv.off + 255) & ~(size_t)255;
    return RG_OK;
}

extern "C" int rg_ctx_create(rg_ctx **out, const rg_image_geom *img, const rg_grid_geom *grid, rg_dtype dtype,
                             const rg_params *params, int32_t nk_max, int32_t pcg_max, void *ws, size_t ws_bytes,
                             void *stream) {
    if (!out || !params) return RG_EINVAL;
    *out = nullptr;
    size_t need = 0;
    int st = rg_workspace_size(img, grid, dtype, nk_max, pcg_max, &need);
    if (st != RG_OK) return st;
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return RG_EINVAL;
    rg_ctx *c = (rg_ctx *)calloc(1, sizeof(rg_ctx));
    if (!c) return RG_ENOMEM;
    c->img = *img;
    c->grid = *grid;
    c->dtype = dtype;
    c->P = *params;
    c->nk_max = nk_max;
    c->pcg_max = pcg_max;
    c->st = (cudaStream_t)stream;
    derive(c);
    Carver cv{(char *)ws, 0};
    layout(c, cv);
    c->tg.eta2 = (float)(params->eta * params->eta);
    c->tg.tma = (encode_field_map(&c->map_dT, c->tg.n, c->tg.TY, c->lin_dT) &&
                 encode_field_map(&c->map_a, c->tg.n, c->tg.TY, c->lin_a))
                    ? 1
                    : 0;
    c->cg.tma = (encode_field_map(&c->map_col_dT, c->cg.n, 16, c->lin_dT, kColBoxX) &&
                 encode_field_map(&c->map_col_a, c->cg.n, 16, c->lin_a, kColBoxX))
                    ? 1
                    : 0;
    c->bcur = &c->bA;
    c->hook_poll = 1 << 20;
    c->ev_pool = new std::vector<cudaEvent_t>();
    c->ev_used = new std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>();
    *out = c;
    return RG_OK;
}

extern "C" int rg_ctx_destroy(rg_ctx *c) {
    if (!c) return RG_OK;
    if (c->ev_used) {
        for (auto &u : *c->ev_used) {
            cudaEventDestroy(u.second.first);
            cudaEventDestroy(u.second.second);
        }
        delete c->ev_used;
    }
    if (c->ev_pool) {
        for (auto e : *c->ev_pool) cudaEventDestroy(e);
        delete c->ev_pool;
    }
    if (c->gst) {
        cudaStreamDestroy(c->gst);
        cudaEventDestroy(c->gev[0]);
        cudaEventDestroy(c->gev[1]);
    }
    free(c);
    return RG_OK;
}

extern "C" int rg_profile(rg_ctx *c, int32_t enable) {
    if (!c) return RG_EINVAL;
    c->prof = enable != 0;
    return RG_OK;
}

extern "C" int rg_profile_read(rg_ctx *c, int32_t kernel, double *total_ms, int64_t *launches) {
    if (!c || !total_ms || !launches) return RG_EINVAL;
    *total_ms = 0.0;
    *launches = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> keep;
    for (auto &u : *c->ev_used) {
        if (u.first != kernel) {
            keep.push_back(u);
            continue;
        }
        float ms = 0.f;
        CK(cudaEventSynchronize(u.second.second));
        CK(cudaEventElapsedTime(&ms, u.second.first, u.second.second));
        *total_ms += ms;
        *launches += 1;
        c->ev_pool->push_back(u.second.first);
        c->ev_pool->push_back(u.second.second);
    }
    c->ev_used->swap(keep);
    return RG_OK;
}

extern "C" int64_t rg_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" int rg_set_params(rg_ctx *c, const rg_params *p) {
    if (!c || !p || !(p->eta > 0.0) || p->alpha < 0 || p->gamma < 0 || p->delta < 0 || p->tau < 0)
        return set_err(c, RG_EINVAL, "rg_set_params: invalid parameters");
    c->P = *p;
    c->tg.eta2 = (float)(p->eta * p->eta);
    c->minv_valid = false;
    return RG_OK;
}

extern "C" int rg_get_params(const rg_ctx *c, rg_params *p) {
    if (!c || !p) return RG_EINVAL;
    *p = c->P;
    return RG_OK;
}

extern "C" int rg_set_stream(rg_ctx *c, void *stream) {
    if (!c) return RG_EINVAL;
    c->st = (cudaStream_t)stream;
    return RG_OK;
}

extern "C" int rg_set_tile(rg_ctx *c, int32_t tile_y) {
    if (!c) return RG_EINVAL;
    if (tile_y != 8 && tile_y != 16) return set_err(c, RG_EINVAL, "rg_set_tile: tile height %d not in {8, 16}", tile_y);
    const float eta2 = c->tg.eta2;
    tile_geom(&c->img, &c->grid, c->tg, tile_y);
    c->tg.eta2 = eta2;
    c->nA = c->tg.nb[0] * c->tg.nb[1] * c->tg.nb[2];
    c->nD = c->nA;
    for (int a = 0; a < 3; ++a) {
        c->bA.nb[a] = c->tg.nb[a];
        c->bA.C[a] = c->tg.C[a];
    }
    c->bA.box = c->tg.box;
    c->tg.tma = (encode_field_map(&c->map_dT, c->tg.n, c->tg.TY, c->lin_dT) &&
                 encode_field_map(&c->map_a, c->tg.n, c->tg.TY, c->lin_a))
                    ? 1
                    : 0;
    c->minv_valid = false;
    return RG_OK;
}

extern "C" int rg_set_images(rg_ctx *c, const void *R, const void *T) {
    if (!c || !R || !T) return set_err(c, RG_EINVAL, "rg_set_images: NULL image");
    c->R = R;
    c->T = T;
    c->has_lin = false;
    return RG_OK;
}

// keypoint launch arguments of the context (geometry, keypoints, index)
static KpArgs kp_args(const rg_ctx *c) {
    KpArgs k;
    for (int i = 0; i < 3; ++i) {
        k.m[i] = c->grid.m[i];
        k.ig[i] = (float)(1.0 / c->g[i]);
    }
    k.nk = c->nk;
    k.kx = c->kx;
    k.ky = c->ky;
    k.u = k.v = nullptr;
    k.scale = 1.f;
    k.out = nullptr;
    k.part = nullptr;
    k.ix = c->kpix;
    return k;
}

extern "C" int rg_set_keypoints(rg_ctx *c, int32_t nk, const float *x, const float *y) {
    if (!c) return RG_EINVAL;
    if (nk < 0 || nk > c->nk_max || (nk > 0 && (!x || !y)))
        return set_err(c, RG_EINVAL, "rg_set_keypoints: nk=%d exceeds nk_max=%d or NULL arrays", nk, c->nk_max);
    c->nk = nk;
    c->kx = x;
    c->ky = y;
    c->minv_valid = false;
    if (nk > 0) {
        const KpArgs k = kp_args(c);
        for (int step = 0; step < 3; ++step) LAUNCH(7, launch_kp_index(k, step, c->st));
    }
    return RG_OK;
}

// ---------------------------------------------------------------- internals
static int run_tile(rg_ctx *c, int mode, const float *field) {
    if (!c->R || !c->T) return set_err(c, RG_EINVAL, "images not set");
    if (!c->err_zeroed) {
        CK(cudaMemsetAsync(c->tma_err, 0, 4 * sizeof(int), c->st));
        c->err_zeroed = true;
    }
    auto fill = [&](auto &a) {
        a.g = c->tg;
        a.u = field;
        a.lin_dT = c->lin_dT;
        a.lin_a = c->lin_a;
        a.st_dT = c->lin_dT;
        a.st_a = c->lin_a;
        a.boxes = c->boxA;
        a.dpart = c->dpart;
        a.map_dT = c->map_dT;
        a.map_a = c->map_a;
        a.err = c->tma_err;
        a.skip = c->skip;
        a.poll_limit = c->hook_poll;
        a.no_tma = c->hook_no_tma;
    };
    const int pid = mode == MODE_MATVEC ? 0 : (mode == MODE_OBJ ? 2 : (mode == MODE_DIAG ? 10 : 1));
    c->bcur = &c->bA;
    if ((mode == MODE_MATVEC || mode == MODE_DIAG) && !c->general_only && gn_product_supported(c->cg)) {
        // the column-marching kernel (node boxes per column of the volume)
        ColArgs a;
        a.g = c->cg;
        a.v = field;
        a.boxes = c->boxA;
        a.map_dT = c->map_col_dT;
        a.map_a = c->map_col_a;
        a.err = c->tma_err;
        a.skip = c->skip;
        a.poll_limit = c->hook_poll;
        a.no_tma = c->hook_no_tma;
        LAUNCH(pid, launch_gn_product(a, mode == MODE_DIAG, c->st));
        c->bcur = &c->bM;
        return RG_OK;
    }
    if ((mode == MODE_MATVEC || mode == MODE_DIAG) && !c->general_only && gn_matvec_supported(c->tg)) {
        // the GN product and its diagonal read only the stored linearisation, not the images
        TileArgs<float> a;
        fill(a);
        a.R = a.T = nullptr;
        LAUNCH(pid, launch_gn_matvec(a, mode == MODE_DIAG, c->st));
        return RG_OK;
    }
    c->nD = c->nA;
    // the column-marching pass where it covers the volume with at least one
    // column per SM (narrower volumes keep the z-chunked tile pass, whose
    // tiles fill the GPU)
    const bool gcol = mode != MODE_MATVEC && mode != MODE_DIAG && !c->general_only && c->pass_sel != 2 &&
                      ngf_gcol_supported(c->cg) &&
                      (c->pass_sel == 1 || c->cg.nb[0] * c->cg.nb[1] >= device_sm_count());
    if (gcol) {
        // objective, gradient and linearisation: the column-marching pass
        auto gfill = [&](auto &g) {
            g.g = c->cg;
            for (int i = 0; i < 3; ++i) {
                g.invh[i] = c->tg.invh[i];
                g.invh_rel[i] = c->tg.invh_rel[i];
            }
            g.eta2 = c->tg.eta2;
            g.u = field;
            g.st_dT = c->lin_dT;
            g.st_a = c->lin_a;
            g.boxes = c->boxA;
            g.dpart = c->dpart;
            g.skip = c->skip;
        };
        if (c->dtype == RG_F32) {
            GcolArgs<float> g;
            gfill(g);
            g.R = (const float *)c->R;
            g.T = (const float *)c->T;
            LAUNCH(pid, launch_ngf_gcol(mode, g, c->st));
        } else {
            GcolArgs<__half> g;
            gfill(g);
            g.R = (const __half *)c->R;
            g.T = (const __half *)c->T;
            LAUNCH(pid, launch_ngf_gcol(mode, g, c->st));
        }
        c->bcur = &c->bM;
        c->nD = c->cg.nb[0] * c->cg.nb[1];
        return RG_OK;
    }
    // objective, gradient and linearisation: the persistent pass where the tile shape allows
    const bool grad_kernel =
        mode != MODE_MATVEC && mode != MODE_DIAG && !c->general_only && ngf_grad_supported(c->tg);
    if (c->dtype == RG_F32) {
        TileArgs<float> a;
        fill(a);
        a.R = (const float *)c->R;
        a.T = (const float *)c->T;
        if (grad_kernel) LAUNCH(pid, launch_ngf_grad(mode, a, c->st));
        else LAUNCH(pid, launch_ngf_tile(mode, a, c->st));
    } else {
        TileArgs<__half> a;
        fill(a);
        a.R = (const __half *)c->R;
        a.T = (const __half *)c->T;
        if (grad_kernel) LAUNCH(pid, launch_ngf_grad(mode, a, c->st));
        else LAUNCH(pid, launch_ngf_tile(mode, a, c->st));
    }
    return RG_OK;
}

static int run_vcc(rg_ctx *c, const float *u, const float *v, int diag = 0) {
    VccArgs a;
    a.diag = diag;
    for (int i = 0; i < 3; ++i) {
        a.m[i] = c->grid.m[i];
        a.ig[i] = (float)(1.0 / c->g[i]);
        a.nb[i] = c->bB.nb[i];
    }
    a.box = c->bB.box;
    a.u = u;
    a.v = v;
    a.wscale = 1.f;
    a.boxes = c->boxB;
    a.epart = c->vpart;
    a.fold = c->fold;
    a.dmin = c->dmin;
    a.dmax = c->dmax;
    a.skip = c->skip;
    LAUNCH((diag ? 10 : (a.v ? 4 : 3)), launch_vcc(a, c->st));
    return RG_OK;
}

// Node passes: w = L v and its energy partials when v is given (energy: keep
// the partials), then out = sA (NGF boxes) + sB (VCC boxes) + sC L^T w when
// out is given.
static int run_nodes(rg_ctx *c, const float *v, bool energy, float *out, double sA, double sB, double sC, bool useA,
                     bool useB, double *dpart = nullptr) {
    NodeArgs a;
    for (int i = 0; i < 3; ++i) {
        a.m[i] = c->grid.m[i];
        a.ig2[i] = (float)(1.0 / (c->g[i] * c->g[i]));
    }
    a.boxA = useA ? c->boxA : nullptr;
    a.gA = *c->bcur;
    a.sA = (float)sA;
    a.boxB = useB ? c->boxB : nullptr;
    a.gB = c->bB;
    a.sB = (float)sB;
    a.v = v;
    a.w = v ? c->curv_w : nullptr;
    a.sC = (float)sC;
    a.rpart = energy ? c->rpart : nullptr;
    a.out = out;
    a.dvec = v;
    a.dpart = v ? dpart : nullptr;
    a.skip = c->skip;
    if (v) LAUNCH(5, launch_curv(a, c->st));
    if (out) LAUNCH(6, launch_nodes(a, c->st));
    return RG_OK;
}

static int run_kp(rg_ctx *c, const float *u, const float *v, double scale, float *out, bool energy) {
    if (c->nk <= 0) return RG_OK;
    KpArgs k = kp_args(c);
    k.u = u;
    k.v = v;
    k.scale = (float)scale;
    k.out = out;
    k.part = energy ? c->kpart : nullptr;
    k.skip = c->skip;
    LAUNCH(7, launch_kp(k, c->st));
    if (out) LAUNCH(7, launch_kp_gather(k, c->st));
    return RG_OK;
}

static int run_terms(rg_ctx *c, double *terms, bool useD, bool useR, bool useV, bool useK, bool latch = true) {
    TermsArgs t;
    t.dpart = useD ? c->dpart : nullptr;
    t.nd = c->nD;
    t.dscale = c->hbar;
    t.rpart = useR ? c->rpart : nullptr;
    t.nr = c->nR;
    t.rscale = 0.5 * c->ghat;
    t.vpart = useV ? c->vpart : nullptr;
    t.nv = c->nB;
    t.vscale = c->ghat;
    t.fold = c->fold;
    t.kpart = (useK && c->nk > 0) ? c->kpart : nullptr;
    t.nkp = kp_blocks(c->nk);
    t.alpha = c->P.alpha;
    t.gamma = c->P.gamma;
    t.delta = c->P.delta;
    t.dmin = c->dmin;
    t.dmax = c->dmax;
    t.dminmax = c->dminmax;
    t.terms = terms;
    t.nonfinite = latch ? c->tma_err + 2 : nullptr;
    t.skip = c->skip;
    LAUNCH(8, launch_terms(t, c->st));
    return RG_OK;
}

// The extremes of the Jacobian bounds d of Eq. (8) at u into dminmax (a
// volume-term pass of its own, for when the objective does not evaluate it).
static int run_range(rg_ctx *c, const float *u) {
    int st;
    if ((st = run_vcc(c, u, nullptr))) return st;
    return run_terms(c, c->range_terms, false, false, true, false, false);
}

// Objective (and gradient) of Eq. (11).
static int evaluate(rg_ctx *c, const float *u, double *terms, float *grad, bool store_lin) {
    int mode = grad ? (store_lin ? MODE_GRADLIN : MODE_GRAD) : (store_lin ? MODE_LIN : MODE_OBJ);
    int st;
    if ((st = run_tile(c, mode, u))) return st;
    const bool vcc = c->P.gamma != 0.0;
    if (vcc && (st = run_vcc(c, u, nullptr))) return st;
    if ((st = run_nodes(c, u, true, grad, c->hbar, c->P.gamma * c->ghat, c->P.alpha * c->ghat, true, vcc))) return st;
    if ((st = run_kp(c, u, nullptr, c->P.delta, grad, true))) return st;
    if ((st = run_terms(c, terms ? terms : c->terms_tmp, true, true, vcc, true))) return st;
    if (store_lin) {
        CK(cudaMemcpyAsync(c->lin_u, u, sizeof(float) * 3 * c->M, cudaMemcpyDeviceToDevice, c->st));
        c->has_lin = true;
        c->minv_valid = false;
    }
    return RG_OK;
}

extern "C" int ngf_objective(rg_ctx *c, const float *u, double *terms) {
    if (!c || !u || !terms) return set_err(c, RG_EINVAL, "ngf_objective: NULL argument");
    return evaluate(c, u, terms, nullptr, false);
}

extern "C" int ngf_gradient(rg_ctx *c, const float *u, double *terms, float *grad) {
    if (!c || !u || !grad) return set_err(c, RG_EINVAL, "ngf_gradient: NULL argument");
    return evaluate(c, u, terms, grad, false);
}

extern "C" int gn_linearize(rg_ctx *c, const float *u, double *terms, float *grad) {
    if (!c || !u) return set_err(c, RG_EINVAL, "gn_linearize: NULL argument");
    return evaluate(c, u, terms, grad, true);
}

// H v; with dpart, also the per-block partials of v . H v when the node pass
// forms H v completely (no keypoint term after it): *ndpart is their count,
// else 0.
static int matvec(rg_ctx *c, const float *v, float *Hv, double *dpart = nullptr, int *ndpart = nullptr) {
    int st;
    if ((st = run_tile(c, MODE_MATVEC, v))) return st;
    const bool vcc = c->P.gamma != 0.0;
    if (vcc && (st = run_vcc(c, c->lin_u, v))) return st;
    const bool dq = dpart && c->nk <= 0;
    if (ndpart) *ndpart = dq ? c->nR : 0;
    if ((st = run_nodes(c, v, false, Hv, c->hbar, c->P.gamma * c->ghat, c->P.alpha * c->ghat, true, vcc,
                        dq ? dpart : nullptr)))
        return st;
    if ((st = run_kp(c, c->lin_u, v, c->P.delta, Hv, false))) return st;
    return RG_OK;
}

extern "C" int gn_matvec(rg_ctx *c, const float *v, float *Hv) {
    if (!c || !v || !Hv) return set_err(c, RG_EINVAL, "gn_matvec: NULL argument");
    if (!c->has_lin) return set_err(c, RG_EINVAL, "gn_matvec: no linearisation (call gn_linearize first)");
    return matvec(c, v, Hv);
}

extern "C" int regularizer_apply(rg_ctx *c, int32_t which, const float *u, const float *v, double *energy,
                                 float *out) {
    if (!c || !u || !out) return set_err(c, RG_EINVAL, "regularizer_apply: NULL argument");
    int st;
    if (which == RG_CURV) {
        if (v) {
            if ((st = run_nodes(c, u, true, nullptr, 0, 0, 0, false, false))) return st;   // energy at u
            if (energy && (st = run_terms(c, c->terms_tmp, false, true, false, false))) return st;
            if ((st = run_nodes(c, v, false, out, 0, 0, c->ghat, false, false))) return st;
        } else {
            if ((st = run_nodes(c, u, true, out, 0, 0, c->ghat, false, false))) return st;
            if (energy && (st = run_terms(c, c->terms_tmp, false, true, false, false))) return st;
        }
        if (energy) CK(cudaMemcpyAsync(energy, c->terms_tmp + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    } else if (which == RG_VCC) {
        if (v) {
            if ((st = run_vcc(c, u, nullptr))) return st;   // energy at u
            if (energy && (st = run_terms(c, c->terms_tmp, false, false, true, false))) return st;
            if ((st = run_vcc(c, u, v))) return st;
        } else {
            if ((st = run_vcc(c, u, nullptr))) return st;
            if (energy && (st = run_terms(c, c->terms_tmp, false, false, true, false))) return st;
        }
        if ((st = run_nodes(c, nullptr, false, out, 0, c->ghat, 0, false, true))) return st;
        if (energy) CK(cudaMemcpyAsync(energy, c->terms_tmp + 2, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    } else if (which == RG_KP) {
        CK(cudaMemsetAsync(out, 0, sizeof(float) * 3 * c->M, c->st));
        if (c->nk > 0) {
            KpArgs k = kp_args(c);
            k.u = u; k.v = v; k.scale = 1.f; k.out = out; k.part = c->kpart;
            LAUNCH(7, launch_kp(k, c->st));
            LAUNCH(7, launch_kp_gather(k, c->st));
        }
        if (energy) {
            if ((st = run_terms(c, c->terms_tmp, false, false, false, true))) return st;
            CK(cudaMemcpyAsync(energy, c->terms_tmp + 3, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        }
    } else {
        return set_err(c, RG_EINVAL, "regularizer_apply: unknown term %d", which);
    }
    return RG_OK;
}

// Jacobi preconditioner at the stored linearisation: NGF diagonal without
// the cross terms of the central-difference adjoint, exact curvature, VCC and
// keypoint diagonals, plus tau; reciprocal stored in minv.
static int ensure_minv(rg_ctx *c) {
    if (c->minv_valid) return RG_OK;
    int st;
    if ((st = run_tile(c, MODE_DIAG, c->lin_u))) return st;
    const bool vcc = c->P.gamma != 0.0;
    if (vcc && (st = run_vcc(c, c->lin_u, nullptr, 1))) return st;
    if ((st = run_nodes(c, nullptr, false, c->minv, 2.0 * c->hbar, c->P.gamma * c->ghat, 0.0, true, vcc))) return st;
    float ig2[3];
    for (int i = 0; i < 3; ++i) ig2[i] = (float)(1.0 / (c->g[i] * c->g[i]));
    LAUNCH(10, launch_jacobi_diag(1, c->grid.m, ig2, c->P.alpha * c->ghat, c->P.tau, c->minv, c->st));
    if (c->nk > 0 && c->P.delta != 0.0) LAUNCH(10, launch_kp_diag(kp_args(c), 2.0 * c->P.delta, c->minv, c->st));
    LAUNCH(10, launch_invert(3 * c->M, c->minv, c->st));
    c->minv_valid = true;
    return RG_OK;
}

__global__ void pcg_stats_kernel(const PcgScalars *sc, double *stats) {
    stats[0] = sc->steps;
    stats[1] = sc->r0;
    stats[2] = sc->rend;
}

// The PCG's operands and vectors in the context's workspace.
static PcgArgs pcg_args(rg_ctx *c) {
    PcgArgs a;
    a.n = 3 * c->M;
    a.stride = pcg_stride(a.n);
    a.minv = c->minv;
    a.Rh = c->Rh;
    a.d = c->d;
    a.part = c->pcgpart;
    a.rzpart = c->rzpart;
    a.apart = c->apart;
    a.ticket = reinterpret_cast<unsigned *>(c->tma_err + 1);
    a.sc = c->sc;
    a.rzh = c->rzh;
    return a;
}

// PCG set-up: the preconditioner (when stale) and the start vectors.
static int pcg_prepare(rg_ctx *c, const float *g, float *p, int iters) {
    if (iters > c->pcg_max)
        return set_err(c, RG_EINVAL, "PCG: %d steps requested, the workspace holds %d (pcg_max)", iters, c->pcg_max);
    if (((uintptr_t)g | (uintptr_t)p) & 15)
        return set_err(c, RG_EINVAL, "PCG: g and p must be 16-byte aligned");
    int st;
    if ((st = ensure_minv(c))) return st;
    if (!c->err_zeroed) {
        CK(cudaMemsetAsync(c->tma_err, 0, 4 * sizeof(int), c->st));
        c->err_zeroed = true;
    }
    LAUNCH(9, launch_pcg_start(pcg_args(c), g, p, c->st));
    return RG_OK;
}

// PCG wrap-up: the final residual norm and the statistics.
static int pcg_finish(rg_ctx *c, double *stats) {
    const PcgArgs a = pcg_args(c);
    const int nb = vec_blocks(a.n);
    LAUNCH(9, launch_dot_slot(a.n, c->Rh, a.stride, c->sc, c->vecpart, c->st));
    LAUNCH(9, launch_pcg_scalar(4, c->vecpart, nb, c->sc, c->st));
    if (stats) {
        ProfScope ps_(c, 9);
        pcg_stats_kernel<<<1, 1, 0, c->st>>>(c->sc, stats);
        CK(cudaGetLastError());
    }
    return RG_OK;
}

// PCG with full reorthogonalisation (classical Gram-Schmidt of each new
// residual against all earlier ones in the preconditioner's inner product);
// same iterates as plain PCG in exact arithmetic, kept so in FP32.  Scalars,
// dots and coefficients in FP64.
static int pcg(rg_ctx *c, const float *g, float *p, int iters, double *stats) {
    int st;
    if ((st = pcg_prepare(c, g, p, iters))) return st;
    const PcgArgs a = pcg_args(c);
    for (int k = 0; k < iters; ++k) {
        int napart = 0;   // d.q partials: from the node pass, else from the alpha kernel
        if ((st = matvec(c, c->d, c->q, c->apart, &napart))) return st;
        if (!napart) LAUNCH(9, launch_pcg_alpha(a, c->q, &napart, c->st));
        LAUNCH(9, launch_pcg_step(a, c->q, napart, k, c->st));
        LAUNCH(9, launch_pcg_reorth(a, k, c->st));
        LAUNCH(9, launch_pcg_dir(a, p, k, c->st));
    }
    return pcg_finish(c, stats);
}

// Whether the persistent batched PCG (pcg_batch.cu) can take this context's
// PCG steps: the column GN-product kernel covers its volume and H has no
// keypoint term (its node sums use atomics outside the node pass).
static bool batch_pcg_ok(const rg_ctx *c) { return !c->general_only && c->nk <= 0 && pcg_batch_supported(c->cg); }

// The operands of one PCG step of the context (the GN product H d into q as
// matvec forms it, the vectors of pcg), with s the PCG iterate.
static void batch_pair(rg_ctx *c, float *s, BatchPair &b) {
    ColArgs &a = b.col;
    a = ColArgs();
    a.g = c->cg;
    a.v = c->d;
    a.boxes = c->boxA;
    a.map_dT = c->map_col_dT;
    a.map_a = c->map_col_a;
    a.err = c->tma_err;
    a.skip = nullptr;
    a.poll_limit = c->hook_poll;
    a.no_tma = c->hook_no_tma;
    const bool vcc = c->P.gamma != 0.0;
    VccArgs &v = b.vcc;
    v = VccArgs();
    v.diag = 0;
    for (int i = 0; i < 3; ++i) {
        v.m[i] = c->grid.m[i];
        v.ig[i] = (float)(1.0 / c->g[i]);
        v.nb[i] = c->bB.nb[i];
    }
    v.box = c->bB.box;
    v.u = c->lin_u;
    v.v = c->d;
    v.wscale = 1.f;
    v.boxes = c->boxB;
    v.epart = c->vpart;
    v.fold = c->fold;
    v.dmin = c->dmin;
    v.dmax = c->dmax;
    NodeArgs &n = b.nodes;
    n = NodeArgs();
    for (int i = 0; i < 3; ++i) {
        n.m[i] = c->grid.m[i];
        n.ig2[i] = (float)(1.0 / (c->g[i] * c->g[i]));
    }
    n.boxA = c->boxA;
    n.gA = c->bM;
    n.sA = (float)c->hbar;
    n.boxB = vcc ? c->boxB : nullptr;
    n.gB = c->bB;
    n.sB = (float)(c->P.gamma * c->ghat);
    n.v = c->d;
    n.w = c->curv_w;
    n.sC = (float)(c->P.alpha * c->ghat);
    n.rpart = nullptr;
    n.out = c->q;
    n.dvec = c->d;
    n.dpart = c->apart;
    b.pcg = pcg_args(c);
    b.s = s;
    b.vcc_on = vcc ? 1 : 0;
}

extern "C" int gn_pcg_solve(rg_ctx *c, const float *g, float *p, int32_t iters, double *stats) {
    if (!c || !g || !p || iters < 0) return set_err(c, RG_EINVAL, "gn_pcg_solve: bad argument");
    if (!c->has_lin) return set_err(c, RG_EINVAL, "gn_pcg_solve: no linearisation (call gn_linearize first)");
    return pcg(c, g, p, iters, stats);
}

static int read_terms(rg_ctx *c, double *terms_dev, double *host5, double *dm2 = nullptr) {
    int err = 0;
    CK(cudaMemcpyAsync(host5, terms_dev, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (dm2) CK(cudaMemcpyAsync(dm2, c->dminmax, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(&err, c->tma_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (err) return set_err(c, RG_ETIMEOUT, "a kernel gave up waiting for a TMA transfer");
    return RG_OK;
}

static int set_delta_adaptive(rg_ctx *c, const float *u) {
    // delta such that D = delta K at the start (Sec. II-D2)
    int st;
    double h5[5];
    rg_params P = c->P;
    c->P.delta = 1.0;
    if ((st = evaluate(c, u, c->terms_tmp, nullptr, false))) return st;
    if ((st = read_terms(c, c->terms_tmp, h5))) return st;
    P.delta = (c->nk > 0 && h5[3] > 0.0) ? h5[0] / h5[3] : 0.0;
    c->P = P;
    c->minv_valid = false;
    return RG_OK;
}

// ------------------------------------------------ device-driven schedule
// The same iteration as gn_solve_impl's host loop with the decisions taken on
// the GPU (gn_loop.cu): every line-search try is launched, and the tries after
// the accepted one skip all their work.
struct SkipScope {
    rg_ctx *c;
    SkipScope(rg_ctx *c_, const int *flag) : c(c_) { c->skip = flag; }
    ~SkipScope() { c->skip = nullptr; }
};

struct StreamSwap {   // the context's launches go to another stream for a scope
    rg_ctx *c;
    cudaStream_t saved;
    StreamSwap(rg_ctx *c_, cudaStream_t s) : c(c_), saved(c_->st) { c->st = s; }
    ~StreamSwap() { c->st = saved; }
};

// part: 0 the whole iteration; 1 up to the PCG start, 2 from the PCG
// wrap-up on (the PCG steps in between run elsewhere: the persistent batched
// PCG of register_pyramid_batch)
static int gn_iteration_device(rg_ctx *c, float *u, const rg_schedule *s, int part = 0) {
    int st;
    const long n = 3 * c->M;
    if (part != 2) {
        if ((st = evaluate(c, u, c->terms_tmp, c->tg_, true))) return st;
        LAUNCH(9, launch_gn_begin(c->gn, c->terms_tmp, c->dminmax, c->st));
        if (part == 1) return pcg_prepare(c, c->tg_, c->ts, s->pcg_iters);
        if ((st = pcg(c, c->tg_, c->ts, s->pcg_iters, c->terms_tmp + 5))) return st;
    } else {
        if ((st = pcg_finish(c, c->terms_tmp + 5))) return st;
    }
    LAUNCH(9, launch_dot(n, c->tg_, c->ts, c->vecpart, c->st));
    LAUNCH(9, launch_gn_slope(c->gn, c->vecpart, vec_blocks(n), c->st));
    {
        SkipScope sk(c, &c->gn->done);
        double t = 1.0;
        for (int k = 0; k <= s->ls_max; ++k) {
            LAUNCH(9, launch_axpy_copy(n, (float)t, u, c->ts, c->tu, c->st, c->skip));
            if ((st = evaluate(c, c->tu, c->terms_tmp, nullptr, false))) return st;
            LAUNCH(9, launch_gn_armijo(c->gn, c->terms_tmp, c->dminmax, t, s->armijo_c, c->st));
            t *= 0.5;
        }
    }
    LAUNCH(9, launch_gn_accept(c->gn, n, c->tu, u, c->st));
    if (c->P.gamma == 0.0) {   // the objective left the volume term out: a range pass at the new iterate
        if ((st = run_range(c, u))) return st;
        LAUNCH(9, launch_gn_range(c->gn, c->dminmax, c->st));
    }
    LAUNCH(9, launch_gn_report(c->gn, c->terms_tmp + 5, c->gnrep, kGnRows, c->P.det_lo, c->P.det_hi, c->st));
    return RG_OK;
}

// gn_iters iterations on c->st: launched one by one, or captured once into a
// CUDA graph and replayed (the iteration's launches and pointers do not
// change between iterations)
static int gn_run_device(rg_ctx *c, float *u, const rg_schedule *s, bool graph) {
    if (!c->err_zeroed) {
        CK(cudaMemsetAsync(c->tma_err, 0, 4 * sizeof(int), c->st));
        c->err_zeroed = true;
    }
    CK(cudaMemsetAsync(c->gn, 0, sizeof(GnState), c->st));
    if (!graph) {
        for (int it = 0; it < s->gn_iters; ++it) {
            const int st = gn_iteration_device(c, u, s);
            if (st) return st;
        }
        return RG_OK;
    }
    cudaGraph_t g = nullptr;
    const long long l0 = c->launches;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed));
    const int st = gn_iteration_device(c, u, s);
    const cudaError_t ce = cudaStreamEndCapture(c->st, &g);
    const long long per = c->launches - l0;   // counted while capturing; nothing ran yet
    c->launches -= per;
    g_launches.fetch_sub(per, std::memory_order_relaxed);
    if (st != RG_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != RG_OK ? st : set_err(c, RG_ECUDA, "gn_solve: capture failed: %s", cudaGetErrorString(ce));
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return set_err(c, RG_ECUDA, "gn_solve: graph instantiation: %s", cudaGetErrorString(ie));
    int rc = RG_OK;
    for (int it = 0; it < s->gn_iters; ++it) {
        const cudaError_t le = cudaGraphLaunch(ge, c->st);
        if (le != cudaSuccess) {
            rc = set_err(c, RG_ECUDA, "gn_solve: graph launch: %s", cudaGetErrorString(le));
            break;
        }
        c->launches += per;
        g_launches.fetch_add(per, std::memory_order_relaxed);
    }
    cudaGraphExecDestroy(ge);
    return rc;
}

// Device-driven schedule on the context's private stream, ordered after and
// before the caller's stream by events; one host synchronisation at the end.
static int ensure_private_stream(rg_ctx *c) {
    if (c->gst) return RG_OK;
    cudaStream_t gs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaStreamDestroy(gs);
        return set_err(c, RG_ECUDA, "gn_solve: event creation failed");
    }
    c->gst = gs;
    c->gev[0] = e0;
    c->gev[1] = e1;
    return RG_OK;
}

static int gn_solve_device(rg_ctx *c, float *u, const rg_schedule *s, double *report, bool graph) {
    int est;
    if ((est = ensure_private_stream(c))) return est;
    const cudaStream_t user = c->st;
    CK(cudaEventRecord(c->gev[0], user));
    CK(cudaStreamWaitEvent(c->gst, c->gev[0], 0));
    int st;
    {
        StreamSwap sw(c, c->gst);
        st = gn_run_device(c, u, s, graph);
    }
    CK(cudaEventRecord(c->gev[1], c->gst));
    CK(cudaStreamWaitEvent(user, c->gev[1], 0));
    if (st) return st;
    GnState hs;
    std::vector<double> rows(RG_REPORT_COLS * (size_t)s->gn_iters);
    int err = 0;
    CK(cudaMemcpyAsync(&hs, c->gn, sizeof hs, cudaMemcpyDeviceToHost, c->gst));
    CK(cudaMemcpyAsync(rows.data(), c->gnrep, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost, c->gst));
    CK(cudaMemcpyAsync(&err, c->tma_err, sizeof(int), cudaMemcpyDeviceToHost, c->gst));
    CK(cudaStreamSynchronize(c->gst));
    if (err) return set_err(c, RG_ETIMEOUT, "a kernel gave up waiting for a TMA transfer");
    const int nrows = hs.halted ? hs.halt_it + 1 : s->gn_iters;
    if (report) memcpy(report, rows.data(), sizeof(double) * RG_REPORT_COLS * (size_t)nrows);
    if (hs.halted)
        return hs.status == RG_EFOLD ? set_err(c, RG_EFOLD, "gn_solve: fold at the current iterate")
                                     : set_err(c, RG_ENONFINITE, "gn_solve: non-finite objective");
    return RG_OK;
}

static int gn_solve_impl(rg_ctx *c, float *u, const rg_schedule *s, double *report, bool adapt) {
    int st;
    if (adapt && (st = set_delta_adaptive(c, u))) return st;
    if ((s->flags & RG_SCHED_AUTOTUNE) && (st = rg_autotune(c, u, nullptr, nullptr))) return st;
    if ((s->flags & (RG_SCHED_DEVICE | RG_SCHED_GRAPH)) && s->gn_iters > 0 && s->gn_iters <= kGnRows && !c->prof)
        return gn_solve_device(c, u, s, report, (s->flags & RG_SCHED_GRAPH) != 0);
    const long n = 3 * c->M;
    double h5[5], slope, dm0[2], dm[2];
    for (int it = 0; it < s->gn_iters; ++it) {
        double *rep = report ? report + RG_REPORT_COLS * it : nullptr;
        if (rep)
            for (int k = 0; k < RG_REPORT_COLS; ++k) rep[k] = 0.0;
        if ((st = evaluate(c, u, c->terms_tmp, c->tg_, true))) return st;
        if ((st = read_terms(c, c->terms_tmp, h5, dm0))) return st;
        const double J0 = h5[4];
        if (!isfinite(J0)) {
            if (rep) { rep[0] = it; rep[1] = J0; rep[7] = isinf(J0) ? RG_EFOLD : RG_ENONFINITE; }
            return isinf(J0) ? set_err(c, RG_EFOLD, "gn_solve: fold at the current iterate")
                             : set_err(c, RG_ENONFINITE, "gn_solve: non-finite objective");
        }
        if ((st = pcg(c, c->tg_, c->ts, s->pcg_iters, c->terms_tmp + 5))) return st;
        // slope g.p, summed on the host in a fixed order from the FP64 partials
        LAUNCH(9, launch_dot(n, c->tg_, c->ts, c->vecpart, c->st));
        {
            const int nbv = vec_blocks(n);
            double hp[152 * 8], pst[3];
            CK(cudaMemcpyAsync(hp, c->vecpart, sizeof(double) * nbv, cudaMemcpyDeviceToHost, c->st));
            CK(cudaMemcpyAsync(pst, c->terms_tmp + 5, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            slope = 0.0;
            for (int i = 0; i < nbv; ++i) slope += hp[i];
            if (rep) rep[6] = pst[0];
        }
        double t = 1.0, acc_t = 0.0, Jn = J0;
        int evals = 0;
        for (int k = 0; k <= s->ls_max; ++k) {
            LAUNCH(9, launch_axpy_copy(n, (float)t, u, c->ts, c->tu, c->st));
            if ((st = evaluate(c, c->tu, c->terms_tmp, nullptr, false))) return st;
            if ((st = read_terms(c, c->terms_tmp, h5, dm))) return st;
            ++evals;
            if (isfinite(h5[4]) && h5[4] <= std::fma(s->armijo_c * t, slope, J0)) {
                acc_t = t;
                Jn = h5[4];
                dm0[0] = dm[0];
                dm0[1] = dm[1];
                break;
            }
            t *= 0.5;
        }
        if (acc_t > 0.0) CK(cudaMemcpyAsync(u, c->tu, sizeof(float) * n, cudaMemcpyDeviceToDevice, c->st));
        if (rep) {
            if (c->P.gamma == 0.0) {   // the objective left the volume term out: a range pass at the new iterate
                if ((st = run_range(c, u))) return st;
                CK(cudaMemcpyAsync(dm0, c->dminmax, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
                CK(cudaStreamSynchronize(c->st));
            }
            rep[0] = it; rep[1] = J0; rep[2] = slope; rep[3] = acc_t; rep[4] = Jn; rep[5] = evals; rep[7] = 0;
            rep[8] = dm0[0]; rep[9] = dm0[1];
            rep[10] = (dm0[0] >= c->P.det_lo && dm0[1] <= c->P.det_hi) ? 1.0 : 0.0;
        }
    }
    CK(cudaStreamSynchronize(c->st));
    return RG_OK;
}

extern "C" int gn_solve(rg_ctx *c, float *u, const rg_schedule *s, double *report) {
    if (!c || !u || !s || s->gn_iters < 0 || s->pcg_iters < 0 || s->ls_max < 0)
        return set_err(c, RG_EINVAL, "gn_solve: bad argument");
    return gn_solve_impl(c, u, s, report, c->P.delta_adaptive != 0);
}

// ---------------------------------------------------------------- autotuner
// Tile shape and kernel family per problem geometry: 16-row tiles on the
// persistent kernels, 16-row tiles on the general column kernel, 8-row tiles
// on the general kernel.  Each is timed with CUDA events on the context's
// stream (one linearisation pass and three GN products after one untimed
// round) and scored as a Gauss-Newton iteration, gradient pass + 30 products.
// The choice is cached per process by geometry, image type and active terms.
namespace {
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;
}  // namespace

static TuneKey tune_key(const rg_ctx *c) {
    return TuneKey{c->img.n[0], c->img.n[1], c->img.n[2], c->grid.m[0], c->grid.m[1], c->grid.m[2], (int)c->dtype,
                   c->P.gamma != 0.0, c->nk > 0};
}

// general: 0 the specialised kernels with the objective / gradient pass by
// size, 1 the general tile kernels, 2 / 3 the specialised kernels with the
// column-marching / tile pass
static int apply_tile(rg_ctx *c, int ty, int general) {
    const int st = rg_set_tile(c, ty);
    if (st != RG_OK) return st;
    c->general_only = general == 1;
    c->pass_sel = general == 2 ? 1 : (general == 3 ? 2 : 0);
    c->has_lin = false;
    c->minv_valid = false;
    return RG_OK;
}

extern "C" int rg_autotune(rg_ctx *c, const float *u, int32_t *tile_y, int32_t *general) {
    if (!c || !u) return set_err(c, RG_EINVAL, "rg_autotune: NULL argument");
    if (!c->R || !c->T) return set_err(c, RG_EINVAL, "rg_autotune: images not set");
    const TuneKey key = tune_key(c);
    std::pair<int, int> best{16, 0};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        // the column-marching pass where it applies, the tile pass, the general kernels
        std::vector<std::pair<int, int>> cand;
        if (ngf_gcol_supported(c->cg)) cand.push_back({16, 2});
        cand.push_back({16, 3});
        cand.push_back({16, 1});
        cand.push_back({8, 1});
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        for (auto &x : e)
            if (cudaEventCreate(&x) != cudaSuccess) {
                for (auto y : e)
                    if (y) cudaEventDestroy(y);
                return set_err(c, RG_ECUDA, "rg_autotune: event creation failed");
            }
        double best_score = 1e300;
        int st = RG_OK;
        for (const auto &cd : cand) {
            if ((st = apply_tile(c, cd.first, cd.second))) break;
            float tg = 0.f, tm = 0.f;
            for (int round = 0; round < 2 && st == RG_OK; ++round) {
                if (cudaEventRecord(e[0], c->st) != cudaSuccess) st = set_err(c, RG_ECUDA, "rg_autotune: event");
                if (!st) st = evaluate(c, u, c->terms_tmp, c->tg_, true);
                if (!st && cudaEventRecord(e[1], c->st) != cudaSuccess) st = set_err(c, RG_ECUDA, "rg_autotune");
                for (int k = 0; k < 3 && !st; ++k) st = matvec(c, c->tg_, c->q);
                if (!st && cudaEventRecord(e[2], c->st) != cudaSuccess) st = set_err(c, RG_ECUDA, "rg_autotune");
                if (!st && cudaEventSynchronize(e[2]) != cudaSuccess) st = set_err(c, RG_ECUDA, "rg_autotune");
                if (!st) {
                    cudaEventElapsedTime(&tg, e[0], e[1]);
                    cudaEventElapsedTime(&tm, e[1], e[2]);
                }
            }
            if (st) break;
            const double score = tg + 30.0 * tm / 3.0;
            if (score < best_score) {
                best_score = score;
                best = cd;
            }
        }
        for (auto x : e) cudaEventDestroy(x);
        if (st) {
            apply_tile(c, 16, 0);
            return st;
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best;
    }
    int st = apply_tile(c, best.first, best.second);
    if (st) return st;
    if (tile_y) *tile_y = best.first;
    if (general) *general = best.second;
    return RG_OK;
}

// ---------------------------------------------------------------- pyramid
static void level_geom(const rg_image_geom *img, const rg_grid_geom *fin, int l, rg_image_geom &il, rg_grid_geom &gl) {
    for (int a = 0; a < 3; ++a) {
        il.n[a] = img->n[a] >> l;
        il.h[a] = img->h[a] * (double)(1 << l);
        gl.m[a] = ((fin->m[a] - 1) >> l) + 1;
    }
}

static int pyramid_check(const rg_image_geom *img, const rg_grid_geom *fin, int levels) {
    if (levels < 1 || levels > 8) return RG_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (img->n[a] % (1 << (levels - 1)) || (fin->m[a] - 1) % (1 << (levels - 1))) return RG_EINVAL;
    for (int l = 0; l < levels; ++l) {
        rg_image_geom il;
        rg_grid_geom gl;
        level_geom(img, fin, l, il, gl);
        if (check_geom(&il, &gl) != RG_OK) return RG_EINVAL;
    }
    return RG_OK;
}

extern "C" int rg_pyramid_workspace_size(const rg_image_geom *img, const rg_grid_geom *fin, rg_dtype dtype,
                                         int32_t levels, int32_t nk_max, int32_t pcg_max, size_t *bytes) {
    if (!bytes || pyramid_check(img, fin, levels) != RG_OK) return RG_EINVAL;
    size_t total = 0, es = dtype == RG_F16 ? 2 : 4;
    for (int l = 0; l < levels; ++l) {
        rg_image_geom il;
        rg_grid_geom gl;
        level_geom(img, fin, l, il, gl);
        size_t w;
        if (rg_workspace_size(&il, &gl, dtype, nk_max, pcg_max, &w) != RG_OK) return RG_EINVAL;
        total += w;
        long N = (long)il.n[0] * il.n[1] * il.n[2], M = (long)gl.m[0] * gl.m[1] * gl.m[2];
        if (l > 0) total += 2 * ((N * es + 255) & ~(size_t)255);
        total += (3 * M * sizeof(float) + 255) & ~(size_t)255;
    }
    *bytes = total;
    return RG_OK;
}

extern "C" int register_pyramid(const rg_image_geom *img, const void *R, const void *T, rg_dtype dtype,
                                const rg_grid_geom *fin, const rg_params *params, const rg_schedule *s, int32_t nk,
                                const float *kx, const float *ky, float *u_inout, double *report, void *ws,
                                size_t ws_bytes, void *stream) {
    if (!img || !R || !T || !fin || !params || !s || !u_inout || !ws || ((uintptr_t)ws & 255)) return RG_EINVAL;
    const int levels = s->levels;
    size_t need;
    if (rg_pyramid_workspace_size(img, fin, dtype, levels, nk, s->pcg_iters, &need) != RG_OK || ws_bytes < need)
        return RG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    rg_ctx *c = nullptr;   // for CK in this scope
    char *base = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t b) {
        off = (off + 255) & ~(size_t)255;
        char *p = base + off;
        off += b;
        return (void *)p;
    };
    const size_t es = dtype == RG_F16 ? 2 : 4;
    const void *Rl[8], *Tl[8];
    float *ul[8];
    rg_image_geom il[8];
    rg_grid_geom gl[8];
    Rl[0] = R;
    Tl[0] = T;
    for (int l = 0; l < levels; ++l) {
        level_geom(img, fin, l, il[l], gl[l]);
        long N = (long)il[l].n[0] * il[l].n[1] * il[l].n[2], M = (long)gl[l].m[0] * gl[l].m[1] * gl[l].m[2];
        if (l > 0) {
            void *r = take(N * es), *t = take(N * es);
            LAUNCH(10, launch_restrict(il[l - 1].n, dtype == RG_F16, Rl[l - 1], r, st));
            LAUNCH(10, launch_restrict(il[l - 1].n, dtype == RG_F16, Tl[l - 1], t, st));
            Rl[l] = r;
            Tl[l] = t;
        }
        ul[l] = (float *)take(3 * M * sizeof(float));
    }
    const int Lc = levels - 1;
    if (Lc == 0) CK(cudaMemcpyAsync(ul[0], u_inout, sizeof(float) * 3 * (long)fin->m[0] * fin->m[1] * fin->m[2],
                                    cudaMemcpyDeviceToDevice, st));
    else LAUNCH(10, launch_inject_grid(fin->m, 1 << Lc, u_inout, gl[Lc].m, ul[Lc], st));
    rg_params P = *params;
    int status = RG_OK;
    for (int l = Lc; l >= 0; --l) {
        size_t w;
        if (rg_workspace_size(&il[l], &gl[l], dtype, nk, s->pcg_iters, &w) != RG_OK) return RG_EINVAL;
        void *wl = take(w);
        rg_ctx *cl = nullptr;
        int e = rg_ctx_create(&cl, &il[l], &gl[l], dtype, &P, nk, s->pcg_iters, wl, w, stream);
        if (e != RG_OK) return e;
        e = rg_set_images(cl, Rl[l], Tl[l]);
        if (e == RG_OK && nk > 0) e = rg_set_keypoints(cl, nk, kx, ky);
        if (e != RG_OK) {
            rg_ctx_destroy(cl);
            return e;
        }
        status = gn_solve_impl(cl, ul[l], s, report ? report + (long)(Lc - l) * s->gn_iters * RG_REPORT_COLS : nullptr,
                               P.delta_adaptive != 0 && l == Lc);
        P.delta = cl->P.delta;
        rg_ctx_destroy(cl);
        if (status != RG_OK) return status;
        if (l > 0) LAUNCH(10, launch_prolong_grid(gl[l].m, ul[l], ul[l - 1], st));
    }
    CK(cudaMemcpyAsync(u_inout, ul[0], sizeof(float) * 3 * (long)fin->m[0] * fin->m[1] * fin->m[2],
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return status;
}

// Many pairs through the multilevel schedule in lockstep: at each level one
// CUDA graph holds every pair's device-driven Gauss-Newton iteration as a
// parallel branch (the context's private stream, forked from and joined to the
// caller's stream), and is replayed gn_iters times, so one graph launch
// advances all pairs.  Per pair the same kernels run in the same order as in
// register_pyramid with RG_SCHED_GRAPH.
extern "C" int register_pyramid_batch(int32_t npairs, const rg_image_geom *img, const void *const *R,
                                      const void *const *T, rg_dtype dtype, const rg_grid_geom *fin,
                                      const rg_params *params, const rg_schedule *s, float *const *u_inout,
                                      double *report, void *const *ws, const size_t *ws_bytes, void *stream) {
    if (npairs < 1 || !img || !R || !T || !fin || !params || !s || !u_inout || !ws || !ws_bytes) return RG_EINVAL;
    if (s->gn_iters < 1 || s->gn_iters > kGnRows || s->levels < 1 || s->levels > 8 || s->ls_max < 0)
        return RG_EINVAL;
    const int levels = s->levels, Lc = levels - 1;
    const bool persistent = (s->flags & RG_SCHED_PERSISTENT) && s->pcg_iters >= 1;
    const bool hook_barrier = (s->flags & RG_SCHED_HOOK_BARRIER) != 0;
    rg_ctx *c = nullptr;   // for CK / LAUNCH in this scope
    const size_t es = dtype == RG_F16 ? 2 : 4;
    struct Pair {
        char *base;
        size_t off;
        const void *Rl[8], *Tl[8];
        float *ul[8];
        rg_image_geom il[8];
        rg_grid_geom gl[8];
        rg_params P;
        rg_ctx *cl;
        void *take(size_t b) {
            off = (off + 255) & ~(size_t)255;
            char *p = base + off;
            off += b;
            return p;
        }
    };
    std::vector<Pair> ps(npairs);
    for (int p = 0; p < npairs; ++p) {
        size_t need;
        if (!R[p] || !T[p] || !u_inout[p] || !ws[p] || ((uintptr_t)ws[p] & 255) ||
            rg_pyramid_workspace_size(&img[p], &fin[p], dtype, levels, 0, s->pcg_iters, &need) != RG_OK ||
            ws_bytes[p] < need)
            return RG_EINVAL;
    }
    // all work on a private stream (a capture cannot run on the legacy default
    // stream), ordered after and, at the end, before the caller's stream
    const cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, edge = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&edge, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(edge, user) != cudaSuccess || cudaStreamWaitEvent(st, edge, 0) != cudaSuccess) {
        if (fork) cudaEventDestroy(fork);
        if (edge) cudaEventDestroy(edge);
        cudaStreamDestroy(st);
        return RG_ECUDA;
    }
    // join[p]: pair p's first branch; join[npairs + p]: its branch after the
    // persistent PCG launch; join[2 npairs]: the fork of those branches
    std::vector<cudaEvent_t> join(2 * npairs + 1, nullptr);
    for (auto &e : join)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
    auto release = [&]() {
        for (auto &q : ps)
            if (q.cl) {
                rg_ctx_destroy(q.cl);
                q.cl = nullptr;
            }
        for (auto e : join)
            if (e) cudaEventDestroy(e);
        cudaEventRecord(edge, st);   // the caller's stream continues after the batch
        cudaStreamWaitEvent(user, edge, 0);
        cudaStreamSynchronize(st);
        cudaEventDestroy(fork);
        cudaEventDestroy(edge);
        cudaStreamDestroy(st);
    };
    for (auto e : join)
        if (!e) {
            release();
            return RG_ECUDA;
        }
    int status = RG_OK;
    for (int p = 0; p < npairs && status == RG_OK; ++p) {
        Pair &q = ps[p];
        q.base = (char *)ws[p];
        q.off = 0;
        q.P = *params;
        q.cl = nullptr;
        q.Rl[0] = R[p];
        q.Tl[0] = T[p];
        for (int l = 0; l < levels; ++l) {
            level_geom(&img[p], &fin[p], l, q.il[l], q.gl[l]);
            const long N = (long)q.il[l].n[0] * q.il[l].n[1] * q.il[l].n[2];
            const long M = (long)q.gl[l].m[0] * q.gl[l].m[1] * q.gl[l].m[2];
            if (l > 0) {
                void *r = q.take(N * es), *t = q.take(N * es);
                if (launch_restrict(q.il[l - 1].n, dtype == RG_F16, q.Rl[l - 1], r, st) != cudaSuccess ||
                    launch_restrict(q.il[l - 1].n, dtype == RG_F16, q.Tl[l - 1], t, st) != cudaSuccess)
                    status = RG_ECUDA;
                g_launches.fetch_add(2, std::memory_order_relaxed);
                q.Rl[l] = r;
                q.Tl[l] = t;
            }
            q.ul[l] = (float *)q.take(3 * M * sizeof(float));
        }
        const long Mf = (long)fin[p].m[0] * fin[p].m[1] * fin[p].m[2];
        if (Lc == 0) {
            if (cudaMemcpyAsync(q.ul[0], u_inout[p], sizeof(float) * 3 * Mf, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
                status = RG_ECUDA;
        } else {
            if (launch_inject_grid(fin[p].m, 1 << Lc, u_inout[p], q.gl[Lc].m, q.ul[Lc], st) != cudaSuccess)
                status = RG_ECUDA;
            g_launches.fetch_add(1, std::memory_order_relaxed);
        }
    }
    // pairs whose schedule halted (fold or non-finite objective) leave the batch
    std::vector<int> halted(npairs, 0);
    if (report) memset(report, 0, sizeof(double) * (size_t)npairs * levels * s->gn_iters * RG_REPORT_COLS);
    std::vector<double> rows(RG_REPORT_COLS * (size_t)s->gn_iters);
    for (int l = Lc; l >= 0 && status == RG_OK; --l) {
        // this level's contexts (delta adapted on the host at the coarsest level)
        int nact = 0;
        for (int p = 0; p < npairs && status == RG_OK; ++p) {
            if (halted[p]) continue;
            ++nact;
            Pair &q = ps[p];
            size_t w = 0;
            if (rg_workspace_size(&q.il[l], &q.gl[l], dtype, 0, s->pcg_iters, &w) != RG_OK) {
                status = RG_EINVAL;
                break;
            }
            void *wl = q.take(w);
            status = rg_ctx_create(&q.cl, &q.il[l], &q.gl[l], dtype, &q.P, 0, s->pcg_iters, wl, w, (void *)st);
            if (status) break;
            rg_set_images(q.cl, q.Rl[l], q.Tl[l]);
            if (q.P.delta_adaptive && l == Lc) status = set_delta_adaptive(q.cl, q.ul[l]);
            if (!status) status = ensure_private_stream(q.cl);
            if (!status && cudaMemsetAsync(q.cl->tma_err, 0, 4 * sizeof(int), st) != cudaSuccess) status = RG_ECUDA;
            if (!status && cudaMemsetAsync(q.cl->gn, 0, sizeof(GnState), st) != cudaSuccess) status = RG_ECUDA;
            q.cl->err_zeroed = true;
        }
        if (status || nact == 0) break;
        // one graph: every active pair's iteration as a branch forked from st
        long long counted = 0;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            status = RG_ECUDA;
            break;
        }
        int cst = cudaEventRecord(fork, st) == cudaSuccess ? RG_OK : RG_ECUDA;
        // pairs whose PCG steps the persistent batched kernel takes (the rest
        // run their whole iteration in their branch)
        std::vector<int> pers;
        for (int p = 0; p < npairs && cst == RG_OK; ++p) {
            if (halted[p]) continue;
            rg_ctx *cl = ps[p].cl;
            const bool inp = persistent && batch_pcg_ok(cl);
            if (inp) pers.push_back(p);
            if (cudaStreamWaitEvent(cl->gst, fork, 0) != cudaSuccess) {
                cst = RG_ECUDA;
                break;
            }
            const long long l0 = cl->launches;
            {
                StreamSwap sw(cl, cl->gst);
                cst = gn_iteration_device(cl, ps[p].ul[l], s, inp ? 1 : 0);
            }
            counted += cl->launches - l0;
            cl->launches = l0;
            if (!cst && (cudaEventRecord(join[p], cl->gst) != cudaSuccess ||
                         cudaStreamWaitEvent(st, join[p], 0) != cudaSuccess))
                cst = RG_ECUDA;
        }
        if (!cst && !pers.empty()) {
            // every branch has joined: the cooperative launch has the GPU to itself
            for (size_t g0 = 0; g0 < pers.size() && !cst; g0 += kBatchMax) {
                const int ng = (int)std::min(pers.size() - g0, (size_t)kBatchMax);
                std::vector<BatchPair> bp(ng);
                for (int i = 0; i < ng; ++i) batch_pair(ps[pers[g0 + i]].cl, ps[pers[g0 + i]].cl->ts, bp[i]);
                unsigned *ctl = ps[pers[g0]].cl->bctl;
                if (cudaMemsetAsync(ctl, 0, sizeof(unsigned) * kBatchCtlWords, st) != cudaSuccess ||
                    launch_pcg_batch(bp.data(), ng, s->pcg_iters, ctl, hook_barrier ? (1 << 12) : (1 << 22),
                                     hook_barrier ? 1 : 0, st) != cudaSuccess)
                    cst = RG_ECUDA;
                counted += 1;
            }
            if (!cst && cudaEventRecord(join[2 * npairs], st) != cudaSuccess) cst = RG_ECUDA;
            for (size_t i = 0; i < pers.size() && !cst; ++i) {
                const int p = pers[i];
                rg_ctx *cl = ps[p].cl;
                if (cudaStreamWaitEvent(cl->gst, join[2 * npairs], 0) != cudaSuccess) {
                    cst = RG_ECUDA;
                    break;
                }
                const long long l0 = cl->launches;
                {
                    StreamSwap sw(cl, cl->gst);
                    cst = gn_iteration_device(cl, ps[p].ul[l], s, 2);
                }
                counted += cl->launches - l0;
                cl->launches = l0;
                if (!cst && (cudaEventRecord(join[npairs + p], cl->gst) != cudaSuccess ||
                             cudaStreamWaitEvent(st, join[npairs + p], 0) != cudaSuccess))
                    cst = RG_ECUDA;
            }
        }
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        g_launches.fetch_sub(counted, std::memory_order_relaxed);   // captured, not run
        if (cst || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            status = cst ? cst : RG_ECUDA;
            break;
        }
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            status = RG_ECUDA;
            break;
        }
        for (int it = 0; it < s->gn_iters && status == RG_OK; ++it) {
            if (cudaGraphLaunch(ge, st) != cudaSuccess) status = RG_ECUDA;
            else g_launches.fetch_add(counted, std::memory_order_relaxed);
        }
        cudaGraphExecDestroy(ge);
        if (status) break;
        // outcomes: one synchronisation for all pairs
        std::vector<GnState> hs(npairs);
        std::vector<double> rep((size_t)npairs * rows.size());
        std::vector<int> err(npairs, 0);
        for (int p = 0; p < npairs && status == RG_OK; ++p) {
            if (halted[p]) continue;
            rg_ctx *cl = ps[p].cl;
            if (cudaMemcpyAsync(&hs[p], cl->gn, sizeof(GnState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(rep.data() + (size_t)p * rows.size(), cl->gnrep, sizeof(double) * rows.size(),
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(&err[p], cl->tma_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
                status = RG_ECUDA;
        }
        if (!status && cudaStreamSynchronize(st) != cudaSuccess) status = RG_ECUDA;
        for (int p = 0; p < npairs && status == RG_OK; ++p) {
            if (halted[p]) continue;
            if (err[p]) {
                status = RG_ETIMEOUT;
                break;
            }
            const int nrows = hs[p].halted ? hs[p].halt_it + 1 : s->gn_iters;
            if (report)
                memcpy(report + ((size_t)p * levels + (Lc - l)) * s->gn_iters * RG_REPORT_COLS,
                       rep.data() + (size_t)p * rows.size(), sizeof(double) * RG_REPORT_COLS * (size_t)nrows);
            if (hs[p].halted) halted[p] = hs[p].status != 0 ? hs[p].status : RG_ENONFINITE;
        }
        for (int p = 0; p < npairs; ++p) {
            Pair &q = ps[p];
            if (!q.cl) continue;
            q.P.delta = q.cl->P.delta;
            rg_ctx_destroy(q.cl);
            q.cl = nullptr;
            if (!status && !halted[p] && l > 0) {
                if (launch_prolong_grid(q.gl[l].m, q.ul[l], q.ul[l - 1], st) != cudaSuccess) status = RG_ECUDA;
                else g_launches.fetch_add(1, std::memory_order_relaxed);
            }
        }
    }
    for (int p = 0; p < npairs && status == RG_OK; ++p) {
        if (halted[p]) continue;   // keeps its start value
        const long Mf = (long)fin[p].m[0] * fin[p].m[1] * fin[p].m[2];
        if (cudaMemcpyAsync(u_inout[p], ps[p].ul[0], sizeof(float) * 3 * Mf, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            status = RG_ECUDA;
    }
    if (status == RG_OK)
        for (int p = 0; p < npairs; ++p)
            if (halted[p]) {
                status = halted[p];
                break;
            }
    if (cudaStreamSynchronize(st) != cudaSuccess && !status) status = RG_ECUDA;
    release();
    return status;
}

extern "C" int rg_restrict_image(const int32_t *n, rg_dtype dtype, const void *in, void *out, void *stream) {
    if (!n || !in || !out || n[0] % 2 || n[1] % 2 || n[2] % 2) return RG_EINVAL;
    rg_ctx *c = nullptr;
    LAUNCH(10, launch_restrict(n, dtype == RG_F16, in, out, (cudaStream_t)stream));
    return RG_OK;
}

extern "C" int rg_prolong_grid(const int32_t *mc, const float *uc, float *uf, void *stream) {
    if (!mc || !uc || !uf) return RG_EINVAL;
    rg_ctx *c = nullptr;
    LAUNCH(10, launch_prolong_grid(mc, uc, uf, (cudaStream_t)stream));
    return RG_OK;
}

extern "C" int rg_sync(rg_ctx *c) {
    if (!c) return RG_EINVAL;
    CK(cudaStreamSynchronize(c->st));
    if (!c->err_zeroed) return RG_OK;   // nothing launched yet
    int f[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(f, c->tma_err, sizeof f, cudaMemcpyDeviceToHost));
    if (!f[0] && !f[2]) return RG_OK;
    CK(cudaMemsetAsync(c->tma_err, 0, sizeof(int), c->st));
    CK(cudaMemsetAsync(c->tma_err + 2, 0, sizeof(int), c->st));
    CK(cudaStreamSynchronize(c->st));
    if (f[0]) return set_err(c, RG_ETIMEOUT, "a kernel gave up waiting for a TMA transfer");
    return set_err(c, RG_ENONFINITE, "an objective evaluated since the last check was not finite (NaN or Inf in the inputs)");
}

extern "C" int rg_debug_hook(rg_ctx *c, int32_t what, int32_t value) {
    if (!c) return RG_EINVAL;
    if (what == RG_HOOK_NO_TMA) c->hook_no_tma = value != 0;
    else if (what == RG_HOOK_POLL_LIMIT && value > 0) c->hook_poll = value;
    else if (what == RG_HOOK_PASS && value >= 0 && value <= 2) c->pass_sel = value;
    else return set_err(c, RG_EINVAL, "rg_debug_hook: unknown hook %d or bad value %d", what, value);
    return RG_OK;
}

extern "C" const char *rg_last_error(const rg_ctx *c) { return c ? c->err : "no context"; }

extern "C" const char *rg_version(void) { return "ngfreg 0.1 (sm_103a)"; }
