// w5ct_api.cu -- the C ABI of libw5ct (declared in include/w5ct.h): context,
// device memory, state transfer, the RK4 + CT step driver, reductions.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "w5ct.h"
#include "w5ct_adjoint.cuh"
#include "w5ct_fused.cuh"
#include "w5ct_internal.h"

using namespace w5ct;

namespace {
constexpr int kRedBlocks = 1024;     // partial-record count of the deterministic reductions
thread_local char g_create_err[512] = "no error";
}  // namespace

void w5ct::set_global_error(const char *text) { snprintf(g_create_err, sizeof(g_create_err), "%s", text); }

struct w5ct_ctx {
    w5ct_config cfg;
    cudaStream_t stream = nullptr;
    int nx = 0, ny = 0, nz = 0;
    long long n = 0;
    double dx = 0, dy = 0, dz = 0;
    bool have_grid = false, have_state = false;
    size_t real_size = 8;
    void *slab = nullptr;
    // FP64 state and accumulators
    double *q0 = nullptr;            // 5 contiguous planes
    double *b0 = nullptr;            // 3 contiguous planes
    double *acc = nullptr;           // 5 planes
    double *oacc = nullptr;          // 3 planes
    // arithmetic-type buffers (float or double)
    void *qs = nullptr, *bs = nullptr, *bc = nullptr;        // 5, 3, 3 planes
    void *q0r = nullptr, *b0r = nullptr;                     // q^n, b^n in float (aliases q0, b0 in FP64)
    void *Fx = nullptr, *Fy = nullptr, *Fz = nullptr;        // 5 planes each
    void *Sx = nullptr, *Sy = nullptr, *Sz = nullptr;        // 2 planes each
    // small device scalars
    double *dt_dev = nullptr;
    unsigned long long *smax = nullptr;
    int *flag = nullptr;
    unsigned long long *hits = nullptr;
    double *part = nullptr;          // kRedBlocks x 8
    double *red_out = nullptr;       // 8
    const double **planes = nullptr; // 8 device pointers
    // several patches (npatch > 1): planes hold the patches back to back
    int npatch = 0;
    std::vector<PatchGeom> pg;       // host copy of the patch table
    PatchGeom *pg_dev = nullptr;     // device patch table
    // sweep tiles: per axis, the patches' tiles grouped by tile variant
    // (segment [seg_off, seg_off + seg_n) of tiles_buf); pvar[axis][p] is
    // the variant of patch p
    std::vector<signed char> pvar[3];
    int4 *tiles_buf = nullptr;
    int seg_off[3][kMaxTileVariants] = {};
    int seg_n[3][kMaxTileVariants] = {};
    int sweep_t2[3] = {0, 0, 0};     // single patch: tile height of the sweep along each axis
    int schedule = 0;                // batched sweeps: 0 = one launch per axis and variant, 1 = persistent,
                                     // 2 = the whole step in one persistent launch (fused)
    // fused step (schedule 2): work items, per-patch targets and counters in one allocation
    void *fused_buf = nullptr;
    int4 *fused_items = nullptr;
    int nfused = 0;
    int *fused_ncb = nullptr, *fused_ntile = nullptr, *fused_done = nullptr, *fused_qa = nullptr;
    int4 *fused_check = nullptr;     // one-item list of w5ct_fused_wait_check
    int fused_blocks = 0;
    int fused_lag = 0;               // skew of the fused work list in patches (0: phase-major)
    int fused_group = 16;             // sweep tiles per work item of the fused step
    int pgrid[kMaxTileVariants] = {};   // resident blocks of the persistent sweep per variant
    int *pcounters = nullptr;        // work-queue counters: 4 stages x kMaxTileVariants
    long long sweep_units = 0;       // axis-sweeps covered by the timed event pairs
    int4 *cells_dev = nullptr;       // 256-cell blocks of every patch
    int ncells = 0;
    // adjoint work buffers (w5ct_adjoint_step): allocated on first use
    void *adj_slab = nullptr;
    // captured step (w5ct_step_graph)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;
    // timing and accounting
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    long long launches = 0;
    char err[512];
};

namespace {

// state, fluxes and every kernel in double (W5CT_FP64 and W5CT_FP64_DW)
inline bool ctx_fp64(const w5ct_ctx *c) { return c->cfg.precision != W5CT_FP32_BULK; }

int fail(w5ct_ctx *c, int code, const char *fmt, ...) {
    char *buf = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define W5_CUDA(c, call)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail((c), W5CT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename Real>
Phys<Real> make_phys(const w5ct_config &c) {
    Phys<Real> K;
    K.gamma = (Real)c.gamma;
    K.gm1 = (Real)(c.gamma - 1.0);
    K.g1 = (Real)(0.5 * (c.gamma - 1.0));
    K.g2 = (Real)((c.gamma - 2.0) / (c.gamma - 1.0));
    double ew = c.weno_variant == W5CT_WENO_JS ? c.eps_js : c.eps_z;
    double eb2 = c.eps_b * c.eps_b;
    if (sizeof(Real) == 4) {
        if (c.weno_variant != W5CT_WENO_JS && ew < 1e-30) ew = 1e-30;   // 1e-40 is subnormal in float
        if (eb2 < 1.17549435e-38) eb2 = 1.17549435e-38;
    }
    K.eps_w = (Real)ew;
    K.eps_b = (Real)c.eps_b;
    K.eps_b2 = (Real)eb2;
    K.rho_min = (Real)c.rho_min;
    K.p_min = (Real)c.p_min;
    // float eigenbasis bound: rounding amplification at most ~2^12 (a
    // relative error of 2.4e-4 in the projected fluxes of near-vacuum-pressure
    // interfaces); inactive wherever beta is above ~1e-3
    K.cs2_rel = sizeof(Real) == 4 ? (Real)(1.0 / 4096.0) : (Real)0;
    K.floors = c.floors;
    return K;
}

template <typename Real>
Real *plane(void *base, long long n, int f) {
    return reinterpret_cast<Real *>(base) + (size_t)f * (size_t)n;
}

void free_grid(w5ct_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->graph_kernels = 0;
    if (c->slab) cudaFree(c->slab);
    c->slab = nullptr;
    if (c->tiles_buf) cudaFree(c->tiles_buf);
    c->tiles_buf = nullptr;
    if (c->adj_slab) cudaFree(c->adj_slab);
    c->adj_slab = nullptr;
    if (c->fused_buf) cudaFree(c->fused_buf);
    c->fused_buf = nullptr;
    c->nfused = 0;
    for (int a = 0; a < 3; ++a) c->pvar[a].clear();
    c->have_grid = false;
    c->have_state = false;
    c->npatch = 0;
    c->pg.clear();
}

// geometry of patch p as the single-patch kernels see it
PatchGeom patch_of(const w5ct_ctx *c, int p) { return c->pg[p]; }

dim3 cell_grid(const w5ct_ctx *c) { return dim3((c->nx + 31) / 32, (c->ny + 7) / 8, c->nz); }

int n_variants(const w5ct_ctx *c) {
    return ctx_fp64(c) ? num_tile_variants<double>() : num_tile_variants<float>();
}

void variant_shape(const w5ct_ctx *c, int axis, int v, int &bx, int &t2) {
    if (ctx_fp64(c))
        tile_shape<double>(axis, v, bx, t2);
    else
        tile_shape<float>(axis, v, bx, t2);
}

// the tiles of patch p (geometry g) for a sweep along `axis` in tiles of
// bx lanes x t2 faces
void append_tiles(std::vector<int4> &out, int p, const PatchGeom &g, int axis, int bx, int t2) {
    const int nbx = (g.nx + bx - 1) / bx;
    const int tag = p | (axis << kItemAxisShift);
    if (axis == 0 || axis == 1) {
        for (int k = 0; k < g.nz; ++k)
            for (int j = 0; j < (g.ny + t2 - 1) / t2; ++j)
                for (int i = 0; i < nbx; ++i) out.push_back(make_int4(tag, i, j, k));
    } else {
        for (int k = 0; k < (g.nz + t2 - 1) / t2; ++k)
            for (int j = 0; j < g.ny; ++j)
                for (int i = 0; i < nbx; ++i) out.push_back(make_int4(tag, i, j, k));
    }
}

// Model of a tile variant's cost per useful face: lanes and rows padded to
// whole tiles, times the cell box's halo along the sweep axis (phase 1 is
// about a tenth of the per-face work).  The default choice before any
// measurement.
double tile_model_cost(const PatchGeom &g, int axis, int bx, int t2) {
    const int n2 = axis == 2 ? g.nz : g.ny;
    const double pad = (double)(((g.nx + bx - 1) / bx) * bx) / g.nx * (double)(((n2 + t2 - 1) / t2) * t2) / n2;
    const int len = axis == 0 ? bx : t2;
    return pad * (1.0 + 0.1 * (len + 5.0) / len);
}

void default_variants(w5ct_ctx *c) {
    const int nv = n_variants(c);
    for (int a = 0; a < 3; ++a) {
        c->pvar[a].assign(c->npatch, 0);
        for (int p = 0; p < c->npatch; ++p) {
            double best = 0;
            for (int v = 0; v < nv; ++v) {
                int bx, t2;
                variant_shape(c, a, v, bx, t2);
                const double cost = tile_model_cost(c->pg[p], a, bx, t2);
                if (v == 0 || cost < best * (1.0 - 1e-9)) {
                    best = cost;
                    c->pvar[a][p] = (signed char)v;
                }
            }
        }
    }
}

// (Re)build the device tile tables from pvar: per axis, the tiles of every
// patch grouped by variant.  Drops a captured step graph (it holds the old
// table).
int build_tiles(w5ct_ctx *c) {
    std::vector<int4> all;
    const int nv = n_variants(c);
    // variant-major, then axis: the three axes' tiles of one variant are
    // contiguous (the work list of the persistent sweep)
    for (int v = 0; v < kMaxTileVariants; ++v) {
        for (int a = 0; a < 3; ++a) {
            c->seg_off[a][v] = (int)all.size();
            if (v < nv) {
                int bx, t2;
                variant_shape(c, a, v, bx, t2);
                for (int p = 0; p < c->npatch; ++p)
                    if (c->pvar[a][p] == v) append_tiles(all, p, c->pg[p], a, bx, t2);
            }
            c->seg_n[a][v] = (int)all.size() - c->seg_off[a][v];
        }
    }
    if (all.size() > (size_t)0x7fffffff) return fail(c, W5CT_ERR_ARG, "too many sweep tiles");
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->tiles_buf || c->fused_buf) W5_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->tiles_buf) {
        cudaFree(c->tiles_buf);
        c->tiles_buf = nullptr;
    }
    // the fused step's work list follows the variants: rebuilt on next use
    if (c->fused_buf) {
        cudaFree(c->fused_buf);
        c->fused_buf = nullptr;
        c->nfused = 0;
    }
    W5_CUDA(c, cudaMalloc(&c->tiles_buf, sizeof(int4) * all.size()));
    W5_CUDA(c, cudaMemcpy(c->tiles_buf, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice));
    return W5CT_OK;
}

int record_event(w5ct_ctx *c) {
    if (!c->timing) return W5CT_OK;
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e;
        W5_CUDA(c, cudaEventCreate(&e));
        c->ev.push_back(e);
    }
    W5_CUDA(c, cudaEventRecord(c->ev[c->ev_used++], c->stream));
    return W5CT_OK;
}

template <typename Real>
int launch_cellb(w5ct_ctx *c) {
    const long long n = c->n;
    if (c->npatch > 1) {
        cellb_batched_kernel<Real><<<c->ncells, kCellBlock, 0, c->stream>>>(
            c->pg_dev, c->cells_dev, plane<Real>(c->bs, n, 0), plane<Real>(c->bs, n, 1), plane<Real>(c->bs, n, 2),
            plane<Real>(c->bc, n, 0), plane<Real>(c->bc, n, 1), plane<Real>(c->bc, n, 2));
    } else {
        cellb_kernel<Real><<<cellb_grid(c->nx, c->ny, c->nz), dim3(32, 8), 0, c->stream>>>(
            c->nx, c->ny, c->nz, cellb_chunk(c->nx, c->ny, c->nz), plane<Real>(c->bs, n, 0),
            plane<Real>(c->bs, n, 1), plane<Real>(c->bs, n, 2), plane<Real>(c->bc, n, 0), plane<Real>(c->bc, n, 1),
            plane<Real>(c->bc, n, 2));
    }
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return W5CT_OK;
}

// maxima S_d of every patch into smax[3 p + d]
template <typename Real>
int launch_speed(w5ct_ctx *c) {
    const long long n = c->n;
    W5_CUDA(c, cudaMemsetAsync(c->smax, 0, 3 * sizeof(unsigned long long) * (size_t)c->npatch, c->stream));
    if (c->npatch > 1) {
        speed_batched_kernel<Real><<<c->ncells, kCellBlock, 0, c->stream>>>(
            c->pg_dev, c->cells_dev, plane<Real>(c->qs, n, 0), plane<Real>(c->qs, n, 1), plane<Real>(c->qs, n, 2),
            plane<Real>(c->qs, n, 3), plane<Real>(c->qs, n, 4), plane<Real>(c->bc, n, 0), plane<Real>(c->bc, n, 1),
            plane<Real>(c->bc, n, 2), make_phys<Real>(c->cfg), c->smax, c->flag);
    } else {
        long long nb = (n + kRedThreads - 1) / kRedThreads;
        if (nb > 4 * 152) nb = 4 * 152;
        speed_kernel<Real><<<(unsigned)nb, kRedThreads, 0, c->stream>>>(
            n, c->nx, c->ny, plane<Real>(c->qs, n, 0), plane<Real>(c->qs, n, 1), plane<Real>(c->qs, n, 2),
            plane<Real>(c->qs, n, 3), plane<Real>(c->qs, n, 4), plane<Real>(c->bc, n, 0), plane<Real>(c->bc, n, 1),
            plane<Real>(c->bc, n, 2), make_phys<Real>(c->cfg), c->smax, c->flag);
    }
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return W5CT_OK;
}

// dt of every patch from the maxima (one launch)
int launch_dt(w5ct_ctx *c, double *dt_copy) {
    if (c->npatch > 1) {
        dt_batched_kernel<<<(c->npatch + 127) / 128, 128, 0, c->stream>>>(c->pg_dev, c->npatch, c->smax, c->cfg.cfl,
                                                                        c->dt_dev, dt_copy);
    } else {
        dt_kernel<<<1, 1, 0, c->stream>>>(c->smax, c->cfg.cfl, c->dx, c->dy, c->dz, c->dt_dev, dt_copy);
    }
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return W5CT_OK;
}

template <typename Real, int S>
void launch_update_stage(w5ct_ctx *c, const UpdateArgs<Real> &u) {
    if (c->npatch > 1)
        update_batched_kernel<Real, S><<<c->ncells, kCellBlock, 0, c->stream>>>(u, c->pg_dev, c->cells_dev, u.dt);
    else
        update_kernel<Real, S><<<cell_grid(c), dim3(32, 8), 0, c->stream>>>(u);
}

// The stage-update arguments of the context's buffers (dt from dt_dev).
template <typename Real>
UpdateArgs<Real> update_args(w5ct_ctx *c, const double *dt_dev) {
    const long long n = c->n;
    UpdateArgs<Real> u;
    u.nx = c->nx;
    u.ny = c->ny;
    u.nz = c->nz;
    u.rdx = (Real)(1.0 / c->dx);
    u.rdy = (Real)(1.0 / c->dy);
    u.rdz = (Real)(1.0 / c->dz);
    u.drdx = 1.0 / c->dx;
    u.drdy = 1.0 / c->dy;
    u.drdz = 1.0 / c->dz;
    for (int f = 0; f < 5; ++f) {
        u.Fx[f] = plane<Real>(c->Fx, n, f);
        u.Fy[f] = plane<Real>(c->Fy, n, f);
        u.Fz[f] = plane<Real>(c->Fz, n, f);
        u.q0[f] = c->q0 + (size_t)f * n;
        u.acc[f] = c->acc + (size_t)f * n;
        u.qs[f] = plane<Real>(c->qs, n, f);
        u.q0r[f] = plane<Real>(c->q0r, n, f);
    }
    for (int f = 0; f < 2; ++f) {
        u.Sx[f] = plane<Real>(c->Sx, n, f);
        u.Sy[f] = plane<Real>(c->Sy, n, f);
        u.Sz[f] = plane<Real>(c->Sz, n, f);
    }
    for (int f = 0; f < 3; ++f) {
        u.b0[f] = c->b0 + (size_t)f * n;
        u.oacc[f] = c->oacc + (size_t)f * n;
        u.bs[f] = plane<Real>(c->bs, n, f);
        u.b0r[f] = plane<Real>(c->b0r, n, f);
    }
    u.dt = dt_dev;
    return u;
}

// Work items of the fused step (see w5ct_fused.cuh), the per-patch targets
// and the counters, in one allocation; the resident-block count.
int build_fused(w5ct_ctx *c) {
    if (c->fused_buf) return W5CT_OK;
    std::vector<int4> items;
    std::vector<int> ncb(c->npatch), ntile(c->npatch, 0);
    const bool fp64 = ctx_fp64(c);
    for (int p = 0; p < c->npatch; ++p) {
        const PatchGeom &g = c->pg[p];
        ncb[p] = (int)(((long long)g.nx * g.ny * g.nz + kFusedCells - 1) / kFusedCells);
    }
    // The items of each (patch, phase) -- phases 5 s + {0: cell field, 1: CFL
    // blocks, 2: dt, 3: sweep tiles, 4: update} of stage s -- are ordered by
    // the key p + lag * phase (ties: the earlier phase first).  With lag >=
    // npatch this is phase-major (every patch's cell fields, then every
    // patch's sweeps, then every patch's updates); a smaller lag skews the
    // list so that the memory-bound updates and cell fields of some patches
    // run beside the sweeps of others.  Every dependency of an item (the same
    // patch, an earlier phase) has a smaller key and lies earlier in the
    // list, so the launch completes whatever the residency.
    struct Group {
        long long key;
        int phase, p;
        std::vector<int4> items;
    };
    std::vector<Group> groups;
    const long long lag = c->fused_lag > 0 ? c->fused_lag : c->npatch;
    auto group = [&](int p, int phase) -> std::vector<int4> & {
        groups.push_back(Group{(long long)p + lag * phase, phase, p, {}});
        return groups.back().items;
    };
    for (int st = 0; st < 4; ++st) {
        for (int p = 0; p < c->npatch; ++p) {
            const PatchGeom &g = c->pg[p];
            {
                std::vector<int4> &it = group(p, 5 * st + 0);
                for (int q = 0; q < ncb[p]; ++q) it.push_back(make_int4(p, fused_tag(FI_CELLB, st, 0, 0), q * kFusedCells, 0));
            }
            if (st == 0) {
                std::vector<int4> &it = group(p, 1);
                for (int q = 0; q < ncb[p]; ++q) it.push_back(make_int4(p, fused_tag(FI_SPEED, 0, 0, 0), q * kFusedCells, 0));
                group(p, 2).push_back(make_int4(p, fused_tag(FI_DT, 0, 0, 0), 0, 0));
            }
            // per axis: the tiles of one of the fused kernel's tile variants
            // (one tile per block; float: 32 x 8, 16 x 16, 8 x 16), the one
            // with the least padded lanes and rows and halo share by the
            // tile cost model, one tile per item
            std::vector<int4> &sw = group(p, 5 * st + 3);
            for (int a = 0; a < 3; ++a) {
                const int nfv = fp64 ? fused_variants<double>() : fused_variants<float>();
                int v = 0, bx = 0, t2 = 0;
                double best = 0;
                for (int w = 0; w < nfv; ++w) {
                    int bw, hw;
                    if (fp64)
                        fused_tile_shape<double>(w, bw, hw);
                    else
                        fused_tile_shape<float>(w, bw, hw);
                    const double cost = tile_model_cost(g, a, bw, hw);
                    if (w == 0 || cost < best * (1.0 - 1e-9)) {
                        best = cost;
                        v = w;
                        bx = bw;
                        t2 = hw;
                    }
                }
                const long long nbx = (g.nx + bx - 1) / bx;
                const long long nb1 = a == 2 ? g.ny : (g.ny + t2 - 1) / t2;
                const long long nb2 = a == 2 ? (g.nz + t2 - 1) / t2 : g.nz;
                const long long ntiles = nbx * nb1 * nb2;
                const long long grp = c->fused_group > 0 ? c->fused_group : 1;
                for (long long L = 0; L < ntiles; L += grp)
                    sw.push_back(make_int4(p, fused_tag(FI_SWEEP, st, a, v), (int)L, (int)std::min(grp, ntiles - L)));
            }
            if (st == 0) ntile[p] = (int)sw.size();
            std::vector<int4> &up = group(p, 5 * st + 4);
            for (int q = 0; q < ncb[p]; ++q) up.push_back(make_int4(p, fused_tag(FI_UPDATE, st, 0, 0), q * kFusedCells, 0));
        }
    }
    std::stable_sort(groups.begin(), groups.end(), [](const Group &x, const Group &y) {
        return x.key != y.key ? x.key < y.key : x.phase < y.phase;
    });
    for (const Group &gr : groups) items.insert(items.end(), gr.items.begin(), gr.items.end());
    if (items.size() > (size_t)0x7fffffff) return fail(c, W5CT_ERR_ARG, "too many work items for the fused step");
    const size_t P = (size_t)c->npatch;
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += align256(b); return o; };
    const size_t o_it = take(sizeof(int4) * items.size()), o_ncb = take(sizeof(int) * P), o_nt = take(sizeof(int) * P);
    const size_t o_done = take(sizeof(int) * 14 * P), o_qa = take(sizeof(int) * 2), o_chk = take(sizeof(int4));
    W5_CUDA(c, cudaMalloc(&c->fused_buf, bytes));
    char *b = (char *)c->fused_buf;
    c->fused_items = (int4 *)(b + o_it);
    c->fused_ncb = (int *)(b + o_ncb);
    c->fused_ntile = (int *)(b + o_nt);
    c->fused_done = (int *)(b + o_done);
    c->fused_qa = (int *)(b + o_qa);
    c->fused_check = (int4 *)(b + o_chk);
    c->nfused = (int)items.size();
    // the failure-path check's list: patch 0's first stage-0 update alone
    // (its sweep counter is never raised)
    const int4 chk = make_int4(0, fused_tag(FI_UPDATE, 0, 0, 0), 0, 0);
    W5_CUDA(c, cudaMemcpy(c->fused_check, &chk, sizeof(int4), cudaMemcpyHostToDevice));
    W5_CUDA(c, cudaMemcpy(c->fused_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    W5_CUDA(c, cudaMemcpy(c->fused_ncb, ncb.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    W5_CUDA(c, cudaMemcpy(c->fused_ntile, ntile.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    size_t smem = 0;
    const cudaError_t e = fp64 ? fused_grid<double>(c->cfg.weno_variant, c->fused_blocks, smem)
                               : fused_grid<float>(c->cfg.weno_variant, c->fused_blocks, smem);
    W5_CUDA(c, e);
    return W5CT_OK;
}

// Bound of a fused-step wait: 2^22 sleeps of 256 ns, about a second.
constexpr long long kFusedSpinLimit = 1LL << 22;

// One step of every patch in one persistent launch: dts given (device,
// npatch doubles) or, when dts_in is NULL, from each patch's CFL condition
// (copied to dts_out when not NULL).  `check`: run the one-item list of the
// failure-path check instead, waits bounded by spin_limit.
template <typename Real>
int fused_step_impl(w5ct_ctx *c, const double *dts_in, double *dts_out, bool check = false,
                    long long spin_limit = kFusedSpinLimit) {
    int rc = build_fused(c);
    if (rc) return rc;
    const long long n = c->n;
    cudaStream_t st = c->stream;
    const size_t P = (size_t)c->npatch;
    W5_CUDA(c, cudaMemsetAsync(c->fused_done, 0, sizeof(int) * 14 * P, st));
    W5_CUDA(c, cudaMemsetAsync(c->fused_qa, 0, sizeof(int) * 2, st));
    if (!dts_in) W5_CUDA(c, cudaMemsetAsync(c->smax, 0, 3 * sizeof(unsigned long long) * P, st));
    FusedArgs<Real> A;
    void *Fax[3] = {c->Fx, c->Fy, c->Fz};
    void *Sax[3] = {c->Sx, c->Sy, c->Sz};
    for (int ax = 0; ax < 3; ++ax) {
        SweepArgs<Real> &a = A.a[ax];
        a.nx = c->nx;
        a.ny = c->ny;
        a.nz = c->nz;
        for (int f = 0; f < 5; ++f) a.q[f] = plane<Real>(c->qs, n, f);
        for (int f = 0; f < 3; ++f) a.bc[f] = plane<Real>(c->bc, n, f);
        for (int f = 0; f < 5; ++f) a.F[f] = plane<Real>(Fax[ax], n, f);
        for (int f = 0; f < 2; ++f) a.S[f] = plane<Real>(Sax[ax], n, f);
        a.K = make_phys<Real>(c->cfg);
        a.flag = c->flag;
        a.hits = c->hits;
    }
    A.u = update_args<Real>(c, c->dt_dev);
    for (int f = 0; f < 3; ++f) {
        A.bs[f] = plane<Real>(c->bs, n, f);
        A.bc[f] = plane<Real>(c->bc, n, f);
    }
    A.pgs = c->pg_dev;
    A.items = check ? c->fused_check : c->fused_items;
    A.nitems = check ? 1 : c->nfused;
    A.ncb = c->fused_ncb;
    A.ntile = c->fused_ntile;
    A.ctr.queue = c->fused_qa;
    A.ctr.abort = c->fused_qa + 1;
    A.ctr.done = c->fused_done;
    A.ctr.npatch = c->npatch;
    A.cfl = dts_in ? 0 : 1;
    A.cfl_number = c->cfg.cfl;
    A.dts = dts_in ? const_cast<double *>(dts_in) : c->dt_dev;
    A.dts_out = dts_in ? nullptr : dts_out;
    A.smax = c->smax;
    A.spin_limit = spin_limit;
    int e0 = record_event(c);
    if (e0) return e0;
    W5_CUDA(c, launch_fused_step<Real>(c->cfg.weno_variant, A, c->fused_blocks, st));
    c->launches++;
    e0 = record_event(c);
    if (e0) return e0;
    if (c->timing) c->sweep_units += 12;
    return W5CT_OK;
}

int fused_step(w5ct_ctx *c, const double *dts_in, double *dts_out) {
    return ctx_fp64(c) ? fused_step_impl<double>(c, dts_in, dts_out)
                                         : fused_step_impl<float>(c, dts_in, dts_out);
}

// The three sweeps of a stage over every patch: schedule 0 launches one
// kernel per axis and tile variant; schedule 1 one persistent kernel per
// variant over the three axes' tiles, with the work-queue counters
// counters[v] (zero on entry).  Each timed group is bracketed by events.
template <typename Real>
int launch_batched_sweeps(w5ct_ctx *c, const SweepArgs<Real> (&a3)[3], int schedule, int *counters) {
    const int variant = c->cfg.weno_variant;
    if (schedule == 1) {
        int rc = record_event(c);
        if (rc) return rc;
        for (int v = 0; v < kMaxTileVariants; ++v) {
            const int first = c->seg_off[0][v], last = c->seg_off[2][v] + c->seg_n[2][v];
            if (last == first) continue;
            W5_CUDA(c, launch_sweep_persistent<Real>(variant, v, a3, c->pg_dev, c->tiles_buf + first, last - first,
                                                     counters + v, c->pgrid[v], c->stream));
            c->launches++;
        }
        rc = record_event(c);
        if (rc) return rc;
        if (c->timing) c->sweep_units += 3;
        return W5CT_OK;
    }
    for (int ax = 0; ax < 3; ++ax) {
        int rc = record_event(c);
        if (rc) return rc;
        for (int v = 0; v < kMaxTileVariants; ++v) {
            if (!c->seg_n[ax][v]) continue;
            W5_CUDA(c, launch_sweep_batched<Real>(ax, variant, v, a3[ax], c->pg_dev, c->tiles_buf + c->seg_off[ax][v],
                                                  c->seg_n[ax][v], c->stream));
            c->launches++;
        }
        rc = record_event(c);
        if (rc) return rc;
        if (c->timing) c->sweep_units += 1;
    }
    return W5CT_OK;
}

template <typename Real>
int run_step(w5ct_ctx *c, const double *dt_dev, bool cellb_done, int last_stage = 3, void *stage_store = nullptr) {
    const long long n = c->n;
    SweepArgs<Real> a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    for (int f = 0; f < 5; ++f) a.q[f] = plane<Real>(c->qs, n, f);
    for (int f = 0; f < 3; ++f) a.bc[f] = plane<Real>(c->bc, n, f);
    a.K = make_phys<Real>(c->cfg);
    a.flag = c->flag;
    a.hits = c->hits;
    a.dw = c->cfg.precision == W5CT_FP64_DW;

    const UpdateArgs<Real> u = update_args<Real>(c, dt_dev);

    void *Fax[3] = {c->Fx, c->Fy, c->Fz};
    void *Sax[3] = {c->Sx, c->Sy, c->Sz};
    const int variant = c->cfg.weno_variant;
    if (c->npatch > 1 && c->schedule == 1)
        W5_CUDA(c, cudaMemsetAsync(c->pcounters, 0, 4 * kMaxTileVariants * sizeof(int), c->stream));
    for (int s = 0; s < 4; ++s) {
        if (stage_store) {
            // the stage state (5 + 3 planes) before stage s, for the adjoint
            Real *dst = reinterpret_cast<Real *>(stage_store) + (size_t)s * 8 * (size_t)n;
            W5_CUDA(c, cudaMemcpyAsync(dst, c->qs, 5 * (size_t)n * sizeof(Real), cudaMemcpyDeviceToDevice, c->stream));
            W5_CUDA(c, cudaMemcpyAsync(dst + 5 * (size_t)n, c->bs, 3 * (size_t)n * sizeof(Real),
                                       cudaMemcpyDeviceToDevice, c->stream));
        }
        if (s > last_stage) break;
        if (!(s == 0 && cellb_done)) {
            int rc = launch_cellb<Real>(c);
            if (rc) return rc;
        }
        if (c->npatch > 1) {
            SweepArgs<Real> a3[3] = {a, a, a};
            for (int ax = 0; ax < 3; ++ax) {
                for (int f = 0; f < 5; ++f) a3[ax].F[f] = plane<Real>(Fax[ax], n, f);
                for (int f = 0; f < 2; ++f) a3[ax].S[f] = plane<Real>(Sax[ax], n, f);
            }
            int rc = launch_batched_sweeps<Real>(c, a3, c->schedule, c->pcounters + s * kMaxTileVariants);
            if (rc) return rc;
        } else {
            for (int ax = 0; ax < 3; ++ax) {
                for (int f = 0; f < 5; ++f) a.F[f] = plane<Real>(Fax[ax], n, f);
                for (int f = 0; f < 2; ++f) a.S[f] = plane<Real>(Sax[ax], n, f);
                int rc = record_event(c);
                if (rc) return rc;
                W5_CUDA(c, launch_sweep<Real>(ax, variant, c->sweep_t2[ax], a, c->stream));
                c->launches++;
                rc = record_event(c);
                if (rc) return rc;
                if (c->timing) c->sweep_units += 1;
            }
        }
        switch (s) {
            case 0: launch_update_stage<Real, 0>(c, u); break;
            case 1: launch_update_stage<Real, 1>(c, u); break;
            case 2: launch_update_stage<Real, 2>(c, u); break;
            default: launch_update_stage<Real, 3>(c, u); break;
        }
        c->launches++;
        W5_CUDA(c, cudaGetLastError());
    }
    return W5CT_OK;
}

int step_impl(w5ct_ctx *c, const double *dt_dev, bool cellb_done) {
    if (ctx_fp64(c)) return run_step<double>(c, dt_dev, cellb_done);
    return run_step<float>(c, dt_dev, cellb_done);
}

int check_ready(w5ct_ctx *c) {
    if (!c) return W5CT_ERR_ARG;
    if (!c->have_grid) return fail(c, W5CT_ERR_STATE, "no grid: call w5ct_init_grid first");
    if (!c->have_state) return fail(c, W5CT_ERR_STATE, "no state: call w5ct_set_state first");
    return W5CT_OK;
}

int read_flag(w5ct_ctx *c, int *flag_out) {
    int f = 0;
    W5_CUDA(c, cudaMemcpyAsync(&f, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    *flag_out = f;
    return W5CT_OK;
}

// S_d of every patch into out[3 p + d] (host, 3 * npatch doubles)
int speeds_impl(w5ct_ctx *c, double *out) {
    int rc = ctx_fp64(c) ? launch_cellb<double>(c) : launch_cellb<float>(c);
    if (rc) return rc;
    rc = ctx_fp64(c) ? launch_speed<double>(c) : launch_speed<float>(c);
    if (rc) return rc;
    std::vector<unsigned long long> bits(3 * (size_t)c->npatch);
    W5_CUDA(c, cudaMemcpyAsync(bits.data(), c->smax, bits.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               c->stream));
    int flag = 0;
    rc = read_flag(c, &flag);
    if (rc) return rc;
    for (size_t d = 0; d < bits.size(); ++d) memcpy(&out[d], &bits[d], sizeof(double));
    if (flag & 2) return fail(c, W5CT_ERR_TIMEOUT, "a wait of the fused step expired; the state is not valid");
    if (flag) return fail(c, W5CT_ERR_NONPHYSICAL, "non-physical state (rho <= 0, P <= 0 or NaN)");
    return W5CT_OK;
}

int check_patch(w5ct_ctx *c, int patch) {
    if (patch < 0 || patch >= c->npatch) return fail(c, W5CT_ERR_ARG, "patch index %d out of range", patch);
    return W5CT_OK;
}

}  // namespace

extern "C" {

int w5ct_config_default(w5ct_config *cfg) {
    if (!cfg) return W5CT_ERR_ARG;
    memset(cfg, 0, sizeof(*cfg));
    cfg->gamma = 5.0 / 3.0;
    cfg->cfl = 0.8;
    cfg->weno_variant = W5CT_WENO_Z;
    cfg->precision = W5CT_FP64;
    cfg->eps_js = 1e-6;
    cfg->eps_z = 1e-40;
    cfg->eps_b = 1e-30;
    cfg->floors = 0;
    cfg->rho_min = 1e-8;
    cfg->p_min = 1e-8;
    cfg->stream = nullptr;
    return W5CT_OK;
}

int w5ct_create(const w5ct_config *cfg, w5ct_ctx **out) {
    if (!cfg || !out) return fail(nullptr, W5CT_ERR_ARG, "null argument");
    *out = nullptr;
    if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return fail(nullptr, W5CT_ERR_ARG, "gamma must be > 1 and cfl > 0");
    if (cfg->weno_variant != W5CT_WENO_JS && cfg->weno_variant != W5CT_WENO_Z)
        return fail(nullptr, W5CT_ERR_ARG, "unknown weno_variant %d", cfg->weno_variant);
    if (cfg->precision != W5CT_FP64 && cfg->precision != W5CT_FP32_BULK && cfg->precision != W5CT_FP64_DW)
        return fail(nullptr, W5CT_ERR_ARG, "unknown precision %d", cfg->precision);
    if (!(cfg->eps_js > 0.0) || !(cfg->eps_z > 0.0) || !(cfg->eps_b > 0.0))
        return fail(nullptr, W5CT_ERR_ARG, "epsilons must be positive");
    if (cfg->floors && (!(cfg->rho_min > 0.0) || !(cfg->p_min > 0.0)))
        return fail(nullptr, W5CT_ERR_ARG, "floors need rho_min > 0 and p_min > 0");
    w5ct_ctx *c = new (std::nothrow) w5ct_ctx();
    if (!c) return fail(nullptr, W5CT_ERR_ARG, "out of host memory");
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cfg->stream;
    c->real_size = cfg->precision == W5CT_FP32_BULK ? sizeof(float) : sizeof(double);
    snprintf(c->err, sizeof(c->err), "no error");
    *out = c;
    return W5CT_OK;
}

int w5ct_destroy(w5ct_ctx *c) {
    if (!c) return W5CT_OK;
    if (c->have_grid) cudaStreamSynchronize(c->stream);
    free_grid(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
    return W5CT_OK;
}

int w5ct_set_stream(w5ct_ctx *c, void *stream) {
    if (!c) return W5CT_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    c->cfg.stream = stream;
    return W5CT_OK;
}

int w5ct_init_grid(w5ct_ctx *c, int npatch, const int *n3, const double *dx3) {
    if (!c) return W5CT_ERR_ARG;
    if (!n3 || !dx3) return fail(c, W5CT_ERR_ARG, "null n3 or dx3");
    if (npatch < 1 || npatch > (1 << 24)) return fail(c, W5CT_ERR_ARG, "npatch must be in 1 .. 2^24 (got %d)", npatch);
    long long ntot = 0;
    for (int p = 0; p < npatch; ++p) {
        const int *m = n3 + 3 * p;
        const double *h = dx3 + 3 * p;
        if (m[0] < 1 || m[1] < 1 || m[2] < 1) return fail(c, W5CT_ERR_ARG, "patch %d: grid sizes must be >= 1", p);
        if (m[0] > 65535 * 32 || m[1] > 65535 * 8 || m[2] > 65535)
            return fail(c, W5CT_ERR_ARG, "patch %d: grid too large for the launch geometry", p);
        if (npatch > 1 && (long long)m[0] * m[1] * m[2] > (1LL << 30))
            return fail(c, W5CT_ERR_ARG, "patch %d: more than 2^30 cells in a batch of patches", p);
        if (!(h[0] > 0) || !(h[1] > 0) || !(h[2] > 0)) return fail(c, W5CT_ERR_ARG, "patch %d: spacings must be > 0", p);
        ntot += (long long)m[0] * m[1] * m[2];
    }
    free_grid(c);
    c->npatch = npatch;
    c->pg.resize(npatch);
    long long off = 0;
    for (int p = 0; p < npatch; ++p) {
        PatchGeom &g = c->pg[p];
        g.nx = n3[3 * p];
        g.ny = n3[3 * p + 1];
        g.nz = n3[3 * p + 2];
        g.pad = 0;
        g.off = off;
        g.dx = dx3[3 * p];
        g.dy = dx3[3 * p + 1];
        g.dz = dx3[3 * p + 2];
        g.rdx = 1.0 / g.dx;
        g.rdy = 1.0 / g.dy;
        g.rdz = 1.0 / g.dz;
        off += (long long)g.nx * g.ny * g.nz;
    }
    c->nx = n3[0];
    c->ny = n3[1];
    c->nz = n3[2];
    c->n = ntot;
    c->dx = dx3[0];
    c->dy = dx3[1];
    c->dz = dx3[2];
    // cell blocks of the batched cell-wise kernels: (patch, first cell)
    std::vector<int4> cells;
    if (npatch > 1) {
        for (int p = 0; p < npatch; ++p) {
            const PatchGeom &g = c->pg[p];
            const long long np = (long long)g.nx * g.ny * g.nz;
            for (long long q = 0; q < np; q += kCellBlock) cells.push_back(make_int4(p, (int)q, 0, 0));
        }
        c->ncells = (int)cells.size();
    }
    const size_t n = (size_t)c->n, rs = c->real_size;
    size_t bytes_total = 0;
    auto take = [&](size_t bytes) { size_t o = bytes_total; bytes_total += align256(bytes); return o; };
    const size_t o_q0 = take(5 * n * 8), o_b0 = take(3 * n * 8), o_acc = take(5 * n * 8), o_oacc = take(3 * n * 8);
    const size_t o_qs = take(5 * n * rs), o_bs = take(3 * n * rs), o_bc = take(3 * n * rs);
    const size_t o_Fx = take(5 * n * rs), o_Fy = take(5 * n * rs), o_Fz = take(5 * n * rs);
    const size_t o_Sx = take(2 * n * rs), o_Sy = take(2 * n * rs), o_Sz = take(2 * n * rs);
    const bool fp32 = !ctx_fp64(c);
    const size_t o_q0r = fp32 ? take(5 * n * rs) : 0, o_b0r = fp32 ? take(3 * n * rs) : 0;
    const size_t np = (size_t)npatch;
    const size_t o_dt = take(8 * np), o_smax = take(24 * np), o_flag = take(4), o_hits = take(8);
    const size_t o_part = take((size_t)kRedBlocks * 8 * 8), o_red = take(64), o_pl = take(64);
    const size_t o_pg = take(sizeof(PatchGeom) * np);
    const size_t o_pc = take(sizeof(int) * 4 * kMaxTileVariants);
    size_t o_cells = 0;
    if (npatch > 1) o_cells = take(sizeof(int4) * cells.size());
    void *slab = nullptr;
    cudaError_t e = cudaMalloc(&slab, bytes_total);
    if (e != cudaSuccess) return fail(c, W5CT_ERR_CUDA, "cudaMalloc(%zu bytes): %s", bytes_total, cudaGetErrorString(e));
    char *b = (char *)slab;
    c->slab = slab;
    c->q0 = (double *)(b + o_q0);
    c->b0 = (double *)(b + o_b0);
    c->acc = (double *)(b + o_acc);
    c->oacc = (double *)(b + o_oacc);
    c->qs = b + o_qs;
    c->bs = b + o_bs;
    c->bc = b + o_bc;
    c->Fx = b + o_Fx;
    c->Fy = b + o_Fy;
    c->Fz = b + o_Fz;
    c->Sx = b + o_Sx;
    c->Sy = b + o_Sy;
    c->Sz = b + o_Sz;
    c->q0r = fp32 ? (void *)(b + o_q0r) : (void *)c->q0;
    c->b0r = fp32 ? (void *)(b + o_b0r) : (void *)c->b0;
    c->dt_dev = (double *)(b + o_dt);
    c->smax = (unsigned long long *)(b + o_smax);
    c->flag = (int *)(b + o_flag);
    c->hits = (unsigned long long *)(b + o_hits);
    c->part = (double *)(b + o_part);
    c->red_out = (double *)(b + o_red);
    c->planes = (const double **)(b + o_pl);
    c->pg_dev = (PatchGeom *)(b + o_pg);
    c->pcounters = (int *)(b + o_pc);
    W5_CUDA(c, cudaMemcpy(c->pg_dev, c->pg.data(), sizeof(PatchGeom) * np, cudaMemcpyHostToDevice));
    if (npatch > 1) {
        c->cells_dev = (int4 *)(b + o_cells);
        W5_CUDA(c, cudaMemcpy(c->cells_dev, cells.data(), sizeof(int4) * cells.size(), cudaMemcpyHostToDevice));
        default_variants(c);
        int rc = build_tiles(c);
        if (rc) return rc;
    }
    W5_CUDA(c, ctx_fp64(c) ? prepare_sweeps<double>() : prepare_sweeps<float>());
    {
        int dev = 0, sms = 0;
        W5_CUDA(c, cudaGetDevice(&dev));
        W5_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        for (int ax = 0; ax < 3; ++ax)
            c->sweep_t2[ax] = ctx_fp64(c) ? choose_sweep_t2<double>(ax, c->nx, c->ny, c->nz, sms)
                                                            : choose_sweep_t2<float>(ax, c->nx, c->ny, c->nz, sms);
    }
    c->schedule = 0;
    for (int v = 0; v < n_variants(c); ++v) {
        const cudaError_t eg = ctx_fp64(c) ? persistent_grid<double>(c->cfg.weno_variant, v, c->pgrid[v])
                                                             : persistent_grid<float>(c->cfg.weno_variant, v, c->pgrid[v]);
        W5_CUDA(c, eg);
    }
    W5_CUDA(c, cudaMemsetAsync(c->flag, 0, 4, c->stream));
    W5_CUDA(c, cudaMemsetAsync(c->hits, 0, 8, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_grid = true;
    return W5CT_OK;
}

int w5ct_set_state(w5ct_ctx *c, int patch, const double *cons, const double *bface, int on_device) {
    if (!c) return W5CT_ERR_ARG;
    if (!c->have_grid) return fail(c, W5CT_ERR_STATE, "no grid: call w5ct_init_grid first");
    if (check_patch(c, patch)) return W5CT_ERR_ARG;
    if (!cons || !bface) return fail(c, W5CT_ERR_ARG, "null cons or bface");
    const size_t n = (size_t)c->n;
    const PatchGeom g = patch_of(c, patch);
    const size_t np = (size_t)g.nx * g.ny * g.nz, off = (size_t)g.off;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->npatch == 1) {
        W5_CUDA(c, cudaMemcpyAsync(c->q0, cons, 5 * n * sizeof(double), kind, c->stream));
        W5_CUDA(c, cudaMemcpyAsync(c->b0, bface, 3 * n * sizeof(double), kind, c->stream));
    } else {
        for (int f = 0; f < 5; ++f)
            W5_CUDA(c, cudaMemcpyAsync(c->q0 + f * n + off, cons + f * np, np * sizeof(double), kind, c->stream));
        for (int f = 0; f < 3; ++f)
            W5_CUDA(c, cudaMemcpyAsync(c->b0 + f * n + off, bface + f * np, np * sizeof(double), kind, c->stream));
    }
    if (ctx_fp64(c)) {
        for (int f = 0; f < 5; ++f)
            W5_CUDA(c, cudaMemcpyAsync((double *)c->qs + f * n + off, c->q0 + f * n + off, np * 8,
                                       cudaMemcpyDeviceToDevice, c->stream));
        for (int f = 0; f < 3; ++f)
            W5_CUDA(c, cudaMemcpyAsync((double *)c->bs + f * n + off, c->b0 + f * n + off, np * 8,
                                       cudaMemcpyDeviceToDevice, c->stream));
    } else {
        long long nb = ((long long)np + 255) / 256;
        if (nb > 8 * 152) nb = 8 * 152;
        for (int f = 0; f < 5; ++f) {
            to_real_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((long long)np, c->q0 + f * n + off,
                                                                      (float *)c->qs + f * n + off);
            to_real_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((long long)np, c->q0 + f * n + off,
                                                                      (float *)c->q0r + f * n + off);
        }
        for (int f = 0; f < 3; ++f) {
            to_real_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((long long)np, c->b0 + f * n + off,
                                                                      (float *)c->bs + f * n + off);
            to_real_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((long long)np, c->b0 + f * n + off,
                                                                      (float *)c->b0r + f * n + off);
        }
        c->launches += 16;
        W5_CUDA(c, cudaGetLastError());
    }
    W5_CUDA(c, cudaMemsetAsync(c->flag, 0, 4, c->stream));
    W5_CUDA(c, cudaMemsetAsync(c->hits, 0, 8, c->stream));
    if (!on_device) W5_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_state = true;
    return W5CT_OK;
}

int w5ct_get_state(w5ct_ctx *c, int patch, double *cons, double *bface, double *bcell, int on_device) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (check_patch(c, patch)) return W5CT_ERR_ARG;
    const size_t n = (size_t)c->n;
    const PatchGeom g = patch_of(c, patch);
    const size_t np = (size_t)g.nx * g.ny * g.nz, off = (size_t)g.off;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cons)
        for (int f = 0; f < 5; ++f)
            W5_CUDA(c, cudaMemcpyAsync(cons + f * np, c->q0 + f * n + off, np * 8, kind, c->stream));
    if (bface)
        for (int f = 0; f < 3; ++f)
            W5_CUDA(c, cudaMemcpyAsync(bface + f * np, c->b0 + f * n + off, np * 8, kind, c->stream));
    if (bcell) {
        // the FP64 accumulator planes are free between steps
        cellb_kernel<double><<<cellb_grid(g.nx, g.ny, g.nz), dim3(32, 8), 0, c->stream>>>(
            g.nx, g.ny, g.nz, cellb_chunk(g.nx, g.ny, g.nz), c->b0 + off, c->b0 + n + off, c->b0 + 2 * n + off,
            c->acc + off, c->acc + n + off, c->acc + 2 * n + off);
        c->launches++;
        W5_CUDA(c, cudaGetLastError());
        for (int f = 0; f < 3; ++f)
            W5_CUDA(c, cudaMemcpyAsync(bcell + f * np, c->acc + f * n + off, np * 8, kind, c->stream));
    }
    int flag = 0;
    rc = read_flag(c, &flag);
    if (rc) return rc;
    if (flag & 2) return fail(c, W5CT_ERR_TIMEOUT, "a wait of the fused step expired; the state is not valid");
    if (flag) return fail(c, W5CT_ERR_NONPHYSICAL, "non-physical state (rho <= 0, P <= 0 or NaN) met in a step");
    return W5CT_OK;
}

int w5ct_step(w5ct_ctx *c, double dt) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!(dt > 0.0) || !(dt < 1e300)) return fail(c, W5CT_ERR_ARG, "dt must be finite and > 0 (got %g)", dt);
    if (c->npatch > 1)
        fill_kernel<<<(c->npatch + 127) / 128, 128, 0, c->stream>>>(c->dt_dev, c->npatch, dt);
    else
        set_scalar_kernel<<<1, 1, 0, c->stream>>>(c->dt_dev, dt);
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    if (c->npatch > 1 && c->schedule == 2) return fused_step(c, c->dt_dev, nullptr);
    return step_impl(c, c->dt_dev, false);
}

int w5ct_step_dev(w5ct_ctx *c, const double *dt_dev) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!dt_dev) return fail(c, W5CT_ERR_ARG, "null dt_dev");
    if (c->npatch > 1 && c->schedule == 2) return fused_step(c, dt_dev, nullptr);
    return step_impl(c, dt_dev, false);
}

int w5ct_step_cfl(w5ct_ctx *c, double *dt_dev_out) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->npatch > 1 && c->schedule == 2) return fused_step(c, nullptr, dt_dev_out);
    rc = ctx_fp64(c) ? launch_cellb<double>(c) : launch_cellb<float>(c);
    if (rc) return rc;
    rc = ctx_fp64(c) ? launch_speed<double>(c) : launch_speed<float>(c);
    if (rc) return rc;
    rc = launch_dt(c, dt_dev_out);
    if (rc) return rc;
    return step_impl(c, c->dt_dev, true);
}

int w5ct_max_signal_speed(w5ct_ctx *c, int patch, double out[3]) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (check_patch(c, patch)) return W5CT_ERR_ARG;
    if (!out) return fail(c, W5CT_ERR_ARG, "null out");
    std::vector<double> S(3 * (size_t)c->npatch);
    rc = speeds_impl(c, S.data());
    for (int d = 0; d < 3; ++d) out[d] = S[3 * patch + d];
    return rc;
}

int w5ct_cfl_dt(w5ct_ctx *c, double *dt) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!dt) return fail(c, W5CT_ERR_ARG, "null dt");
    std::vector<double> S(3 * (size_t)c->npatch);
    rc = speeds_impl(c, S.data());
    if (rc) return rc;
    double best = 0.0;
    for (int p = 0; p < c->npatch; ++p) {
        const PatchGeom &g = c->pg[p];
        const double v = c->cfg.cfl / (S[3 * p] / g.dx + S[3 * p + 1] / g.dy + S[3 * p + 2] / g.dz);
        if (p == 0 || v < best) best = v;
    }
    *dt = best;
    return W5CT_OK;
}

int w5ct_div_b_norm(w5ct_ctx *c, int patch, double *linf, double *l2) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (check_patch(c, patch)) return W5CT_ERR_ARG;
    if (!linf || !l2) return fail(c, W5CT_ERR_ARG, "null output");
    const size_t n = (size_t)c->n;
    const PatchGeom g = patch_of(c, patch);
    const size_t off = (size_t)g.off;
    divb_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(g.nx, g.ny, g.nz, c->b0 + off, c->b0 + n + off,
                                                                   c->b0 + 2 * n + off, 1.0 / g.dx, 1.0 / g.dy,
                                                                   1.0 / g.dz, c->part);
    finalize_kernel<<<1, kRedThreads, 0, c->stream>>>(c->part, kRedBlocks, 2, 2, 1u, c->red_out);
    c->launches += 2;
    W5_CUDA(c, cudaGetLastError());
    double out[2];
    W5_CUDA(c, cudaMemcpyAsync(out, c->red_out, sizeof(out), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    *linf = out[0];
    *l2 = sqrt(out[1] / ((double)g.nx * g.ny * g.nz));
    return W5CT_OK;
}

int w5ct_conserved_totals(w5ct_ctx *c, int patch, double out[8]) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (check_patch(c, patch)) return W5CT_ERR_ARG;
    if (!out) return fail(c, W5CT_ERR_ARG, "null out");
    const size_t n = (size_t)c->n;
    const PatchGeom g = patch_of(c, patch);
    const size_t off = (size_t)g.off;
    const long long np = (long long)g.nx * g.ny * g.nz;
    const double *pl[8];
    for (int f = 0; f < 5; ++f) pl[f] = c->q0 + f * n + off;
    for (int f = 0; f < 3; ++f) pl[5 + f] = c->b0 + f * n + off;
    W5_CUDA(c, cudaMemcpyAsync((void *)c->planes, pl, sizeof(pl), cudaMemcpyHostToDevice, c->stream));
    sums_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(np, 8, c->planes, c->part);
    finalize_kernel<<<1, kRedThreads, 0, c->stream>>>(c->part, kRedBlocks, 8, 8, 0u, c->red_out);
    c->launches += 2;
    W5_CUDA(c, cudaGetLastError());
    W5_CUDA(c, cudaMemcpyAsync(out, c->red_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    const double dv = g.dx * g.dy * g.dz;
    for (int f = 0; f < 8; ++f) out[f] *= dv;
    return W5CT_OK;
}

}  // extern "C"

namespace {

template <typename Real>
SweepArgs<Real> sweep_args(w5ct_ctx *c, int ax) {
    const long long n = c->n;
    SweepArgs<Real> a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    for (int f = 0; f < 5; ++f) a.q[f] = plane<Real>(c->qs, n, f);
    for (int f = 0; f < 3; ++f) a.bc[f] = plane<Real>(c->bc, n, f);
    void *Fax[3] = {c->Fx, c->Fy, c->Fz};
    void *Sax[3] = {c->Sx, c->Sy, c->Sz};
    for (int f = 0; f < 5; ++f) a.F[f] = plane<Real>(Fax[ax], n, f);
    for (int f = 0; f < 2; ++f) a.S[f] = plane<Real>(Sax[ax], n, f);
    a.K = make_phys<Real>(c->cfg);
    a.flag = c->flag;
    a.hits = c->hits;
    a.dw = c->cfg.precision == W5CT_FP64_DW;
    return a;
}

// Measure every tile variant on every patch-size class and keep the fastest.
// A class is the patches with the same (nx, n2), n2 = ny for the x- and
// y-sweeps and nz for the z-sweep (the sizes that decide how full the tiles
// are).  Each class is timed on its own tiles, repeated so that one launch
// covers at least 4M faces (small classes would otherwise time launch
// latency), `reps` launches after one untimed launch.  The sweeps only write
// the flux buffers that every step rewrites; the floor-hit counter and the
// non-physical flag are restored.
template <typename Real>
int autotune_measure(w5ct_ctx *c, int reps) {
    int rc = launch_cellb<Real>(c);
    if (rc) return rc;
    unsigned long long hits0 = 0;
    int flag0 = 0;
    W5_CUDA(c, cudaMemcpyAsync(&hits0, c->hits, sizeof(hits0), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaMemcpyAsync(&flag0, c->flag, sizeof(flag0), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    const int nv = n_variants(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    W5_CUDA(c, cudaEventCreate(&e0));
    W5_CUDA(c, cudaEventCreate(&e1));
    int4 *scratch = nullptr;
    size_t cap = 0;
    std::vector<int4> tl;
    rc = W5CT_OK;
    const int variant = c->cfg.weno_variant;
    for (int ax = 0; ax < 3 && rc == W5CT_OK; ++ax) {
        const SweepArgs<Real> a = sweep_args<Real>(c, ax);
        std::map<std::pair<int, int>, std::vector<int>> cls;
        for (int p = 0; p < c->npatch; ++p)
            cls[std::make_pair(c->pg[p].nx, ax == 2 ? c->pg[p].nz : c->pg[p].ny)].push_back(p);
        for (auto &kv : cls) {
            const std::vector<int> &P = kv.second;
            long long faces = 0;
            for (int p : P) faces += (long long)c->pg[p].nx * c->pg[p].ny * c->pg[p].nz;
            const int R = (int)((4000000LL + faces - 1) / faces);
            float best = 0.f;
            int bestv = 0;
            for (int v = 0; v < nv && rc == W5CT_OK; ++v) {
                int bx, t2;
                variant_shape(c, ax, v, bx, t2);
                tl.clear();
                for (int r = 0; r < R; ++r)
                    for (int p : P) append_tiles(tl, p, c->pg[p], ax, bx, t2);
                if (tl.size() > cap) {
                    if (scratch) cudaFree(scratch);
                    scratch = nullptr;
                    cap = tl.size();
                    cudaError_t e = cudaMalloc(&scratch, sizeof(int4) * cap);
                    if (e != cudaSuccess) {
                        rc = fail(c, W5CT_ERR_CUDA, "autotune: cudaMalloc: %s", cudaGetErrorString(e));
                        break;
                    }
                }
                cudaError_t e = cudaMemcpy(scratch, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = launch_sweep_batched<Real>(ax, variant, v, a, c->pg_dev, scratch, (int)tl.size(), c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r)
                    e = launch_sweep_batched<Real>(ax, variant, v, a, c->pg_dev, scratch, (int)tl.size(), c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = fail(c, W5CT_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
                    break;
                }
                if (v == 0 || ms < best) {
                    best = ms;
                    bestv = v;
                }
            }
            for (int p : P) c->pvar[ax][p] = (signed char)bestv;
        }
    }
    if (scratch) cudaFree(scratch);
    if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
    }
    rc = build_tiles(c);
    if (rc) return rc;
    // schedule (w5ct_set_sweep_schedule): timed on whole steps from a
    // snapshot of the state, which is put back after every trial
    const bool timing = c->timing;
    c->timing = false;
    const size_t n = (size_t)c->n, rs = c->real_size;
    const bool fp32 = !ctx_fp64(c);
    const size_t bq = 8 * n * 8, br = 8 * n * rs, bsnap = bq + br + (fp32 ? br : 0);
    char *snap = nullptr;
    if (cudaMalloc(&snap, bsnap) == cudaSuccess) {
        auto copy_state = [&](bool save) -> cudaError_t {
            struct { void *dev; size_t bytes; } parts[6] = {{c->q0, 5 * n * 8}, {c->b0, 3 * n * 8},
                                                         {c->qs, 5 * n * rs}, {c->bs, 3 * n * rs},
                                                         {fp32 ? c->q0r : nullptr, 5 * n * rs},
                                                         {fp32 ? c->b0r : nullptr, 3 * n * rs}};
            size_t o = 0;
            for (auto &pt : parts) {
                if (!pt.dev) continue;
                cudaError_t e = save ? cudaMemcpyAsync(snap + o, pt.dev, pt.bytes, cudaMemcpyDeviceToDevice, c->stream)
                                     : cudaMemcpyAsync(pt.dev, snap + o, pt.bytes, cudaMemcpyDeviceToDevice, c->stream);
                if (e != cudaSuccess) return e;
                o += pt.bytes;
            }
            return cudaSuccess;
        };
        cudaError_t e = copy_state(true);
        float best = 0.f;
        int best_sc = 0;
        for (int sc = 0; sc < 3 && e == cudaSuccess && rc == W5CT_OK; ++sc) {
            c->schedule = sc;
            if (sc == 2) {
                rc = build_fused(c);
                if (rc) break;
            }
            e = copy_state(false);
            if (e == cudaSuccess) rc = w5ct_step_cfl(c, nullptr);          // untimed
            if (e == cudaSuccess && rc == W5CT_OK) e = cudaEventRecord(e0, c->stream);
            for (int r = 0; r < reps && e == cudaSuccess && rc == W5CT_OK; ++r) rc = w5ct_step_cfl(c, nullptr);
            if (e == cudaSuccess && rc == W5CT_OK) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess && rc == W5CT_OK) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess && rc == W5CT_OK) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rc == W5CT_OK && (sc == 0 || ms < best)) {
                best = ms;
                best_sc = sc;
            }
        }
        if (e == cudaSuccess) e = copy_state(false);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(snap);
        c->schedule = best_sc;
        if (e != cudaSuccess && rc == W5CT_OK) rc = fail(c, W5CT_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    c->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    W5_CUDA(c, cudaMemcpyAsync(c->hits, &hits0, sizeof(hits0), cudaMemcpyHostToDevice, c->stream));
    W5_CUDA(c, cudaMemcpyAsync(c->flag, &flag0, sizeof(flag0), cudaMemcpyHostToDevice, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    return W5CT_OK;
}

// ---------------------------------------------------------------- adjoint

// Work buffers of the adjoint step, in one allocation: stage states
// (4 x 8 planes of Real), then double planes: two sets of stage adjoints
// (5 + 3 each), lamD (5), mu (3), lamO (3), lamF (15), lamS (6), lamBc (3),
// face contributions (48).
constexpr int kAdjDoublePlanes = 2 * 8 + 5 + 3 + 3 + 15 + 6 + 3 + 48;

int ensure_adj(w5ct_ctx *c) {
    if (c->adj_slab) return W5CT_OK;
    const size_t n = (size_t)c->n;
    const size_t bytes = align256(32 * n * c->real_size) + (size_t)kAdjDoublePlanes * n * 8;
    W5_CUDA(c, cudaMalloc(&c->adj_slab, bytes));
    return W5CT_OK;
}

template <typename Real>
int adjoint_step_impl(w5ct_ctx *c, double dt, const double *lq_fin, const double *lb_fin, double *lq_out,
                      double *lb_out) {
    int rc = ensure_adj(c);
    if (rc) return rc;
    const long long nl = c->n;
    const size_t n = (size_t)nl;
    cudaStream_t st = c->stream;
    Real *stage = reinterpret_cast<Real *>(c->adj_slab);
    double *w = reinterpret_cast<double *>((char *)c->adj_slab + align256(32 * n * sizeof(Real)));
    double *set[2] = {w, w + 8 * n};           // stage adjoints: q (5 planes) then b (3 planes)
    double *lamD = w + 16 * n, *mu = lamD + 5 * n, *lamO = mu + 3 * n, *lamF = lamO + 3 * n;
    double *lamS = lamF + 15 * n, *lamBc = lamS + 6 * n, *cb = lamBc + 3 * n;

    unsigned long long hits0 = 0;
    int flag0 = 0;
    W5_CUDA(c, cudaMemcpyAsync(&hits0, c->hits, sizeof(hits0), cudaMemcpyDeviceToHost, st));
    W5_CUDA(c, cudaMemcpyAsync(&flag0, c->flag, sizeof(flag0), cudaMemcpyDeviceToHost, st));
    W5_CUDA(c, cudaStreamSynchronize(st));

    // forward stages 0..2 from the current state, keeping the four stage states
    fill_kernel<<<1, 32, 0, st>>>(c->dt_dev, 1, dt);
    rc = run_step<Real>(c, c->dt_dev, false, 2, stage);
    if (rc) return rc;
    // the context's stage buffers back to the state (as after set_state or a step)
    W5_CUDA(c, cudaMemcpyAsync(c->qs, stage, 5 * n * sizeof(Real), cudaMemcpyDeviceToDevice, st));
    W5_CUDA(c, cudaMemcpyAsync(c->bs, stage + 5 * n, 3 * n * sizeof(Real), cudaMemcpyDeviceToDevice, st));

    // backward through the stages
    W5_CUDA(c, cudaMemcpyAsync(lq_out, lq_fin, 5 * n * 8, cudaMemcpyDeviceToDevice, st));
    W5_CUDA(c, cudaMemcpyAsync(lb_out, lb_fin, 3 * n * 8, cudaMemcpyDeviceToDevice, st));
    const double wc[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double cs[3] = {0.5, 0.5, 1.0};
    const AdjGrid g = {c->nx, c->ny, c->nz, 1.0 / c->dx, 1.0 / c->dy, 1.0 / c->dz};
    const unsigned nb = (unsigned)((n + 255) / 256);
    const Phys<Real> K = make_phys<Real>(c->cfg);
    double *next = nullptr;
    for (int s = 3; s >= 0; --s) {
        double *cur = set[s & 1];
        adj_sources_kernel<<<nb, 256, 0, st>>>(nl, dt * wc[s], s < 3 ? cs[s] * dt : 0.0, lq_fin, lb_fin,
                                               next, next ? next + 5 * n : nullptr, lamD, mu);
        adj_curl_kernel<<<nb, 256, 0, st>>>(g, mu, lamO);
        adj_flux_kernel<<<nb, 256, 0, st>>>(g, lamD, lamO, lamF, lamS);
        // the stage's cell field from its stored face field
        const Real *sq = stage + (size_t)s * 8 * n, *sb = sq + 5 * n;
        cellb_kernel<Real><<<cellb_grid(c->nx, c->ny, c->nz), dim3(32, 8), 0, st>>>(
            c->nx, c->ny, c->nz, cellb_chunk(c->nx, c->ny, c->nz), sb, sb + n, sb + 2 * n,
            plane<Real>(c->bc, nl, 0), plane<Real>(c->bc, nl, 1), plane<Real>(c->bc, nl, 2));
        W5_CUDA(c, cudaMemsetAsync(cur, 0, 5 * n * 8, st));
        W5_CUDA(c, cudaMemsetAsync(lamBc, 0, 3 * n * 8, st));
        for (int ax = 0; ax < 3; ++ax) {
            AdjSweepArgs<Real> aa;
            aa.nx = c->nx;
            aa.ny = c->ny;
            aa.nz = c->nz;
            for (int f = 0; f < 5; ++f) aa.q[f] = sq + (size_t)f * n;
            for (int f = 0; f < 3; ++f) aa.bc[f] = plane<Real>(c->bc, nl, f);
            for (int f = 0; f < 5; ++f) aa.lamF[f] = lamF + (size_t)(5 * ax + f) * n;
            for (int f = 0; f < 2; ++f) aa.lamS[f] = lamS + (size_t)(2 * ax + f) * n;
            aa.cb = cb;
            aa.K = K;
            const cudaError_t ea = c->cfg.weno_variant == W5CT_WENO_JS ? launch_adj_sweep<Real, 0>(ax, aa, st)
                                                                       : launch_adj_sweep<Real, 1>(ax, aa, st);
            W5_CUDA(c, ea);
            double *q[5], *b[3];
            for (int f = 0; f < 5; ++f) q[f] = cur + (size_t)f * n;
            for (int f = 0; f < 3; ++f) b[f] = lamBc + (size_t)f * n;
            if (ax == 0)
                adj_gather_kernel<0><<<nb, 256, 0, st>>>(c->nx, c->ny, c->nz, cb, q[0], q[1], q[2], q[3], q[4], b[0], b[1], b[2]);
            else if (ax == 1)
                adj_gather_kernel<1><<<nb, 256, 0, st>>>(c->nx, c->ny, c->nz, cb, q[0], q[1], q[2], q[3], q[4], b[0], b[1], b[2]);
            else
                adj_gather_kernel<2><<<nb, 256, 0, st>>>(c->nx, c->ny, c->nz, cb, q[0], q[1], q[2], q[3], q[4], b[0], b[1], b[2]);
            c->launches += 2;
        }
        // stage face-field adjoint; both added into the step's outputs
        adj_interp_kernel<<<nb, 256, 0, st>>>(g, lamBc, cur, cur + 5 * n, lq_out, lb_out);
        c->launches += 5;
        W5_CUDA(c, cudaGetLastError());
        next = cur;
    }
    W5_CUDA(c, cudaMemcpyAsync(c->hits, &hits0, sizeof(hits0), cudaMemcpyHostToDevice, st));
    W5_CUDA(c, cudaMemcpyAsync(c->flag, &flag0, sizeof(flag0), cudaMemcpyHostToDevice, st));
    W5_CUDA(c, cudaStreamSynchronize(st));
    return W5CT_OK;
}

}  // namespace

extern "C" {

int w5ct_autotune(w5ct_ctx *c, int mode, int reps) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->npatch == 1) return W5CT_OK;
    const int nv = n_variants(c);
    if (mode >= nv || mode < W5CT_TUNE_MODEL)
        return fail(c, W5CT_ERR_ARG, "autotune mode %d: expected -2 (model), -1 (measure) or a variant 0..%d", mode,
                    nv - 1);
    if (mode == W5CT_TUNE_MEASURE) {
        if (reps < 1 || reps > 100) return fail(c, W5CT_ERR_ARG, "reps must be in 1 .. 100");
        return ctx_fp64(c) ? autotune_measure<double>(c, reps) : autotune_measure<float>(c, reps);
    }
    if (mode == W5CT_TUNE_MODEL) {
        default_variants(c);
    } else {
        for (int a = 0; a < 3; ++a) c->pvar[a].assign(c->npatch, (signed char)mode);
    }
    return build_tiles(c);
}

int w5ct_set_sweep_schedule(w5ct_ctx *c, int schedule) {
    if (!c) return W5CT_ERR_ARG;
    if (!c->have_grid) return fail(c, W5CT_ERR_STATE, "no grid: call w5ct_init_grid first");
    if (schedule < 0 || schedule > 2) return fail(c, W5CT_ERR_ARG, "schedule must be 0, 1 or 2");
    if (schedule != 0 && c->npatch == 1)
        return fail(c, W5CT_ERR_UNSUPPORTED, "the persistent schedules take a batch of patches");
    if (schedule == 2) {
        int rc = build_fused(c);
        if (rc) return rc;
    }
    if (c->schedule != schedule && c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    c->schedule = schedule;
    return W5CT_OK;
}

int w5ct_fused_wait_check(w5ct_ctx *c, long long spin_limit, int *status) {
    if (!c || !status) return W5CT_ERR_ARG;
    if (!c->have_grid || !c->have_state) return fail(c, W5CT_ERR_STATE, "call w5ct_init_grid and set the state first");
    if (c->npatch == 1) return fail(c, W5CT_ERR_UNSUPPORTED, "the fused step takes a batch of patches");
    if (spin_limit < 1 || spin_limit > kFusedSpinLimit)
        return fail(c, W5CT_ERR_ARG, "spin_limit must be in [1, 2^22]");
    int rc = build_fused(c);
    if (rc) return rc;
    int flag0 = 0;
    rc = read_flag(c, &flag0);
    if (rc) return rc;
    rc = ctx_fp64(c) ? fused_step_impl<double>(c, nullptr, nullptr, true, spin_limit)
                                       : fused_step_impl<float>(c, nullptr, nullptr, true, spin_limit);
    if (rc) return rc;
    int flag = 0;
    rc = read_flag(c, &flag);
    if (rc) return rc;
    *status = (flag & 2) ? W5CT_ERR_TIMEOUT : (flag ? W5CT_ERR_NONPHYSICAL : W5CT_OK);
    W5_CUDA(c, cudaMemcpyAsync(c->flag, &flag0, sizeof(flag0), cudaMemcpyHostToDevice, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    return W5CT_OK;
}

int w5ct_sweep_schedule(w5ct_ctx *c, int *schedule) {
    if (!c || !schedule) return W5CT_ERR_ARG;
    *schedule = c->schedule;
    return W5CT_OK;
}

int w5ct_tile_variant(w5ct_ctx *c, int axis, int patch, int out[3]) {
    if (!c || !out) return W5CT_ERR_ARG;
    if (!c->have_grid) return fail(c, W5CT_ERR_STATE, "no grid: call w5ct_init_grid first");
    if (axis < 0 || axis > 2) return fail(c, W5CT_ERR_ARG, "axis must be 0, 1 or 2");
    if (check_patch(c, patch)) return W5CT_ERR_ARG;
    const int v = c->npatch > 1 ? c->pvar[axis][patch] : 0;
    int bx, t2;
    variant_shape(c, axis, v, bx, t2);
    out[0] = v;
    out[1] = bx;
    out[2] = t2;
    return W5CT_OK;
}

int w5ct_adjoint_step(w5ct_ctx *c, double dt, const double *lam_q, const double *lam_b, double *lam_q_out,
                      double *lam_b_out) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->npatch != 1) return fail(c, W5CT_ERR_UNSUPPORTED, "the adjoint step takes one patch");
    if (!(dt > 0.0) || !(dt < 1e300)) return fail(c, W5CT_ERR_ARG, "dt must be finite and > 0 (got %g)", dt);
    if (!lam_q || !lam_b || !lam_q_out || !lam_b_out) return fail(c, W5CT_ERR_ARG, "null adjoint buffer");
    return ctx_fp64(c) ? adjoint_step_impl<double>(c, dt, lam_q, lam_b, lam_q_out, lam_b_out)
                                          : adjoint_step_impl<float>(c, dt, lam_q, lam_b, lam_q_out, lam_b_out);
}

int w5ct_misfit(w5ct_ctx *c, const double *target_cons, const double *target_bface, double *value, double *lam_q,
                double *lam_b) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->npatch != 1) return fail(c, W5CT_ERR_UNSUPPORTED, "the misfit takes one patch");
    if (!target_cons || !target_bface || !value || !lam_q || !lam_b) return fail(c, W5CT_ERR_ARG, "null buffer");
    const double dV = c->dx * c->dy * c->dz;
    misfit_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, dV, c->q0, c->b0, target_cons,
                                                                     target_bface, lam_q, lam_b, c->part);
    finalize_kernel<<<1, kRedThreads, 0, c->stream>>>(c->part, kRedBlocks, 1, 1, 0u, c->red_out);
    c->launches += 2;
    W5_CUDA(c, cudaGetLastError());
    W5_CUDA(c, cudaMemcpyAsync(value, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    return W5CT_OK;
}

static int ic_check(const int n3[3], const double dx3[3]) {
    if (!n3 || !dx3) return W5CT_ERR_ARG;
    if (n3[0] < 1 || n3[1] < 1 || n3[2] < 1) return W5CT_ERR_ARG;
    if ((long long)n3[0] * n3[1] * n3[2] > (1LL << 31)) return W5CT_ERR_ARG;
    if (!(dx3[0] > 0) || !(dx3[1] > 0) || !(dx3[2] > 0)) return W5CT_ERR_ARG;
    return W5CT_OK;
}

int w5ct_ic_from_potential(const int n3[3], const double dx3[3], double gamma, const double B0[3], const double *rho,
                           const double *v, const double *P, const double *A, double *cons, double *bface,
                           void *stream) {
    if (ic_check(n3, dx3) || !B0 || !rho || !v || !P || !A || !cons || !bface || !(gamma > 1.0)) {
        set_global_error("w5ct_ic_from_potential: bad argument");
        return W5CT_ERR_ARG;
    }
    const AdjGrid g = {n3[0], n3[1], n3[2], 1.0 / dx3[0], 1.0 / dx3[1], 1.0 / dx3[2]};
    const long long n = (long long)n3[0] * n3[1] * n3[2];
    const unsigned nb = (unsigned)((n + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    ic_curl_kernel<<<nb, 256, 0, st>>>(g, A, B0[0], B0[1], B0[2], bface);
    ic_cons_kernel<<<nb, 256, 0, st>>>(g, gamma - 1.0, rho, v, P, bface, cons);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return W5CT_ERR_CUDA;
    }
    return W5CT_OK;
}

int w5ct_ic_from_potential_adjoint(const int n3[3], const double dx3[3], const double *rho, const double *v,
                                   const double *bface, const double *lam_cons, const double *lam_bface,
                                   double *lam_rho, double *lam_v, double *lam_A, double *lam_b, void *stream) {
    if (ic_check(n3, dx3) || !rho || !v || !bface || !lam_cons || !lam_bface || !lam_rho || !lam_v || !lam_A ||
        !lam_b) {
        set_global_error("w5ct_ic_from_potential_adjoint: bad argument");
        return W5CT_ERR_ARG;
    }
    const AdjGrid g = {n3[0], n3[1], n3[2], 1.0 / dx3[0], 1.0 / dx3[1], 1.0 / dx3[2]};
    const long long n = (long long)n3[0] * n3[1] * n3[2];
    const unsigned nb = (unsigned)((n + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    // lam_A holds the cell-field adjoint until the last kernel overwrites it
    ic_cons_adjoint_kernel<<<nb, 256, 0, st>>>(g, rho, v, bface, lam_cons, lam_rho, lam_v, lam_A);
    ic_interp_adjoint_kernel<<<nb, 256, 0, st>>>(g, lam_bface, lam_A, lam_b);
    ic_curl_adjoint_kernel<<<nb, 256, 0, st>>>(g, lam_b, lam_A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return W5CT_ERR_CUDA;
    }
    return W5CT_OK;
}

int w5ct_step_graph(w5ct_ctx *c, int nsteps) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (nsteps < 0) return fail(c, W5CT_ERR_ARG, "nsteps must be >= 0");
    if (!c->gexec) {
        // capture one w5ct_step_cfl on a private stream (the legacy default
        // stream cannot be captured); the graph is then launched on the
        // context's stream
        if (!c->cap_stream) W5_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        W5_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaStream_t user = c->stream;
        const bool timing = c->timing;
        const long long l0 = c->launches;
        c->stream = c->cap_stream;
        c->timing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = w5ct_step_cfl(c, nullptr);
            e = cudaStreamEndCapture(c->cap_stream, &graph);
        }
        c->stream = user;
        c->timing = timing;
        c->graph_kernels = c->launches - l0;
        c->launches = l0;
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(c, W5CT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, W5CT_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    for (int s = 0; s < nsteps; ++s) {
        W5_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
        c->launches += c->graph_kernels;
    }
    return W5CT_OK;
}

int w5ct_status(w5ct_ctx *c, long long *floor_hits, int *nonphysical) {
    if (!c) return W5CT_ERR_ARG;
    if (!c->have_grid) return fail(c, W5CT_ERR_STATE, "no grid");
    unsigned long long h = 0;
    W5_CUDA(c, cudaMemcpyAsync(&h, c->hits, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    int f = 0;
    int rc = read_flag(c, &f);
    if (rc) return rc;
    if (floor_hits) *floor_hits = (long long)h;
    if (nonphysical) *nonphysical = f & 1;
    return W5CT_OK;
}

int w5ct_synchronize(w5ct_ctx *c) {
    if (!c) return W5CT_ERR_ARG;
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    return W5CT_OK;
}

int w5ct_set_timing(w5ct_ctx *c, int enable) {
    if (!c) return W5CT_ERR_ARG;
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    c->timing = enable != 0;
    c->ev_used = 0;
    c->sweep_units = 0;
    return W5CT_OK;
}

int w5ct_sweep_timing(w5ct_ctx *c, long long *launches, double *total_ms) {
    if (!c || !launches || !total_ms) return W5CT_ERR_ARG;
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    for (size_t e = 0; e + 1 < c->ev_used; e += 2) {
        float ms = 0.0f;
        W5_CUDA(c, cudaEventElapsedTime(&ms, c->ev[e], c->ev[e + 1]));
        tot += ms;
    }
    *launches = c->sweep_units;
    *total_ms = tot;
    return W5CT_OK;
}

int w5ct_launch_count(w5ct_ctx *c, long long *launches) {
    if (!c || !launches) return W5CT_ERR_ARG;
    *launches = c->launches;
    return W5CT_OK;
}

const char *w5ct_last_error(const w5ct_ctx *c) { return c ? c->err : g_create_err; }

}  // extern "C"
