// w5ct_api.cu -- the C ABI of libw5ct (declared in include/w5ct.h): context,
// device memory, state transfer, the RK4 + CT step driver, reductions.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "w5ct.h"
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
    // timing and accounting
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    long long launches = 0;
    char err[512];
};

namespace {

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
    K.floors = c.floors;
    return K;
}

template <typename Real>
Real *plane(void *base, long long n, int f) {
    return reinterpret_cast<Real *>(base) + (size_t)f * (size_t)n;
}

void free_grid(w5ct_ctx *c) {
    if (c->slab) cudaFree(c->slab);
    c->slab = nullptr;
    c->have_grid = false;
    c->have_state = false;
}

dim3 cell_grid(const w5ct_ctx *c) { return dim3((c->nx + 31) / 32, (c->ny + 7) / 8, c->nz); }

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
    cellb_kernel<Real><<<cell_grid(c), dim3(32, 8), 0, c->stream>>>(
        c->nx, c->ny, c->nz, plane<Real>(c->bs, n, 0), plane<Real>(c->bs, n, 1), plane<Real>(c->bs, n, 2),
        plane<Real>(c->bc, n, 0), plane<Real>(c->bc, n, 1), plane<Real>(c->bc, n, 2));
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return W5CT_OK;
}

template <typename Real>
int launch_speed(w5ct_ctx *c) {
    const long long n = c->n;
    W5_CUDA(c, cudaMemsetAsync(c->smax, 0, 3 * sizeof(unsigned long long), c->stream));
    long long nb = (n + kRedThreads - 1) / kRedThreads;
    if (nb > 4 * 152) nb = 4 * 152;
    speed_kernel<Real><<<(unsigned)nb, kRedThreads, 0, c->stream>>>(
        n, c->nx, c->ny, plane<Real>(c->qs, n, 0), plane<Real>(c->qs, n, 1), plane<Real>(c->qs, n, 2),
        plane<Real>(c->qs, n, 3), plane<Real>(c->qs, n, 4), plane<Real>(c->bc, n, 0), plane<Real>(c->bc, n, 1),
        plane<Real>(c->bc, n, 2), make_phys<Real>(c->cfg), c->smax, c->flag);
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return W5CT_OK;
}

template <typename Real, int S>
void launch_update_stage(w5ct_ctx *c, const UpdateArgs<Real> &u) {
    update_kernel<Real, S><<<cell_grid(c), dim3(32, 8), 0, c->stream>>>(u);
}

template <typename Real>
int run_step(w5ct_ctx *c, const double *dt_dev, bool cellb_done) {
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

    void *Fax[3] = {c->Fx, c->Fy, c->Fz};
    void *Sax[3] = {c->Sx, c->Sy, c->Sz};
    const int variant = c->cfg.weno_variant;
    for (int s = 0; s < 4; ++s) {
        if (!(s == 0 && cellb_done)) {
            int rc = launch_cellb<Real>(c);
            if (rc) return rc;
        }
        for (int ax = 0; ax < 3; ++ax) {
            for (int f = 0; f < 5; ++f) a.F[f] = plane<Real>(Fax[ax], n, f);
            for (int f = 0; f < 2; ++f) a.S[f] = plane<Real>(Sax[ax], n, f);
            int rc = record_event(c);
            if (rc) return rc;
            W5_CUDA(c, launch_sweep<Real>(ax, variant, a, c->stream));
            c->launches++;
            rc = record_event(c);
            if (rc) return rc;
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
    if (c->cfg.precision == W5CT_FP64) return run_step<double>(c, dt_dev, cellb_done);
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

int speeds_impl(w5ct_ctx *c, double out[3]) {
    int rc = c->cfg.precision == W5CT_FP64 ? launch_cellb<double>(c) : launch_cellb<float>(c);
    if (rc) return rc;
    rc = c->cfg.precision == W5CT_FP64 ? launch_speed<double>(c) : launch_speed<float>(c);
    if (rc) return rc;
    unsigned long long bits[3];
    W5_CUDA(c, cudaMemcpyAsync(bits, c->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    int flag = 0;
    rc = read_flag(c, &flag);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d) memcpy(&out[d], &bits[d], sizeof(double));
    if (flag) return fail(c, W5CT_ERR_NONPHYSICAL, "non-physical state (rho <= 0, P <= 0 or NaN)");
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
    if (cfg->precision != W5CT_FP64 && cfg->precision != W5CT_FP32_BULK)
        return fail(nullptr, W5CT_ERR_ARG, "unknown precision %d", cfg->precision);
    if (!(cfg->eps_js > 0.0) || !(cfg->eps_z > 0.0) || !(cfg->eps_b > 0.0))
        return fail(nullptr, W5CT_ERR_ARG, "epsilons must be positive");
    if (cfg->floors && (!(cfg->rho_min > 0.0) || !(cfg->p_min > 0.0)))
        return fail(nullptr, W5CT_ERR_ARG, "floors need rho_min > 0 and p_min > 0");
    w5ct_ctx *c = new (std::nothrow) w5ct_ctx();
    if (!c) return fail(nullptr, W5CT_ERR_ARG, "out of host memory");
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cfg->stream;
    c->real_size = cfg->precision == W5CT_FP64 ? sizeof(double) : sizeof(float);
    snprintf(c->err, sizeof(c->err), "no error");
    *out = c;
    return W5CT_OK;
}

int w5ct_destroy(w5ct_ctx *c) {
    if (!c) return W5CT_OK;
    if (c->have_grid) cudaStreamSynchronize(c->stream);
    free_grid(c);
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
    if (npatch != 1) return fail(c, W5CT_ERR_UNSUPPORTED, "only npatch = 1 is implemented (got %d)", npatch);
    if (n3[0] < 1 || n3[1] < 1 || n3[2] < 1) return fail(c, W5CT_ERR_ARG, "grid sizes must be >= 1");
    if (n3[0] > 65535 * 32 || n3[1] > 65535 * 8 || n3[2] > 65535)
        return fail(c, W5CT_ERR_ARG, "grid too large for the launch geometry");
    if (!(dx3[0] > 0) || !(dx3[1] > 0) || !(dx3[2] > 0)) return fail(c, W5CT_ERR_ARG, "spacings must be > 0");
    free_grid(c);
    c->nx = n3[0];
    c->ny = n3[1];
    c->nz = n3[2];
    c->n = (long long)c->nx * c->ny * c->nz;
    c->dx = dx3[0];
    c->dy = dx3[1];
    c->dz = dx3[2];
    const size_t n = (size_t)c->n, rs = c->real_size;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_q0 = take(5 * n * 8), o_b0 = take(3 * n * 8), o_acc = take(5 * n * 8), o_oacc = take(3 * n * 8);
    const size_t o_qs = take(5 * n * rs), o_bs = take(3 * n * rs), o_bc = take(3 * n * rs);
    const size_t o_Fx = take(5 * n * rs), o_Fy = take(5 * n * rs), o_Fz = take(5 * n * rs);
    const size_t o_Sx = take(2 * n * rs), o_Sy = take(2 * n * rs), o_Sz = take(2 * n * rs);
    const bool fp32 = c->cfg.precision != W5CT_FP64;
    const size_t o_q0r = fp32 ? take(5 * n * rs) : 0, o_b0r = fp32 ? take(3 * n * rs) : 0;
    const size_t o_dt = take(8), o_smax = take(24), o_flag = take(4), o_hits = take(8);
    const size_t o_part = take((size_t)kRedBlocks * 8 * 8), o_red = take(64), o_pl = take(64);
    void *slab = nullptr;
    cudaError_t e = cudaMalloc(&slab, off);
    if (e != cudaSuccess) return fail(c, W5CT_ERR_CUDA, "cudaMalloc(%zu bytes): %s", off, cudaGetErrorString(e));
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
    W5_CUDA(c, cudaMemsetAsync(c->flag, 0, 4, c->stream));
    W5_CUDA(c, cudaMemsetAsync(c->hits, 0, 8, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_grid = true;
    return W5CT_OK;
}

int w5ct_set_state(w5ct_ctx *c, int patch, const double *cons, const double *bface, int on_device) {
    if (!c) return W5CT_ERR_ARG;
    if (!c->have_grid) return fail(c, W5CT_ERR_STATE, "no grid: call w5ct_init_grid first");
    if (patch != 0) return fail(c, W5CT_ERR_ARG, "patch index %d out of range", patch);
    if (!cons || !bface) return fail(c, W5CT_ERR_ARG, "null cons or bface");
    const size_t n = (size_t)c->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    W5_CUDA(c, cudaMemcpyAsync(c->q0, cons, 5 * n * sizeof(double), kind, c->stream));
    W5_CUDA(c, cudaMemcpyAsync(c->b0, bface, 3 * n * sizeof(double), kind, c->stream));
    if (c->cfg.precision == W5CT_FP64) {
        W5_CUDA(c, cudaMemcpyAsync(c->qs, c->q0, 5 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
        W5_CUDA(c, cudaMemcpyAsync(c->bs, c->b0, 3 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        long long nb = ((long long)5 * n + 255) / 256;
        if (nb > 8 * 152) nb = 8 * 152;
        to_real_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((long long)(5 * n), c->q0, (float *)c->qs);
        to_real_kernel<float><<<(unsigned)nb, 256, 0, c->stream>>>((long long)(3 * n), c->b0, (float *)c->bs);
        c->launches += 2;
        W5_CUDA(c, cudaGetLastError());
        W5_CUDA(c, cudaMemcpyAsync(c->q0r, c->qs, 5 * n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        W5_CUDA(c, cudaMemcpyAsync(c->b0r, c->bs, 3 * n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
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
    if (patch != 0) return fail(c, W5CT_ERR_ARG, "patch index %d out of range", patch);
    const size_t n = (size_t)c->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cons) W5_CUDA(c, cudaMemcpyAsync(cons, c->q0, 5 * n * 8, kind, c->stream));
    if (bface) W5_CUDA(c, cudaMemcpyAsync(bface, c->b0, 3 * n * 8, kind, c->stream));
    if (bcell) {
        // the FP64 accumulator planes are free between steps
        cellb_kernel<double><<<cell_grid(c), dim3(32, 8), 0, c->stream>>>(
            c->nx, c->ny, c->nz, c->b0, c->b0 + n, c->b0 + 2 * n, c->acc, c->acc + n, c->acc + 2 * n);
        c->launches++;
        W5_CUDA(c, cudaGetLastError());
        W5_CUDA(c, cudaMemcpyAsync(bcell, c->acc, 3 * n * 8, kind, c->stream));
    }
    int flag = 0;
    rc = read_flag(c, &flag);
    if (rc) return rc;
    if (flag) return fail(c, W5CT_ERR_NONPHYSICAL, "non-physical state (rho <= 0, P <= 0 or NaN) met in a step");
    return W5CT_OK;
}

int w5ct_step(w5ct_ctx *c, double dt) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!(dt > 0.0) || !(dt < 1e300)) return fail(c, W5CT_ERR_ARG, "dt must be finite and > 0 (got %g)", dt);
    set_scalar_kernel<<<1, 1, 0, c->stream>>>(c->dt_dev, dt);
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return step_impl(c, c->dt_dev, false);
}

int w5ct_step_dev(w5ct_ctx *c, const double *dt_dev) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!dt_dev) return fail(c, W5CT_ERR_ARG, "null dt_dev");
    return step_impl(c, dt_dev, false);
}

int w5ct_step_cfl(w5ct_ctx *c, double *dt_dev_out) {
    int rc = check_ready(c);
    if (rc) return rc;
    rc = c->cfg.precision == W5CT_FP64 ? launch_cellb<double>(c) : launch_cellb<float>(c);
    if (rc) return rc;
    rc = c->cfg.precision == W5CT_FP64 ? launch_speed<double>(c) : launch_speed<float>(c);
    if (rc) return rc;
    dt_kernel<<<1, 1, 0, c->stream>>>(c->smax, c->cfg.cfl, c->dx, c->dy, c->dz, c->dt_dev, dt_dev_out);
    c->launches++;
    W5_CUDA(c, cudaGetLastError());
    return step_impl(c, c->dt_dev, true);
}

int w5ct_max_signal_speed(w5ct_ctx *c, int patch, double out[3]) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (patch != 0) return fail(c, W5CT_ERR_ARG, "patch index %d out of range", patch);
    if (!out) return fail(c, W5CT_ERR_ARG, "null out");
    return speeds_impl(c, out);
}

int w5ct_cfl_dt(w5ct_ctx *c, double *dt) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!dt) return fail(c, W5CT_ERR_ARG, "null dt");
    double S[3];
    rc = speeds_impl(c, S);
    if (rc) return rc;
    *dt = c->cfg.cfl / (S[0] / c->dx + S[1] / c->dy + S[2] / c->dz);
    return W5CT_OK;
}

int w5ct_div_b_norm(w5ct_ctx *c, int patch, double *linf, double *l2) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (patch != 0) return fail(c, W5CT_ERR_ARG, "patch index %d out of range", patch);
    if (!linf || !l2) return fail(c, W5CT_ERR_ARG, "null output");
    const size_t n = (size_t)c->n;
    divb_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->nx, c->ny, c->nz, c->b0, c->b0 + n, c->b0 + 2 * n,
                                                                   1.0 / c->dx, 1.0 / c->dy, 1.0 / c->dz, c->part);
    finalize_kernel<<<1, kRedThreads, 0, c->stream>>>(c->part, kRedBlocks, 2, 2, 1u, c->red_out);
    c->launches += 2;
    W5_CUDA(c, cudaGetLastError());
    double out[2];
    W5_CUDA(c, cudaMemcpyAsync(out, c->red_out, sizeof(out), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    *linf = out[0];
    *l2 = sqrt(out[1] / (double)c->n);
    return W5CT_OK;
}

int w5ct_conserved_totals(w5ct_ctx *c, int patch, double out[8]) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (patch != 0) return fail(c, W5CT_ERR_ARG, "patch index %d out of range", patch);
    if (!out) return fail(c, W5CT_ERR_ARG, "null out");
    const size_t n = (size_t)c->n;
    const double *pl[8];
    for (int f = 0; f < 5; ++f) pl[f] = c->q0 + f * n;
    for (int f = 0; f < 3; ++f) pl[5 + f] = c->b0 + f * n;
    W5_CUDA(c, cudaMemcpyAsync((void *)c->planes, pl, sizeof(pl), cudaMemcpyHostToDevice, c->stream));
    sums_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, 8, c->planes, c->part);
    finalize_kernel<<<1, kRedThreads, 0, c->stream>>>(c->part, kRedBlocks, 8, 8, 0u, c->red_out);
    c->launches += 2;
    W5_CUDA(c, cudaGetLastError());
    W5_CUDA(c, cudaMemcpyAsync(out, c->red_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    W5_CUDA(c, cudaStreamSynchronize(c->stream));
    const double dv = c->dx * c->dy * c->dz;
    for (int f = 0; f < 8; ++f) out[f] *= dv;
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
    if (nonphysical) *nonphysical = f;
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
    *launches = (long long)(c->ev_used / 2);
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
