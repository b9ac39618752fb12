/*
 * w5ct.h -- C ABI of libw5ct, a GB300 (sm_103a) implementation of the
 * fifth-order finite-difference WENO + constrained-transport ideal-MHD
 * scheme of Donnert et al., "WENO-Wombat" (arXiv:1812.04278).
 *
 * One context advances one or more independent periodic patches with the
 * paper's scheme:
 *   - the per-axis characteristic flux update (Sec. 2.2, Eq. FWENO, with
 *     the eigenvectors of Appendix A and local Lax-Friedrichs splitting),
 *   - the Ryu et al. transport-flux CT update of the face fields
 *     (Sec. 2.3, Eqs. fct1-fct6, ox1-ox3),
 *   - the classical four-stage RK4 (Sec. 2.1) interleaved with CT
 *     (Sec. 3.1.3), and the CFL time step (Sec. 2.1, Eq. cfl).
 *
 * Conventions shared by every call
 *   Grid: periodic, nx*ny*nz cells, x fastest: cell (i,j,k) has linear
 *     index i + nx*(j + ny*k).  Cell spacings dx, dy, dz.
 *   Conserved cell state "cons": 5 planes of nx*ny*nz doubles, in the order
 *     rho, m_x, m_y, m_z, E (E = total energy, Eq. P).
 *   Face field "bface": 3 planes: b_x at the face (i+1/2, j, k), b_y at
 *     (i, j+1/2, k), b_z at (i, j, k+1/2), each stored at the index of
 *     cell (i, j, k) (the forward face, Sec. 2.3).
 *   Cell field "bcell": 3 planes of the fourth-order face-to-centre
 *     interpolation of bface (Sec. 2.3).
 *   Pointers marked "host or device" are read or written only during the
 *     call; when on_device != 0 they must be device pointers of the current
 *     device, else host pointers.  The library never keeps a caller pointer.
 *   Ownership: the context owns every device buffer it allocates
 *     (cudaMalloc at w5ct_init_grid, cudaFree at w5ct_destroy / re-init).
 *   Streams: all device work is enqueued on the stream given in the
 *     config (a cudaStream_t, NULL = legacy default stream).  Calls that
 *     return values to the host synchronise that stream; w5ct_step* do not.
 *   Errors: every call returns 0 (W5CT_OK) or a negative code below; the
 *     text of the last error is available from w5ct_last_error.  No call
 *     throws, traps or aborts.  A state that becomes non-physical inside a
 *     step (rho <= 0, P <= 0 or NaN after the optional floors) raises a
 *     device flag that the next synchronising call reports as
 *     W5CT_ERR_NONPHYSICAL.
 */
#ifndef W5CT_H
#define W5CT_H

#ifdef __cplusplus
extern "C" {
#endif

#define W5CT_OK 0
#define W5CT_ERR_ARG (-1)          /* invalid argument (null pointer, bad size, dt <= 0, ...) */
#define W5CT_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define W5CT_ERR_STATE (-3)        /* call out of order (e.g. step before set_state) */
#define W5CT_ERR_NONPHYSICAL (-4)  /* rho <= 0, P <= 0 or NaN met inside the scheme */
#define W5CT_ERR_UNSUPPORTED (-5)  /* valid request this build does not implement */
#define W5CT_ERR_TIMEOUT (-6)      /* a bounded device wait of the fused step expired (the
                                      state of that step is not valid) */

#define W5CT_WENO_JS 0             /* Jiang-Shu weights, eps = 1e-6 (Sec. 2.2) */
#define W5CT_WENO_Z 1              /* WENO-Z weights (Sec. 2.2), ratio squared */

#define W5CT_FP64 0                /* every operation in IEEE double */
#define W5CT_FP32_BULK 1           /* flux, eigen and WENO arithmetic in float;
                                      RK stage accumulation, CT EMF accumulation
                                      into the face field and all reductions in
                                      double */
#define W5CT_FP64_DW 2             /* W5CT_FP64 with the WENO part of each
                                      characteristic field's flux (smoothness
                                      indicators, nonlinear weights and the two
                                      interpolants of the LF-split differences;
                                      Sec. 2.2) in double-word arithmetic (pairs
                                      of floats, 48-bit significand) on the FP32
                                      pipe, in the single-patch sweeps of the
                                      default tiles; everything else, every
                                      stored value and every other kernel
                                      (grids too small for those tiles, the
                                      batched, fused and adjoint paths) as
                                      W5CT_FP64 */

typedef struct w5ct_ctx w5ct_ctx;

typedef struct {
    double gamma;        /* adiabatic index (5/3 in the paper's tests) */
    double cfl;          /* Courant number of Eq. (cfl) (0.8 in the paper) */
    int weno_variant;    /* W5CT_WENO_JS or W5CT_WENO_Z */
    int precision;       /* W5CT_FP64, W5CT_FP32_BULK or W5CT_FP64_DW */
    double eps_js;       /* JS epsilon, 1e-6 (Sec. 2.2) */
    double eps_z;        /* WENO-Z epsilon, 1e-40 (Sec. 2.2); FP32_BULK uses
                            max(eps_z, 1e-30) because 1e-40 is subnormal in float */
    double eps_b;        /* degeneracy threshold eps_B, 1e-30 (Appendix A) */
    int floors;          /* 0: none (the paper's default, Sec. 4); 1: rho and P
                            are floored inside primitive recovery only */
    double rho_min;      /* density floor when floors = 1 */
    double p_min;        /* pressure floor when floors = 1 */
    void *stream;        /* cudaStream_t for all device work; NULL = default */
} w5ct_config;

/* Fill *cfg with the paper's defaults: gamma 5/3, CFL 0.8, WENO-Z, FP64,
 * eps 1e-6 / 1e-40 / 1e-30, no floors, default stream. */
int w5ct_config_default(w5ct_config *cfg);

/* Create a context on the current CUDA device.  *out receives the handle.
 * Errors: W5CT_ERR_ARG for a null pointer, gamma <= 1, cfl <= 0 or an
 * unknown variant / precision. */
int w5ct_create(const w5ct_config *cfg, w5ct_ctx **out);

/* Free every device buffer and the context.  ctx may be NULL. */
int w5ct_destroy(w5ct_ctx *ctx);

/* Replace the stream all later device work is enqueued on. */
int w5ct_set_stream(w5ct_ctx *ctx, void *stream);

/* Allocate npatch >= 1 independent periodic patches (the paper's patches,
 * Sec. 3; here each is its own periodic box, with no exchange between them).
 * n3 = {nx, ny, nz} per patch (npatch x 3 ints, each >= 1) and dx3 = {dx, dy,
 * dz} per patch (npatch x 3 doubles > 0), host pointers.  With npatch > 1
 * every step advances all patches together, each kernel launch covering the
 * tiles of every patch; each patch then holds at most 2^30 cells.  Previous
 * buffers are freed. */
int w5ct_init_grid(w5ct_ctx *ctx, int npatch, const int *n3, const double *dx3);

/* Load the state q^n of patch `patch` (0 .. npatch-1): cons (5 planes) and
 * bface (3 planes) of that patch's size, host or device (on_device).  Every
 * patch needs a state before the first step.  The face field should be discretely
 * divergence-free; the scheme keeps its divergence at round-off (Sec. 2.3)
 * but does not remove an initial one. */
int w5ct_set_state(w5ct_ctx *ctx, int patch, const double *cons, const double *bface, int on_device);

/* Read the state back; any of cons / bface / bcell may be NULL.  Synchronises.
 * Returns W5CT_ERR_TIMEOUT if a wait of a fused step (schedule 2) expired
 * since the last check, and W5CT_ERR_NONPHYSICAL if a step met a non-physical
 * state (in both cases the buffers are still written). */
int w5ct_get_state(w5ct_ctx *ctx, int patch, double *cons, double *bface, double *bcell, int on_device);

/* One full RK4 + CT step of size dt > 0 (Secs. 2.1, 2.3, 3.1.3) of every
 * patch: four stages of x-, y- and z-sweeps of the characteristic WENO
 * flux, the transport-flux corrections and corner EMFs, the face-field
 * update and the fourth-order face-to-centre interpolation.  Asynchronous. */
int w5ct_step(w5ct_ctx *ctx, double dt);

/* As w5ct_step with the dt of patch p read from device memory at dt_dev[p]
 * (npatch doubles, read by the kernels when they run), so a sequence of
 * steps can be captured in a CUDA graph. */
int w5ct_step_dev(w5ct_ctx *ctx, const double *dt_dev);

/* One step in which every patch takes its own dt = CFL / sum_d (S_d / dx_d),
 * computed on the device from its current state (Eq. cfl, with S_d from
 * w5ct_max_signal_speed); no host synchronisation.  If dt_dev_out is not
 * NULL the dts used are also written there (device pointer, npatch doubles). */
int w5ct_step_cfl(w5ct_ctx *ctx, double *dt_dev_out);

/* nsteps >= 0 steps as w5ct_step_cfl(ctx, NULL), replayed from a CUDA graph
 * of one step that the first call captures (on a private stream) and later
 * calls reuse; the graph is launched on the context's stream.  The graph is
 * dropped by w5ct_init_grid and w5ct_destroy.  Asynchronous. */
int w5ct_step_graph(w5ct_ctx *ctx, int nsteps);

/* Tile shapes of the batched sweeps (npatch > 1; no counterpart in the
 * paper, whose sweeps run over one patch's pencils).  Each patch is swept
 * along each axis in tiles of BX cells along x times T2 faces or pencils in
 * the second direction, one of these variants:
 *   0: BX = 32, T2 = 16 (FP32_BULK and FP64, every axis)
 *   1: BX = 16, T2 = 16      2: BX = 8, T2 = 16      3: BX = 8, T2 = 8
 * (variants 1-3 in FP32_BULK only).  The variant changes only which threads
 * compute a face, never its arithmetic: results are bit for bit the same.
 * mode = W5CT_TUNE_MEASURE times every variant on every class of patches
 * with the same (nx, ny) (x- and y-sweeps) or (nx, nz) (z-sweep) on the
 * current state, `reps` timed launches each, and keeps the fastest per class
 * (synchronises; needs a state; the flux buffers are overwritten, counters
 * kept) and then the fastest step schedule (w5ct_set_sweep_schedule),
 * timed on whole steps from a snapshot of the state that is put back.
 * mode = W5CT_TUNE_MODEL (the choice w5ct_init_grid makes) takes
 * the variant with the fewest padded lanes and rows per face.  mode = v >= 0
 * forces variant v on every patch.  A captured step graph is dropped.  With
 * npatch = 1 this does nothing and returns W5CT_OK. */
#define W5CT_TUNE_MEASURE (-1)
#define W5CT_TUNE_MODEL (-2)
int w5ct_autotune(w5ct_ctx *ctx, int mode, int reps);

/* Schedule of a batched step (npatch > 1; no counterpart in the paper).
 * 0 (the default after w5ct_init_grid): per stage, one launch per axis and
 * tile variant over all patches' tiles, then one update launch.  1: per
 * stage, one persistent launch per tile variant, as many blocks as fit on the
 * device at once, each block taking tiles of all three axes from a device
 * work queue (an atomically incremented counter, zeroed at the start of every
 * step) until the list is exhausted; no block waits on another.  2: the
 * whole step (cell fields, CFL reduction and dt, the sweeps in 32- or
 * 16-lane tiles, the four stage updates) in one persistent launch over a
 * work queue in which each item waits, with bounded spins, for the earlier
 * items of its own patch that it depends on; an expired wait aborts the
 * launch and the next synchronising call returns W5CT_ERR_TIMEOUT.  Every face and cell is
 * computed from the same source in all schedules; the compiler may contract a
 * few operations differently in the fused kernels, so the results agree to
 * rounding (not bit for bit).  w5ct_autotune(W5CT_TUNE_MEASURE) times whole
 * steps of the three and keeps the fastest.  Changing the schedule drops a
 * captured step graph.  W5CT_ERR_UNSUPPORTED for schedules 1 and 2 with one
 * patch. */
int w5ct_set_sweep_schedule(w5ct_ctx *ctx, int schedule);
int w5ct_sweep_schedule(w5ct_ctx *ctx, int *schedule);

/* Check of the fused step's failure path (npatch > 1, state set; any
 * schedule): launches the fused kernel on a one-item work list whose
 * dependency nothing satisfies, each wait bounded by spin_limit sleeps of
 * 256 ns (1 <= spin_limit <= 2^22).  The wait expires, the launch aborts and
 * ends, and *status receives what a synchronising call then reports
 * (W5CT_ERR_TIMEOUT when the bound works).  The state is not touched and the
 * context's flag is restored afterwards.  Synchronises the stream. */
int w5ct_fused_wait_check(w5ct_ctx *ctx, long long spin_limit, int *status);

/* out[3] = {variant, BX, T2} of the tiles that sweep patch `patch` along
 * `axis` (0, 1, 2).  Host only. */
int w5ct_tile_variant(w5ct_ctx *ctx, int axis, int patch, int out[3]);

/* Adjoint of one step (one patch): the vector-Jacobian product of the map
 * (q^n, b^n) -> (q^{n+1}, b^{n+1}) of w5ct_step(ctx, dt) at the current state.
 * lam_q (5 planes) = dL/dq^{n+1}, lam_b (3 planes) = dL/db^{n+1} in, lam_q_out
 * = dL/dq^n, lam_b_out = dL/db^n out; all device pointers to doubles in the
 * layout of w5ct_set_state, outputs distinct from the inputs.  dt is held
 * fixed (the CFL dt's dependence on the state is not differentiated).  The
 * stages are recomputed from the state (Sec. 2.1), then run backwards: the
 * linear maps (flux divergence, Eq. num; EMF averages, Eqs. ox1-ox3; face
 * update, Sec. 2.3; cell-field interpolation) by their transposes, each
 * sweep by the Jacobian of its face function (cell recovery + Appendix A
 * eigenvectors + LF splitting + WENO, Sec. 2.2) contracted with the flux
 * adjoints.  At max(), |.| and the eps_B switches the derivative is that of
 * the branch the forward step takes.  The arithmetic type of the forward
 * path is kept (float Jacobians for FP32_BULK), accumulation is double.
 * The state is not changed; the floor-hit counter and flag are kept.
 * Synchronises.  W5CT_ERR_UNSUPPORTED for npatch > 1.  (No counterpart in
 * the paper.) */
int w5ct_adjoint_step(w5ct_ctx *ctx, double dt, const double *lam_q, const double *lam_b, double *lam_q_out,
                      double *lam_b_out);

/* L = 1/2 dV sum over the cells of |q - q*|^2 + |b - b*|^2 (five conserved
 * and three face fields of the current state against target_cons,
 * target_bface; dV = dx dy dz) into *value (host), and its gradient dV (q -
 * q*), dV (b - b*) into lam_q, lam_b (device planes).  Fixed summation
 * order.  Synchronises.  One patch. */
int w5ct_misfit(w5ct_ctx *ctx, const double *target_cons, const double *target_bface, double *value, double *lam_q,
                double *lam_b);

/* Initial state from primitive fields and an edge vector potential (no
 * context): b = curl A + B0 with the first-order discrete curl of Sec. 4.1
 * (A_x at (i, j+1/2, k+1/2), A_y at (i+1/2, j, k+1/2), A_z at (i+1/2, j+1/2,
 * k) in cell units from the centre of cell (i, j, k)), cons = (rho, rho v, E)
 * with E from Eq. P and the cell field from the sixth-order face-to-centre
 * interpolation of Sec. 4.14.  rho, P: 1 plane; v, A: 3 planes; cons 5,
 * bface 3 planes out; device pointers, n3 = {nx, ny, nz}, dx3 and B0 on the
 * host; `stream` a cudaStream_t or NULL.  Asynchronous. */
int w5ct_ic_from_potential(const int n3[3], const double dx3[3], double gamma, const double B0[3], const double *rho,
                           const double *v, const double *P, const double *A, double *cons, double *bface,
                           void *stream);

/* Adjoint of w5ct_ic_from_potential in (rho, v, A) with P and B0 fixed:
 * given lam_cons (5 planes) and lam_bface (3 planes), writes lam_rho (1),
 * lam_v (3), lam_A (3) and the total face-field adjoint lam_b (3 planes).
 * bface is the forward output.  Device pointers.  Asynchronous. */
int w5ct_ic_from_potential_adjoint(const int n3[3], const double dx3[3], const double *rho, const double *v,
                                   const double *bface, const double *lam_cons, const double *lam_bface,
                                   double *lam_rho, double *lam_v, double *lam_A, double *lam_b, void *stream);

/* For patch `patch`: S_d = max over its cells of |v_d| + c_fast^d for d = x, y, z (Eq. cfl; the
 * fast speed of Eq. fast with B_n = B_d), out[3] on the host.  Synchronises.
 * FP32_BULK evaluates the speeds in float. */
int w5ct_max_signal_speed(w5ct_ctx *ctx, int patch, double out[3]);

/* dt = CFL / sum_d (S_d / dx_d) on the host, the smallest over the
 * patches (the common dt of a lockstep advance).  Synchronises. */
int w5ct_cfl_dt(w5ct_ctx *ctx, double *dt);

/* Discrete divergence of the face field of patch `patch` at cell centres,
 * (b_x(i) - b_x(i-1))/dx + (b_y(j) - b_y(j-1))/dy + (b_z(k) - b_z(k-1))/dz:
 * *linf its maximum modulus, *l2 its root mean square.  FP64, deterministic.
 * Synchronises. */
int w5ct_div_b_norm(w5ct_ctx *ctx, int patch, double *linf, double *l2);

/* Volume integrals over patch `patch` (sum * dx*dy*dz) of rho, m_x, m_y, m_z, E, b_x, b_y, b_z
 * in out[8] (host).  FP64, fixed summation order (deterministic).
 * Synchronises. */
int w5ct_conserved_totals(w5ct_ctx *ctx, int patch, double out[8]);

/* Number of floor activations (when floors = 1) and the non-physical flag
 * since the last set_state; either pointer may be NULL.  Synchronises. */
int w5ct_status(w5ct_ctx *ctx, long long *floor_hits, int *nonphysical);

/* Block the host until all work of the context's stream is done. */
int w5ct_synchronize(w5ct_ctx *ctx);

/* Kernel timing: when enabled, each launch of the characteristic sweep
 * kernel is bracketed by CUDA events on the context's stream.
 * w5ct_sweep_timing returns the number of sweep launches and their summed
 * device time in milliseconds since timing was last enabled (synchronises). */
int w5ct_set_timing(w5ct_ctx *ctx, int enable);
int w5ct_sweep_timing(w5ct_ctx *ctx, long long *launches, double *total_ms);

/* Number of kernel launches the context has issued since it was created. */
int w5ct_launch_count(w5ct_ctx *ctx, long long *launches);

/* Text of the last error of ctx (or, when ctx is NULL, of the last failed
 * call that has no context: w5ct_create, w5ct_conserved_totals_noalloc).
 * Never NULL; valid until the next call on ctx. */
const char *w5ct_last_error(const w5ct_ctx *ctx);

/* Largest grid (cells) w5ct_conserved_totals_noalloc accepts: 512^3. */
#define W5CT_NOALLOC_MAX_CELLS 134217728LL

/* The reduction of w5ct_conserved_totals for callers that cannot allocate
 * device memory: frameworks that reserve all device memory at start-up and
 * forbid later allocations, and real-time host loops that cannot take the
 * implicit synchronisation of cudaMalloc.  The call copies the totals to the
 * host and synchronises its stream, so it cannot be enqueued on a stream
 * that is being captured.  The paper has no counterpart; it is a
 * convenience of this library.
 *   cons   device pointer, 5 planes of nx*ny*nz doubles (rho, m_x, m_y, m_z, E)
 *   bface  device pointer, 3 planes (b_x, b_y, b_z on the forward faces)
 *   out    host pointer to 8 doubles: the volume integrals, as in
 *          w5ct_conserved_totals (fixed summation order, deterministic)
 *   stream cudaStream_t the work is enqueued on (NULL = default); the call
 *          synchronises it before returning.
 * No context is needed and nothing is allocated: the partial sums live in a
 * fixed 512 KB device array inside the library, which every GPU that loads
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and keeps it
 * for later calls on that device; the kept address is void after the
 * device is reset (cudaDeviceReset), which this library never does.  All
 * calls share the array, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Errors: W5CT_ERR_ARG for null
 * pointers, sizes < 1, spacings <= 0 or more than W5CT_NOALLOC_MAX_CELLS
 * cells (text via w5ct_last_error(NULL)); W5CT_ERR_CUDA. */
int w5ct_conserved_totals_noalloc(const double *cons, const double *bface, int nx, int ny, int nz,
                                  double dx, double dy, double dz, double out[8], void *stream);

#ifdef __cplusplus
}
#endif
#endif /* W5CT_H */
