/*
 * gks.h -- C ABI of the GB300 library for the fifth-order TENO-D gas-kinetic
 * scheme (GKS) with two-stage fourth-order (S2O4) time stepping on structured
 * 1-D and 2-D grids.
 *
 * The problem solved is the conservation law W_t = -div F(W), W(0,x) = W0(x)
 * (paper Sec. 2.2) for the Euler and Navier-Stokes equations of an ideal gas,
 * with W = (rho, rho U, rho V, rho E) in 2-D and (rho, rho U, rho E) in 1-D.
 * One S2O4 step = two stages; each stage reconstructs every cell interface
 * with TENO-D (Sec. 4.2, Eqs. 4.5-4.14; 2-D by the dimension-by-dimension
 * steps of Sec. 3.2 at two Gauss points), merges the two sides into the
 * equilibrium state (Eqs. 2.6, 3.25, 3.26), evaluates the time-dependent BGK
 * flux (Eqs. 2.5, 2.7, 2.9, 2.12) and updates the cells (Sec. 2.2).
 *
 * Conventions for every call:
 *   - Return value: GKS_OK or an error code; gks_last_error() gives text.
 *     No call throws or aborts across this boundary.
 *   - Arrays of cell data are conserved variables, float64, interior cells
 *     only, layout SoA [nvar][ny][nx] row-major (x fastest); nvar = dim + 2,
 *     ny = 1 in 1-D.  The library keeps its own ghosted device copy.
 *   - on_device = 0: pointer is host memory (pageable or pinned); the call
 *     copies and synchronises.  on_device = 1: pointer is device memory owned
 *     by the caller (e.g. a torch tensor's data_ptr) on the current device;
 *     it must stay valid until the call returns.
 *   - All device work is ordered on the context stream (gks_set_stream; the
 *     default is the legacy default stream).  Calls that return host data
 *     synchronise that stream.
 *   - A context is not thread safe; separate contexts are independent.
 *   - The library owns and frees all device memory it allocates.
 */
#ifndef GKS_H
#define GKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gks_ctx gks_ctx;

typedef enum {
    GKS_OK = 0,
    GKS_EINVAL = 1,          /* bad argument (null pointer, size, enum value) */
    GKS_ENOMEM = 2,          /* device or host allocation failed */
    GKS_ECUDA = 3,           /* a CUDA runtime call failed */
    GKS_ENONPHYSICAL = 4,    /* rho <= 0, p <= 0 or non-finite state seen by a kernel */
    GKS_ETIMEOUT = 5,        /* a bounded device-side wait gave up */
    GKS_EUNSUPPORTED = 6     /* valid request the library does not implement */
} gks_status;

/* ghost-layer boundary conditions (paper Sec. 5: periodic, non-reflecting,
 * reflective, symmetric, no-slip adiabatic walls) */
typedef enum {
    GKS_BC_PERIODIC = 0,
    GKS_BC_ZEROGRAD = 1,     /* "non-reflecting": copy of the edge cell */
    GKS_BC_SYMMETRY = 2,     /* mirror, normal velocity negated */
    GKS_BC_NOSLIP = 3,       /* mirror, both velocity components negated (adiabatic wall) */
    GKS_BC_REFLECT = 4,      /* same ghost rule as GKS_BC_SYMMETRY */
    /* State-setting rules (the double Mach reflection, Sec. 5.7), with the
     * states of gks_set_boundary_states; ghost cells are judged by their
     * centres, W* ghosts at t + dt/2. */
    GKS_BC_INFLOW = 5,        /* every ghost = the inflow state */
    GKS_BC_WALL_AFTER_X0 = 6, /* y sides: the inflow state where x < shock_x0, reflecting wall beyond */
    GKS_BC_MOVING_SHOCK = 7   /* y sides: the inflow state behind the moving oblique shock
                                 x_s(y, t) = shock_x0 + (y - y0) cot(theta) + speed t / sin(theta),
                                 the pre-shock state ahead of it */
} gks_bc;

/* States and shock of the state-setting boundary rules: conserved
 * (rho, rho u, rho v, E); 1-D grids use (rho, rho u, -, E) of the same four
 * slots. */
typedef struct {
    double inflow[4];        /* GKS_BC_INFLOW ghosts; behind the shock */
    double pre[4];           /* ahead of the shock */
    double shock_x0;         /* where the shock meets y = y0 at t = 0 */
    double shock_theta;      /* angle of the shock line to the x-axis, radians, in (0, pi) */
    double shock_speed;      /* normal speed of the shock */
} gks_boundary_states;

typedef enum {
    GKS_FP64 = 0,            /* every step in float64 */
    GKS_FP32_FLUX = 1        /* reconstruction + flux in float32, state and S2O4 accumulation in float64 */
} gks_precision;

/* collision time (Sec. 5): 0 -> tau = 0 (smooth inviscid tests),
 * Euler: tau = c1 dt + c2 |pl-pr|/(pl+pr) dt, NS: tau = mu/p + c2 |pl-pr|/(pl+pr) dt */
typedef enum { GKS_TAU_ZERO = 0, GKS_TAU_EULER = 1, GKS_TAU_NS = 2 } gks_tau_mode;

typedef struct {
    int dim;                 /* 1 or 2 */
    int nx, ny;              /* interior cells; ny ignored (= 1) in 1-D; each >= 3 */
    double x0, x1, y0, y1;   /* domain; uniform cells dx = (x1-x0)/nx, dy = (y1-y0)/ny */
    int bc[4];               /* gks_bc for x-low, x-high, y-low, y-high */
    int precision;           /* gks_precision */
} gks_grid_desc;

typedef struct {
    double gamma;            /* ratio of specific heats (default 1.4) */
    double mu;               /* dynamic viscosity, used by GKS_TAU_NS and the viscous time step */
    double Pr;               /* Prandtl number; 1 disables the heat-flux correction */
} gks_gas;

typedef struct {
    double cfl;              /* dt = cfl * min(h/(|U|+a), h^2/(4 nu)), h = min(dx,dy)  (Sec. 5) */
    double c1, c2;           /* collision-time constants (Sec. 5; defaults 0.01, 1) */
    double ct1, ct2;         /* TENO-D cut-offs C_T1, C_T2 normal to the face (Eqs. 4.7, 4.12) */
    double ct1_t, ct2_t;     /* cut-offs of the tangential (Gauss-point) reconstruction */
    double eps;              /* epsilon of Eq. (4.5) (default 1e-40; float32 path clamps to FLT_MIN) */
    int q;                   /* power of Eq. (4.5), integer >= 1 (default 7); TENO5: of Eq. (4.1) */
    int tau_mode;            /* gks_tau_mode */
    int positivity_fallback; /* 1: a reconstructed point state with rho<=0 or p<=0 is replaced
                                by the adjacent cell average with zero slopes (not in the paper) */
    int recon;               /* gks_recon: TENO-D (default) or WENO5-AO */
    double d_hi, d_lo;       /* WENO5-AO linear-weight parameters (Sec. 3.2; default 0.85, 0.85) */
    double eps_ao;           /* WENO5-AO and WENO5-Z epsilon (default 1e-8) */
    int merge;               /* gks_merge: equilibrium state at the interface (default kinetic) */
    int charvars;            /* 1: normal reconstruction in characteristic variables (Sec. 3.1; see
                                below), 0: component-wise on the conserved variables (default) */
} gks_scheme;

/* Reconstruction of the non-equilibrium states (values and slopes at the
 * faces, values at the Gauss points): TENO-D (Sec. 4.2, the paper's scheme)
 * or WENO5-AO (Sec. 3.2, the scheme it is compared with): adaptive-order
 * weights gamma_k (1 + (tau/(beta_k+eps))^2) on the quartic and the three
 * quadratics, gamma_3 = d_hi, gamma_1 = (1-d_hi) d_lo, gamma_0 = gamma_2 =
 * (1-d_hi)(1-d_lo)/2.  Batches and the adjoint take TENO-D only
 * (GKS_EUNSUPPORTED otherwise).
 * WENO5-Z and TENO5 (Sec. 3.1, 4.1) are the paper's conventional path: face
 * values from the three
 * quadratics with WENO-Z weights d_k (1 + tau/(beta_k + eps_ao)), tau =
 * |beta_0 - beta_2| (Eq. 3.5), or TENO5 weights (Eqs. 4.1-4.4: power q, the
 * paper's q = 6, cut-off ct1, epsilon eps); non-equilibrium slopes from the
 * quadratic through the cell average and both face values (Eq. 3.11); the
 * equilibrium state by the kinetic merge of the face values and its slope by
 * the linear Eq. (3.12); in 2-D the non-equilibrium values at the Gauss
 * points by WENO-Z / TENO5 across the rows, the equilibrium state and slopes
 * there by the quartic through the rows' line-averaged merges and Eq. (3.12)
 * slopes (Steps 2-4).  Set q = 6 for TENO5 (the default 7 is TENO-D's). */
typedef enum { GKS_RECON_TENO_D = 0, GKS_RECON_WENO_AO = 1, GKS_RECON_WENO_Z = 2, GKS_RECON_TENO5 = 3 } gks_recon;

/* Reconstruction variables (gks_scheme.charvars, Sec. 3.1: for Euler
 * systems the reconstructed quantities may be the characteristic variables;
 * the paper does not state the projection).  With charvars = 1 the normal
 * reconstruction of each face (in 2-D: of each row of its tangential
 * stencil) runs on C = L W: L = R^-1, R the right eigenvectors of the
 * Jacobian of the normal Euler flux in the face's local frame (normal
 * velocity first; eigenvalues U - c, U, [U,] U + c), evaluated at the
 * arithmetic mean of the two cells adjacent to the face in that row; each
 * characteristic field is reconstructed with TENO-D on its own and the
 * values and slopes are mapped back by R.  The 2-D tangential reconstruction
 * to the Gauss points stays component-wise.  Taken with GKS_RECON_TENO_D on
 * single grids only: other reconstructions, batches and the adjoint return
 * GKS_EUNSUPPORTED. */

/* Equilibrium state W0 and its slopes at an interface point (Sec. 3.2):
 * the kinetic weighting of Eqs. (3.25)-(3.26) (W0 = rho_l <psi>_{u>0} +
 * rho_r <psi>_{u<0}, likewise for the slopes; the paper's scheme), or the
 * arithmetic average of the two reconstructed sides, W0 = (W_l + W_r)/2,
 * W0_n = (W_l,n + W_r,n)/2, W0_t = (W_l,t + W_r,t)/2, which the paper allows
 * for smooth flow.  The non-equilibrium terms are the same either way.  The
 * adjoint takes the kinetic merge only (GKS_EUNSUPPORTED otherwise). */
typedef enum { GKS_MERGE_KINETIC = 0, GKS_MERGE_AVERAGE = 1 } gks_merge;

typedef struct {
    unsigned int error_word; /* bit 0: non-physical state after an update; bit 1: fallback failed */
    long long fallbacks;     /* positivity fallbacks taken since the state was last set */
    double t;                /* simulation time of the stored state */
    long long steps;         /* S2O4 steps taken since the state was last set */
    double dt;               /* the time step the next gks_advance_to step will use */
} gks_diag;

/* TENO-D selection flips between the two precisions (Sec. 4.2: the cut-offs
 * of Eqs. 4.7 and 4.12 act on ratios of smoothness indicators, so near a
 * discontinuity float32 rounding can move a choice; both choices are valid
 * results of the scheme).  Counts on one state: */
typedef struct {
    long long normal_flips;          /* normal selections (per cell, variable and sweep direction)
                                        where the float32 path chooses otherwise than the float64 path */
    long long normal_selections;     /* normal selections compared */
    long long tangential_flips;      /* 2-D: tangential selections (per face, side, variable, stream
                                        [value, normal slope] and direction), each precision on its own
                                        line averages; 0 in 1-D */
    long long tangential_selections; /* tangential selections compared */
    long long unresolved_flips;      /* flips on stencils whose data vary by less than 2^-16 of the
                                        magnitude of the quantity they resolve (cell and line averages:
                                        their own; line-averaged normal slopes: the values' over dx) --
                                        below float32 resolution: uniform regions, where float32
                                        rounding makes the data constant and the float64 choice follows
                                        round-off noise; no value changes beyond rounding.  Not included
                                        in the two counts above */
} gks_flip_count;

/* Create a context for one grid; allocates the ghosted device state.
 * Defaults: gamma 1.4, mu 0, Pr 1, cfl 0.5, c1 0.01, c2 1, C_T 1e-7/1e-5 in
 * both directions, eps 1e-40, q 7, tau Euler, positivity fallback on. */
gks_status gks_create(const gks_grid_desc *desc, gks_ctx **out);
void       gks_destroy(gks_ctx *ctx);
gks_status gks_set_gas(gks_ctx *ctx, const gks_gas *gas);
gks_status gks_set_scheme(gks_ctx *ctx, const gks_scheme *scheme);
/* Data of the state-setting boundary rules (default: all zero).  Copied. */
gks_status gks_set_boundary_states(gks_ctx *ctx, const gks_boundary_states *states);
/* cudaStream_t passed as void*; NULL = legacy default stream */
gks_status gks_set_stream(gks_ctx *ctx, void *stream);

/* Where a state array lives (on_device of gks_set_state / gks_get_state /
 * gks_get_buffer and the batch calls): */
#define GKS_HOST_MEMORY 0        /* host memory; the call returns when the copy is done */
#define GKS_DEVICE_MEMORY 1      /* device memory */
#define GKS_HOST_PINNED_ASYNC 2  /* page-locked host memory, gks_set_state / gks_get_state only: the
                                    copy is enqueued on the context's stream and the call returns at
                                    once; the caller keeps W unchanged (set) or unread (get) until the
                                    stream has passed it (cudaStreamSynchronize or an event).  With
                                    two contexts on two streams, one's copies overlap the other's
                                    steps.  Other values: GKS_EINVAL */

/* Copy conserved cell averages in / out ([nvar][ny][nx], float64).
 * gks_set_state resets t, step count, fallback count and the error word. */
gks_status gks_set_state(gks_ctx *ctx, const double *W, int on_device);
gks_status gks_get_state(gks_ctx *ctx, double *W, int on_device);
/* which: 0 = W (state), 1 = W* (stage-1 output), 2 = stage accumulator
 * W^n - dt/dx dF(W^n) (Sec. 2.2); same layout as gks_get_state.  On the 2-D
 * GKS_FP32_FLUX path W* is held in float32 and the accumulator as a float32
 * increment of W; this call widens them (valid between stage 1 and stage 2). */
gks_status gks_get_buffer(gks_ctx *ctx, int which, double *W, int on_device);

/* CFL time step of the current state (Sec. 5); synchronises. */
gks_status gks_compute_dt(gks_ctx *ctx, double *dt);
/* One S2O4 stage with step dt > 0: stage 1 reads W and writes W* and the
 * accumulator; stage 2 reads W* and the accumulator and writes W. */
gks_status gks_stage(gks_ctx *ctx, int stage, double dt);
/* One S2O4 step; dt <= 0 uses the CFL time step of the current state.
 * Asynchronous; errors flagged by kernels surface at the next synchronising call. */
gks_status gks_step(gks_ctx *ctx, double dt);
/* Advance with CFL steps until t_end (last step clipped to t_end) or
 * max_steps (<= 0: no limit).  Time and step are kept on the device; the
 * loop runs as CUDA-graph replays.  Synchronises. */
gks_status gks_advance_to(gks_ctx *ctx, double t_end, long long max_steps,
                          long long *steps_done, double *t_out);
gks_status gks_get_diagnostics(gks_ctx *ctx, gks_diag *out);

/* Selection flips on the context's current state W (the input of the next
 * step's first stage): the stencil choices of the float32 path (state
 * rounded to float32, the float32 kernels' arithmetic) compared with the
 * float64 path's, every normal and, in 2-D, tangential selection of both
 * sweep directions.  Fills W's ghost layers; allocates and frees a 40-byte
 * counter; synchronises the context's stream.  TENO-D with component-wise
 * variables only (GKS_EUNSUPPORTED otherwise).  Either precision. */
gks_status gks_selection_flips(gks_ctx *ctx, gks_flip_count *out);
/* Text of the last error on this context (never NULL). */
const char *gks_last_error(const gks_ctx *ctx);
const char *gks_status_string(int status);
/* Number of kernel launches this context has issued (graph replays count
 * every kernel node). */
long long  gks_kernel_launches(const gks_ctx *ctx);

/* ---- batched ensemble of independent 1-D problems ---- */

/* A batch holds `count` independent 1-D problems, problem k on [0, lengths[k]]
 * with ncells[k] >= 3 uniform cells and zero-gradient ("non-reflecting",
 * Sec. 5.2) ends, all with the same gas and scheme.  gks_batch_advance_to
 * advances every problem to t_end with its own CFL time steps (Sec. 5) in ONE
 * persistent kernel launch, replayed as a CUDA graph: each block takes the
 * next problem from an atomic queue ordered by decreasing estimated cost
 * (n^2 * max signal speed / length) and runs it to t_end alone.
 * States are packed [3][sum ncells] float64 (rho, rho U, rho E), problem k
 * starting at cell sum_{j<k} ncells[j]; on_device as for gks_set_state. */
typedef struct gks_batch gks_batch;
gks_status gks_batch_create(int count, const int *ncells, const double *lengths, int precision,
                            gks_batch **out);
void       gks_batch_destroy(gks_batch *b);
gks_status gks_batch_set_gas(gks_batch *b, const gks_gas *gas);
gks_status gks_batch_set_scheme(gks_batch *b, const gks_scheme *scheme);
gks_status gks_batch_set_stream(gks_batch *b, void *stream);
/* resets every problem's time, steps, error word; recomputes the cost order */
gks_status gks_batch_set_state(gks_batch *b, const double *W, int on_device);
gks_status gks_batch_get_state(gks_batch *b, double *W, int on_device);
/* max_steps: per problem and call (<= 0: none).  Synchronises.  A problem
 * whose cell averages leave the physical set (rho <= 0 or p <= 0) stops at the
 * end of the step that produced them, keeping that state, its time and step
 * count, with bit 0 of its error word set; the other problems still advance to
 * t_end.  Returns GKS_ENONPHYSICAL if any problem is flagged (count in
 * gks_batch_last_error; which ones in gks_batch_get_progress). */
gks_status gks_batch_advance_to(gks_batch *b, double t_end, long long max_steps);
/* per-problem arrays of length count (any may be NULL) */
gks_status gks_batch_get_progress(gks_batch *b, double *t, long long *steps, unsigned int *err,
                                  long long *fallbacks);
/* launch shape: threads per block 128 or 256, blocks per SM 1..16 */
gks_status gks_batch_set_launch(gks_batch *b, int threads, int blocks_per_sm);
/* Autotuner: times every launch shape (threads 128/256 x 1/2/4/8 blocks per
 * SM) advancing the stored state to t_probe, restores the state, applies the
 * fastest and appends it to a cache file ($GKS_TUNE_CACHE, else
 * ~/.cache/gks_batch_tune.txt) keyed by device, precision, collision model,
 * count and total cells; use_cache = 1 applies a cached entry without timing. */
gks_status gks_batch_tune(gks_batch *b, double t_probe, int use_cache, int *threads, int *blocks_per_sm,
                          double *best_ms);
const char *gks_batch_last_error(const gks_batch *b);
long long  gks_batch_launches(const gks_batch *b);

/* ---- discrete adjoint (2-D, collision-free flux) ---- */

/* Hand-written reverse mode of the 2-D S2O4 step with fixed dt (Sec. 2.2)
 * for the collision-free flux (tau_mode = GKS_TAU_ZERO, the paper's setting
 * for smooth inviscid flow, Sec. 5.1 and 5.5): the transposed Jacobians of
 * the two stages, of the Gauss-point flux (kinetic merge, Euler flux and its
 * compatibility time derivative) and of the TENO-D reconstructions with the
 * stencil selection of the forward pass held fixed, and of the ghost fill.
 * An adjoint object belongs to one context (2-D, tau_mode zero; otherwise
 * GKS_EUNSUPPORTED) and uses that context's state and stream.
 * checkpoint_every = k >= 1: the forward pass keeps W every k steps; the
 * backward pass recomputes one k-step segment at a time, keeping W and W* of
 * each of its steps (device memory: ceil(nsteps/k) + 2k + 6 state-sized
 * arrays plus scratch of about 116 x nx x ny values of the working
 * precision). */
typedef struct gks_adjoint gks_adjoint;
gks_status gks_adjoint_create(gks_ctx *ctx, int checkpoint_every, gks_adjoint **out);
void       gks_adjoint_destroy(gks_adjoint *adj);
/* nsteps steps of fixed dt from the context's current state, keeping
 * checkpoints; leaves the final state W_N in the context.  Synchronises;
 * GKS_ENONPHYSICAL as gks_step. */
gks_status gks_adjoint_forward(gks_adjoint *adj, int nsteps, double dt);
/* gW0 = (dW_N/dW_0)^T gWN for the last forward pass; gWN, gW0 interior
 * [nv][ny][nx] float64 (host, or device with on_device = 1).  Leaves the
 * context at W_N.  Synchronises. */
gks_status gks_adjoint_backward(gks_adjoint *adj, const double *gWN, double *gW0, int on_device);
/* Allocate up front what forward/backward passes of up to nsteps steps
 * need (checkpoints and segment states), so that they allocate nothing. */
gks_status gks_adjoint_reserve(gks_adjoint *adj, int nsteps);
/* kernel launches issued by the adjoint's own kernels (forward steps not counted) */
long long  gks_adjoint_launches(const gks_adjoint *adj);
/* One step's vector-Jacobian product: gin = (dS/dW)^T gout for the S2O4 step
 * S of fixed dt at state W (interior layout as above).  Sets the context's
 * state to S(W).  Allocates and frees a temporary adjoint object. */
gks_status gks_vjp_step(gks_ctx *ctx, const double *W, const double *gout, double *gin, double dt,
                        int on_device);

/* ---- measurement helpers (not part of the paper's method) ---- */

/* Per-kernel timing with CUDA events recorded on the context stream around
 * every directly launched kernel (not inside CUDA graphs).  kind: 0 = stage
 * kernels (2-D sweeps, 1-D stage), 1 = ghost fill, 2 = other (CFL
 * reduction, time commit, parameter kernels).  gks_profile_read synchronises,
 * returns launches and summed milliseconds since the last read, and clears. */
gks_status gks_profile_enable(gks_ctx *ctx, int enable);
gks_status gks_profile_read(gks_ctx *ctx, int kind, long long *launches, double *total_ms);

/* Algorithmic operation count of this library's own stage arithmetic, per
 * cell, obtained by replaying the device functions on the host with a
 * counting scalar (smooth-data branch: large stencil, closed-form time
 * coefficients).  Flops = add/sub + mul + div + sqrt (a fused multiply-add
 * counts 2); exp and erfc are counted separately. */
typedef struct {
    double flops_per_cell_update;            /* one full S2O4 step of one cell */
    double flops_per_cell_sweep;             /* one 2-D sweep (1-D: one stage) kernel, per cell */
    double transcendentals_per_cell_update;  /* exp + erfc */
    double divides_per_cell_update;
    double sqrt_per_cell_update;
    double fp64_flops_per_cell_update;       /* float64 share (all flops on the float64 path) */
} gks_flop_model;
gks_status gks_count_flops(int dim, int precision, int tau_mode, double Pr, gks_flop_model *out);
/* the same for either reconstruction (gks_recon), or GKS_COUNT_TENO_CHARVARS:
 * TENO-D in characteristic variables (gks_scheme.charvars = 1) */
#define GKS_COUNT_TENO_CHARVARS 4
gks_status gks_count_flops_recon(int dim, int precision, int tau_mode, double Pr, int recon,
                                 gks_flop_model *out);

/* Measured arithmetic peak of the current device: fused multiply-adds in 16
 * independent chains per thread on 8 blocks of 256 threads per SM, one launch
 * grown to about target_ms; *tflops counts 2 flops per FMA.  precision:
 * GKS_FP32_FLUX measures float32, GKS_FP64 float64.  Allocates and frees a
 * small output buffer; synchronises the device. */
gks_status gks_alu_peak(int precision, double target_ms, double *tflops);

/* ---- allocation-free 1-D step (the paper has no counterpart) ---- */

/* Largest grid gks_step1d_noalloc accepts. */
#define GKS_NOALLOC_MAX_NX 16384

/* One S2O4 step of a 1-D problem that allocates no device memory, for
 * callers that cannot call cudaMalloc: a host whose device memory belongs to
 * another allocator (a framework's caching allocator or a fixed budget) or a
 * latency-critical loop that cannot take cudaMalloc's implicit device-wide
 * synchronisation.  It computes what gks_create + gks_set_gas +
 * gks_set_scheme + gks_set_state + gks_step(dt) would, without a context.
 *   W_in, W_out: caller-owned device arrays, conserved variables [3][nx]
 *                float64 (rho, rho U, rho E); may not overlap.
 *   dx > 0, dt > 0 (no CFL choice here), bc[2] = x-low, x-high (gks_bc
 *   GKS_BC_PERIODIC .. GKS_BC_REFLECT; periodic on both ends or neither),
 *   gas as for gks_set_gas, precision as gks_grid_desc.
 *   scheme: checked as by gks_set_scheme except that cfl is not used; every
 *   reconstruction (gks_recon) and both merges (gks_merge) are taken;
 *   positivity_fallback must be 1 (the kernels always apply it), else
 *   GKS_EUNSUPPORTED.
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 *   It must not be a capturing stream (the call reads its error word back and
 *   synchronises): a stream under capture gives GKS_EINVAL.
 *   error_word (may be NULL): the step's error word (see gks_diag).
 * Working buffers live in one file-scope static device array sized for
 * GKS_NOALLOC_MAX_NX cells (about 1.6 MB on every GPU that loads the
 * library, kept until the process exits).  nx > GKS_NOALLOC_MAX_NX returns
 * GKS_EUNSUPPORTED; bad arguments GKS_EINVAL; a non-physical result
 * GKS_ENONPHYSICAL.  The first call in a device's context looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and
 * caches it with the context's id.  Every call reuses the same array and
 * resets what must start at zero, so calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller. */
gks_status gks_step1d_noalloc(const double *W_in, double *W_out, int nx, double dx, const int *bc,
                              const gks_gas *gas, const gks_scheme *scheme, int precision, double dt,
                              void *stream, unsigned int *error_word);

#ifdef __cplusplus
}
#endif
#endif /* GKS_H */
