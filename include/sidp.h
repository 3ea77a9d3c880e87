/*
 * libsidp -- sparse invariant-domain-preserving DG-SEM stage update with subcell
 * convex limiting on Cartesian and curved quadrilateral meshes (Pazner, arXiv 2004.08503),
 * for NVIDIA GB300 (sm_103a).  Plain C ABI: pointers and sizes only.
 *
 * Method (one forward-Euler stage, Sec. 4, Eq. subcell-fct / convex-fct):
 *   high-order DG-SEM residual r^H (strong form, Eq. dg-strong / ho-update, Lax-Friedrichs
 *   flux Eq. lax-friedrichs) -> sparsified low-order IDP residual r^L (Eq. dg-idp, graph
 *   viscosity Eq. dij) -> bar states (Eq. bar-states) and local bounds (Sec. 4.1.1, 4.3)
 *   -> subcell antidiffusive fluxes (Sec. 4.1.3) -> nodal limiting coefficients (Zalesak
 *   for the scalar or the density; Euler: specific-entropy minimum by a line search,
 *   Eq. convex-provisional) -> face coefficients and limited update.  Time stepping is
 *   SSP-RK3 with dt = CFL min_i m_i / (2 sum_{j != i} d-hat_ij) (Eq. cfl-low, Sec. 5).
 *
 * Conventions
 *   - Mesh: nx*ny square elements of side h on [x0,x1]x[y0,y1] (h = (x1-x0)/nx = (y1-y0)/ny).
 *     Element e = ey*nx + ex; node i = a*(p+1) + b inside it (a: y index, b: x index) at
 *     (x0 + (ex + xi_b) h, y0 + (ey + xi_a) h), xi the Gauss-Lobatto points on [0,1].
 *     Library node order: global node g = e*(p+1)^2 + i;  N = nx*ny*(p+1)^2.
 *   - Host state arrays are field-major float64 [nc][N] (nc = 1 scalar, 4 Euler with
 *     (rho, rho vx, rho vy, rho E)); they are owned by the caller and copied.
 *   - The library owns all device memory.  Device buffers are only lent out by
 *     sidp_device_state; the pointer stays valid until sidp_destroy.
 *   - Every entry point returns a status and never throws.  sidp_step / sidp_stage
 *     are asynchronous on the context's stream; sidp_get_* synchronise it.
 *   - One context is used by one host thread at a time.
 */
#ifndef SIDP_H
#define SIDP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SIDP_OK = 0,
  SIDP_ERR_ARG = 1,          /* invalid argument or configuration                      */
  SIDP_ERR_CUDA = 2,         /* a CUDA runtime call failed (see sidp_last_error)        */
  SIDP_ERR_NONFINITE = 3,    /* the state holds NaN/Inf                                 */
  SIDP_ERR_BOUNDS = 4,       /* inadmissible state (rho <= 0 or p <= 0 for Euler)       */
  SIDP_ERR_ROOTFIND_CAP = 5, /* the entropy line search hit its iteration cap           */
  SIDP_ERR_STATE = 6,        /* call out of order (e.g. stage 2 before stage 1)         */
  SIDP_ERR_OOM = 7           /* device allocation failed                                */
} sidp_status;

typedef enum {
  SIDP_LAW_BURGERS2D = 1,
  SIDP_LAW_EULER2D = 2,
  SIDP_LAW_ADVECTION2D = 3,
  SIDP_LAW_ADVECTION_VAR2D = 4
} sidp_law;
typedef enum { SIDP_FP64 = 0, SIDP_MIXED = 1 } sidp_precision;
typedef enum {
  SIDP_BC_PERIODIC = 0,
  SIDP_BC_OUTFLOW = 1,
  SIDP_BC_EXACT_STATE = 2,
  SIDP_BC_SLIP_WALL = 3, /* Euler only: ghost = mirror image of the trace (Sec. 5.7 slip wall) */
  SIDP_BC_SPLIT = 4      /* two ghost states split at a moving point: sidp_set_split_boundary */
} sidp_bc;
/* NONE: the high-order DG-SEM target (Eq. dg-strong); LOW_ORDER: the sparse IDP method
 * (Eq. dg-idp); SUBCELL: subcell flux correction with Zalesak (Sec. 4.1.3) and, for Euler, convex
 * entropy limiting (Sec. 4.3); ELEMENTWISE: one coefficient per element (Sec. 4.1.2, 4.2.1), the
 * comparison mode of Sec. 4.1.4.  The smoothness indicator applies to SUBCELL and ELEMENTWISE. */
typedef enum {
  SIDP_LIMITER_NONE = 0,
  SIDP_LIMITER_LOW_ORDER = 1,
  SIDP_LIMITER_SUBCELL = 2,
  SIDP_LIMITER_ELEMENTWISE = 3
} sidp_limiter;

typedef struct {
  int law;          /* sidp_law.  Burgers: f(u) = u^2/2 (1,1) (Sec. 5.5); Euler: Eq. euler-flux;
                       advection: f(u) = beta u with constant beta (Sec. 3.3); variable-velocity
                       advection: f(u) = beta(x) u with beta = (adv_beta[0] + adv_grad[0] y,
                       adv_beta[1] + adv_grad[1] x), divergence-free (Sec. 3.3; the solid body
                       rotation of Sec. 5.4 is adv_beta = (pi, -pi), adv_grad = (-2 pi, 2 pi))    */
  int p;            /* polynomial degree, 1..7                                                   */
  int nx, ny;       /* elements per direction, >= 1, nx * ny < 2^31                              */
  int precision;    /* SIDP_FP64: everything in float64.  SIDP_MIXED: float32 state and stage
                       arithmetic, float64 time step reduction                                   */
  double x0, x1, y0, y1;  /* domain; elements must be square                                     */
  int bc[4];        /* sidp_bc for the W, E, S, N sides.  Periodic must be paired (W with E,
                       S with N).  Outflow: ghost = interior trace.  Exact: ghost traces set by
                       sidp_set_ghost_state.  Slip wall: the trace with its normal momentum
                       negated (Euler).  Split: sidp_set_split_boundary                           */
  double cfl;       /* in (0, 1]; the paper uses 1/2 (Sec. 5)                                    */
  double gamma;     /* Euler ratio of specific heats, 1 < gamma <= 5/3 (wave-speed bound valid)  */
  double adv_beta[2]; /* advection velocity                                                      */
  int limiter;      /* sidp_limiter: HO target only, LO IDP only, subcell or elementwise limiting */
  int smoothness;   /* 1: the subcell-resolution smoothness indicator (Sec. 4.4) relaxes the bounds
                       of the limited field: eps_K u^min + (1 - eps_K) g^min, likewise the maximum   */
  double si_s0;     /* s0; 0 selects log10(p^-4) (Sec. 4.4)                                      */
  double si_kappa;  /* kappa; <= 0 selects 1                                                     */
  double si_gmin, si_gmax; /* global bounds g^min <= g^max of the limited field (scalar or rho)   */
  double adv_grad[2]; /* variable-velocity advection: d beta_x / dy and d beta_y / dx            */
  int unsparsified; /* 0: the sparse low-order operator of the paper (Eq. didp).  1: graph
                       viscosity on the dense DG-SEM operator, the comparison of Sec. 3.4 (every
                       pair of a line of an element coupled; bounds and time step follow).  Single
                       contexts only (a batch rejects it)                                         */
} sidp_config;

typedef struct {
  double t;                     /* simulated time advanced by sidp_step                       */
  long long steps;              /* SSP-RK3 steps taken by sidp_step                            */
  double last_dt;               /* dt of the last step (or of the last sidp_compute_dt)         */
  double mass[4];               /* sum_i m_i u_i per field (Sec. 2.4 conservation)              */
  double umin[4], umax[4];      /* nodal min / max per field                                   */
  double rho_min, p_min;        /* Euler: min density and pressure (0 for scalar laws)          */
  double max_bound_violation;   /* max over stages and nodes of the excess of the limited field
                                   (scalar or rho) over its local bounds, relative to
                                   max(|bound|, max |field| at the last host set_state)         */
  double max_entropy_violation; /* Euler: max over stages of max(0, 1 - sigma(u_i)/K_i)          */
  int rootfind_max_iters;       /* largest iteration count of the entropy line search           */
  long long rootfind_cap_hits;  /* line searches stopped by the iteration cap                   */
  long long nonfinite;          /* number of non-finite values in the current state              */
  long long bound_nudges;       /* SIDP_MIXED, statistics on: stage results of the limited field
                                   that float32 rounding left outside their local bounds (by at
                                   most 8 ulp of the update's operands) and that were set onto the
                                   bound before the store (the post-round acceptance); counted
                                   over stages and nodes since the last set_state              */
} sidp_diag;

typedef struct sidp_ctx sidp_ctx;
typedef struct sidp_batch sidp_batch;

/* Create a context on the current CUDA device.  `cuda_stream` is a cudaStream_t; with NULL the
 * library creates (and later destroys) its own non-blocking stream.  All work of the context is
 * ordered on that stream.  Validates cfg (Sec. 2 mesh
 * and law, Sec. 5 CFL) and allocates 3 state buffers plus small scratch.  On error *out = NULL. */
sidp_status sidp_create(sidp_ctx** out, const sidp_config* cfg, void* cuda_stream);
sidp_status sidp_destroy(sidp_ctx* ctx);

/* Number of nodes N and fields nc. */
sidp_status sidp_sizes(const sidp_ctx* ctx, long long* n_nodes, int* nc);

/* Physical coordinates of all nodes in library node order (caller-owned arrays of N doubles). */
sidp_status sidp_node_coords(const sidp_ctx* ctx, double* x, double* y);

/* Copy a host float64 [nc][N] state in (rounded to float32 in SIDP_MIXED).  Euler states with
 * rho <= 0 or p <= 0 anywhere return SIDP_ERR_BOUNDS (the invariant set of Sec. 4.3) and are
 * not copied; non-finite values return SIDP_ERR_NONFINITE.  Resets the stage sequence. */
sidp_status sidp_set_state(sidp_ctx* ctx, const double* u);

/* Copy a state out as float64 [nc][N].  which = 0: the current solution u^n; 1: the stage-1
 * result u^(1); 2: the stage-2 result u^(2) (SSP-RK3, Sec. 5).  Synchronises the stream. */
sidp_status sidp_get_state(sidp_ctx* ctx, int which, double* u);

/* Asynchronous state transfer in the library's storage type (float64 for SIDP_FP64, float32
 * for SIDP_MIXED), field-major [nc][N], ordered on the context's stream.  Use page-locked host
 * memory for full bandwidth.  No validation and no conversion: the caller owns the contents.
 * The host buffer must stay valid until sidp_synchronize (or any synchronising call). */
sidp_status sidp_upload_state(sidp_ctx* ctx, const void* host);
sidp_status sidp_download_state(sidp_ctx* ctx, int which, void* host);

/* Ghost trace for SIDP_BC_EXACT_STATE on `side` (0 W, 1 E, 2 S, 3 N): float64 [nc][n_side][p+1]
 * with n_side = ny for W/E and nx for S/N, ordered along the side. */
sidp_status sidp_set_ghost_state(sidp_ctx* ctx, int side, const double* u);

/* Parameters of a SIDP_BC_SPLIT side (0 W, 1 E, 2 S, 3 N), as in the double Mach reflection
 * (Sec. 5.7: a prescribed post-shock state that turns into a slip wall along the bottom, and a
 * top boundary state that switches at the exact position of the moving incident shock).  At a
 * face node whose coordinate along the side (y on W/E, x on S/N) is below s0 + speed * t, the
 * ghost state is state_a (float64 [nc], conserved variables), elsewhere state_b, or a slip wall
 * (the mirrored trace, Euler only) when state_b is NULL.  t is the stage time: t^n for the time
 * step and stage 1, t^n + dt for stage 2, t^n + dt/2 for stage 3 (SSP-RK3); sidp_step advances
 * t^n, explicit sidp_stage calls use the current simulated time as t^n.  Until set, a split side
 * behaves as outflow.  SIDP_ERR_STATE if the side is not a split side; the values are copied
 * (synchronous).  Not available in batches. */
sidp_status sidp_set_split_boundary(sidp_ctx* ctx, int side, double s0, double speed, const double* state_a,
                                    const double* state_b);

/* Set the simulated time (for example to resume from a saved state); ordered on the stream. */
sidp_status sidp_set_time(sidp_ctx* ctx, double t);

/* Curved (mapped) quadrilateral meshes: Sec. 2.3 (metric terms G = det J and the rows of
 * G J^-1 at the nodes, masses m_i = w_a w_b G_i, strong-form residual with contravariant fluxes)
 * and Sec. 3.1 (the conservative metric correction, the minimum-norm solution of
 * Eq. metric-perturbation, which makes the sparse low-order operator preserve constants).
 * The mesh keeps the nx x ny element topology and node order of the Cartesian mesh; each node
 * has its own coordinates.  Number of per-node arrays written by sidp_curved_metrics: */
#define SIDP_GEO_FIELDS 13

/* Metric arrays of the curved mesh whose nodes sit at (x[g], y[g]), float64 [N] each in library
 * node order (the two elements of a face give its nodes the same coordinates; across a periodic
 * side they differ by the period).  bc: the four side conditions, periodic, outflow or slip wall
 * (a wall face, like an outflow face, takes the element's own row as its normal).  Computed
 * on the host in float64; needs no GPU.  out: float64 [SIDP_GEO_FIELDS][N], caller-owned:
 *   0-1 row 1 of G J^-1 = (y_eta, -x_eta);  2-3 row 2 = (-y_xi, x_xi)
 *       (reference derivatives of the interpolated map, xi along b, eta along a);
 *   4-7 the corrected rows of Sec. 3.1 (row 1, row 2; x and y components);
 *   8   m_i = w_a w_b G_i;
 *   9-10 at nodes with b = 0 or p: the scaled normal of that element face pointing in +xi, the
 *       mean of the two adjacent elements' row 1 (a non-periodic boundary face: the element's
 *       own); 0 at other nodes;  11-12 the same with a = 0 or p, +eta and row 2.
 * SIDP_ERR_ARG for invalid sizes or sides, or a node with det J <= 0. */
sidp_status sidp_curved_metrics(int p, int nx, int ny, const int* bc, const double* x, const double* y,
                                double* out);

/* Move the context onto the curved mesh with node coordinates x, y (float64 [N] each, copied):
 * computes the metric arrays as sidp_curved_metrics does and keeps them on the device in the
 * stage precision; from then on the time step and the stages use the curved-mesh kernels and
 * sidp_node_coords returns these coordinates.  Supported: laws burgers, advection and euler;
 * limiters none, lo, subcell and elementwise, with or without the smoothness indicator (on the
 * reference element); periodic, outflow and (Euler) slip-wall sides, a wall ghost being the
 * trace with its momentum reflected about the face's unit normal, m - 2 (m . n) n (Sec. 5.7 on
 * mapped faces); not the unsparsified mode (SIDP_ERR_ARG).  The per-stage violation statistics
 * are collected as on Cartesian meshes, by a statistics variant of the curved stage kernel
 * launched while they are on; mass and extrema use m_i.  Synchronous. */
sidp_status sidp_set_geometry(sidp_ctx* ctx, const double* x, const double* y);

/* Lend the device buffer of u^n: *dptr = device pointer of [nc][N] values of type *dtype
 * (0 float64, 1 float32); *field_stride = N.  Valid until sidp_destroy. */
sidp_status sidp_device_state(sidp_ctx* ctx, void** dptr, int* dtype, long long* field_stride);

/* Eq. cfl-low: dt = cfl * min_i m_i / (2 sum_{j != i} d-hat_ij) on u^n; synchronises. */
sidp_status sidp_compute_dt(sidp_ctx* ctx, double* dt);

/* Measured fused multiply-add throughput of the current GPU in flop/s (one FMA = 2 flops):
 * precision SIDP_MIXED for float32, SIDP_FP64 for float64.  The paper has no counterpart: these
 * are the arithmetic ceilings the float32 and float64 stage kernels are placed against, beside
 * the HBM bandwidth.  Independent FMA chains in every thread of an occupancy-filling launch, timed
 * with CUDA events on cuda_stream; runs for a few tens of milliseconds and synchronises. */
sidp_status sidp_fma_peak(int precision, double* flop_per_s, void* cuda_stream);

/* The time step of sidp_compute_dt for a caller-owned device state, with no device allocation.
 * The paper has no counterpart: this serves callers that cannot allocate device memory where
 * they need a time step (an application whose pool allocator owns all device memory, a real-time
 * loop that cannot afford cudaMalloc's synchronisation, code holding only a raw device pointer).
 * d_state: device pointer to the [nc][N] state in the storage type of cfg->precision (float64 or
 * float32), library node order; d_dt: device pointer to one double that receives
 * cfl * min_i m_i / (2 sum_{j != i} d-hat_ij) (0 when no wave moves).  Asynchronous on
 * cuda_stream.  cfg passes the checks of sidp_create (else SIDP_ERR_ARG, before any device
 * access); in addition only periodic and outflow sides, only Burgers, Euler and constant-velocity
 * advection (the variable-velocity law is SIDP_ERR_ARG here) and only the sparsified operator
 * (cfg->unsparsified != 0 is SIDP_ERR_ARG: its smaller time step is not computed here).  Scratch
 * lives in a fixed 512 KiB device array shared by all calls: at most 65536 * 256 = 16,777,216
 * nodes (else SIDP_ERR_ARG), and calls that overlap on the GPU race.  The first call on a device
 * looks the array up (cudaGetSymbolAddress) and caches its address: make it before any stream
 * capture; a device reset (cudaDeviceReset) after it is not supported.  Errors set
 * sidp_last_error(NULL). */
sidp_status sidp_compute_dt_static(const sidp_config* cfg, const void* d_state, double* d_dt, void* cuda_stream);

/* One SSP-RK3 stage with a given dt (k = 1, 2, 3; Sec. 5):
 *   k=1: u^(1) = FE(u^n);  k=2: u^(2) = 3/4 u^n + 1/4 FE(u^(1));  k=3: u^n <- 1/3 u^n + 2/3 FE(u^(2)).
 * FE is the limited forward-Euler update of Eq. subcell-fct / convex-fct.  Asynchronous. */
sidp_status sidp_stage(sidp_ctx* ctx, int k, double dt);

/* nsteps SSP-RK3 steps, each with dt from Eq. cfl-low evaluated on u^n (computed on the
 * device; no host synchronisation).  Asynchronous.  The first call captures one step as a
 * CUDA graph (when use_graph is on) and later calls replay it. */
sidp_status sidp_step(sidp_ctx* ctx, int nsteps);

/* Element tile (elements per CTA along x and y) that the stage kernels use; chosen per
 * (law, p, precision, Cartesian or curved) by timing the candidates at the first sidp_step and once more when the
 * context has taken 10 steps (the first steps of a flow, such as a blast's initial transient,
 * can favour another tile than the rest of the run; that second pass synchronizes the stream
 * once, inside the sidp_step call that reaches step 10).  SIDP_TILE=<index> forces one,
 * SIDP_AUTOTUNE=0 keeps the default, SIDP_TUNE_FILE=<path> persists the settled choices.  The
 * candidates are indices 0..3, tiles of the node kernel (one thread per node), and, for the
 * Euler law, indices 4..5, tiles of the line kernel (one thread per element line).  Both compute
 * the same stage update (Sec. 4 with subcell limiting); they differ in the order of the rounding
 * of sums.  Modes other than subcell limiting without the smoothness indicator run the node
 * kernel with tile 0. */
sidp_status sidp_get_tile(const sidp_ctx* ctx, int* tx, int* ty);

/* The candidate index of the tile in use (see sidp_get_tile): 0..3 node kernel, 4..5 line
 * kernel.  SIDP_ERR_ARG for a null argument. */
sidp_status sidp_get_tile_index(const sidp_ctx* ctx, int* index);

/* Use tile candidate `index` (see sidp_get_tile) from now on, instead of the autotuner's choice.
 * Index 0 is valid in every mode; the others only for subcell limiting without the smoothness
 * indicator and the unsparsified mode: on a Cartesian mesh 1..3 (node kernel) and, for the Euler
 * law, 4..5 (line kernel); on a curved mesh (after sidp_set_geometry) 4, the curved line kernel,
 * for the Euler law.  Otherwise SIDP_ERR_ARG.  SIDP_ERR_STATE between stages 1 and 3 of an
 * explicit step.  sidp_set_geometry returns a context to tile 0 and to autotuning. */
sidp_status sidp_set_tile(sidp_ctx* ctx, int index);

/* Enable (1) or disable (0) CUDA-graph replay in sidp_step (default 1). */
sidp_status sidp_set_graph(sidp_ctx* ctx, int use_graph);

/* Enable (1) / disable (0) the per-stage statistics reported in sidp_diag, on by default: bound
 * and entropy violations and root-search counters.  With them on, a statistics variant of the stage kernel
 * runs (default tile shape); in the float32 form it evaluates the entropy bound accurately and
 * costs about 2.5x a plain stage.  Turn them off for timed runs. */
sidp_status sidp_set_stats(sidp_ctx* ctx, int on);

/* Debug capture: when on, every later stage writes its local bounds (lo, hi of the limited field;
 * K_i = min sigma for Euler) and nodal alpha-tilde to device buffers that sidp_get_bounds copies
 * out (caller-owned arrays of N doubles each; any pointer may be NULL). */
sidp_status sidp_set_debug(sidp_ctx* ctx, int on);
sidp_status sidp_get_bounds(sidp_ctx* ctx, double* lo, double* hi, double* K, double* alpha);

/* Diagnostics of the current state plus the statistics accumulated since the last set_state
 * (struct above).  Synchronises. */
sidp_status sidp_get_diag(sidp_ctx* ctx, sidp_diag* out);

/* Wait for all work queued on the context's stream. */
sidp_status sidp_synchronize(sidp_ctx* ctx);

const char* sidp_status_str(sidp_status s);
/* Message of the last error on this context (static storage when ctx is NULL). */
const char* sidp_last_error(const sidp_ctx* ctx);

/* ---------------------------------------------------------------- batches
 * Many independent problems (each its own mesh size, degree p, domain, periodic/outflow sides
 * and time step) advanced together.  Work is a task table of (instance, element tile) entries
 * grouped by p: each RK stage is one launch per degree group covering every tile of every
 * instance of that degree, and a whole step (per-instance dt included) is one CUDA graph.  All
 * configs of a batch share law, precision, limiter and law parameters.  Instance i's state is
 * exchanged as float64 [nc][N_i] like a single context's. */
sidp_status sidp_batch_create(sidp_batch** out, const sidp_config* cfgs, int count, void* cuda_stream);
sidp_status sidp_batch_destroy(sidp_batch* b);
sidp_status sidp_batch_sizes(const sidp_batch* b, int i, long long* n_nodes, int* nc);
sidp_status sidp_batch_total_nodes(const sidp_batch* b, long long* n_nodes);
/* Node coordinates of instance i (float64 [N_i] each, caller-owned): the Cartesian nodes, or the
 * coordinates given to sidp_batch_set_geometry. */
sidp_status sidp_batch_node_coords(const sidp_batch* b, int i, double* x, double* y);
/* Move instance i onto the curved mesh with node coordinates x, y (float64 [N_i] each, copied),
 * as sidp_set_geometry does for a context (Sec. 2.3 metric terms, Sec. 3.1 correction; the same
 * laws, limiters and sides; SIDP_ERR_ARG otherwise or for a mesh with det J <= 0).  The instance
 * joins the curved group of its degree: one launch per stage over tasks of (instance, block of
 * elements) with the curved-mesh kernels.  Mass and extrema in sidp_batch_get_diag use m_i.
 * Drops the captured step graph and turns the single-launch mode off.  Synchronous. */
sidp_status sidp_batch_set_geometry(sidp_batch* b, int i, const double* x, const double* y);
sidp_status sidp_batch_set_state(sidp_batch* b, int i, const double* u);
sidp_status sidp_batch_get_state(sidp_batch* b, int i, double* u);
/* Instance i's buffer `which` (0: u^n, 1: u^(1), 2: u^(2)) as float64 [nc][N_i] (caller-owned
 * host array); synchronises.  sidp_batch_get_state is which = 0. */
sidp_status sidp_batch_get_buffer(sidp_batch* b, int i, int which, double* u);
/* SSP-RK3 stage k (1, 2 or 3; Sec. 5) of every instance with the time steps dt[0..count-1]
 * (caller-owned host array, copied; finite and >= 0, else SIDP_ERR_ARG): stage 1 writes
 * u^(1) = FE(u^n), stage 2 u^(2) = 3/4 u^n + 1/4 FE(u^(1)), stage 3 u^(n+1) = 1/3 u^n +
 * 2/3 FE(u^(2)) over u^n.  Eager launches of the same kernels the step graph replays; the clocks
 * do not advance.  Synchronises.  For tests and for callers that drive the stages themselves. */
sidp_status sidp_batch_stage(sidp_batch* b, int k, const double* dt);
sidp_status sidp_batch_step(sidp_batch* b, int nsteps);
sidp_status sidp_batch_get_diag(sidp_batch* b, int i, sidp_diag* out);
sidp_status sidp_batch_set_stats(sidp_batch* b, int on);   /* statistics as sidp_set_stats (default on) */
sidp_status sidp_batch_synchronize(sidp_batch* b);
/* Debug capture for every instance, as sidp_set_debug (4 float64 per node of the batch on the
 * device); sidp_batch_get_bounds copies instance i's last-stage local bounds, K and alpha-tilde
 * into caller-owned arrays of N_i doubles (any may be NULL; SIDP_ERR_STATE before capture). */
sidp_status sidp_batch_set_debug(sidp_batch* b, int on);
sidp_status sidp_batch_get_bounds(sidp_batch* b, int i, double* lo, double* hi, double* K, double* alpha);
const char* sidp_batch_last_error(const sidp_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* SIDP_H */
