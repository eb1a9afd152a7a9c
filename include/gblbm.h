/*
 * gblbm.h -- C ABI of the gblbm library: a D2Q9 lattice Boltzmann solver with
 * halfway bounce-back on a voxelised rigid body, and the body force evaluated
 * every step by three schemes, after Kaushal, Succi & Ansumali, "Flow force
 * calculation in Lattice Boltzmann Method" (arXiv:2210.10377).
 *
 * Everything a call computes runs in the library's CUDA kernels (sm_103a).
 * There is no CPU fallback: without a usable GPU every compute call returns
 * LBM_ECUDA.
 *
 * Notation used below (Section II of the paper):
 *   nodes (x, y), 0 <= x < nx, 0 <= y < ny, node index n = y*nx + x;
 *   D2Q9 directions 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
 *                   5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1);
 *   weights 4/9, 1/9 (1..4), 1/36 (5..8); theta0 = 1/3;
 *   f(x, t) pre-collision populations, ft(x, t) post-collision (Eq. CollideAdv);
 *   ft = f + (feq - f)/tau, i.e. the paper's 2*beta equals 1/tau and the
 *   kinematic viscosity is (tau - 1/2)/3 in lattice units.
 *   Population arrays crossing this ABI are double [9][ny][nx], row-major.
 *
 * Ownership: every pointer argument is caller-owned host memory, read or
 * written only during the call.  Device memory is owned by the handle and
 * comes from the allocator in lbm_bc (cudaMalloc when none is given).
 * A handle is not thread-safe; distinct handles are independent.
 * Errors: every call returns an lbm_status; lbm_last_error(h) gives a message
 * (lbm_last_error(NULL) for calls that have no handle).  No C++ exception and
 * no process exit crosses this ABI.
 */
#ifndef GBLBM_H
#define GBLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* an argument is out of range (message says which) */
    LBM_ENOMEM = 2,    /* the allocator returned NULL */
    LBM_ECUDA = 3,     /* a CUDA call failed (no device, launch error, ...) */
    LBM_EUNSTABLE = 4, /* a step produced rho <= 0 or NaN (first step index in the message) */
    LBM_ETIMEOUT = 5,  /* a bounded device wait expired (the step's results are invalid) */
    LBM_ESTATE = 6     /* the request needs a state that does not exist yet */
} lbm_status;

typedef enum {
    /* equilibrium inlet at x = 0 (ft = feq(rho0, (u_in(y), 0))), zero-gradient
     * outlet at x = nx-1 (f(nx-1, y) = f(nx-2, y) after streaming), periodic y */
    LBM_BC_CHANNEL = 0,
    /* periodic in x and y */
    LBM_BC_PERIODIC = 1
} lbm_bc_kind;

typedef enum {
    LBM_F64 = 0,     /* populations stored and collided in FP64 */
    LBM_F32 = 1,     /* stored and collided in FP32 */
    LBM_F32_DEV = 2, /* FP32 storage of g_i = f_i - w_i rho0, FP32 collision */
    LBM_F16_DEV = 3  /* FP16 storage of g_i = f_i - w_i rho0, FP32 collision */
} lbm_storage;

typedef enum {
    /* Momentum exchange, Eq. (MEA): F = sum over fluid-solid links (x_f, i) of
     * c_i [f_i(x_f) + f_opp(i)(x_f)], both on the pre-collision state f(x_f, t)
     * (algorithm A of Fig. basicLadd). */
    LBM_FORCE_MEA_A = 0,
    /* Algorithm B, Eq. (rtt5) with bounce-back: F = 2 sum c_i ft_i(x_f, t). */
    LBM_FORCE_MEA_B = 1,
    /* Discrete Reynolds transport theorem, Eq. (rtt7) (second form) and the
     * Appendix: F(t) = J(t) - J(t+1) + gained(t) - lost(t) over the control
     * volume box, gained/lost = post-collision populations streaming into /
     * out of the box between fluid nodes.  J(t) is summed on the stored
     * post-collision state less the body-force momentum (equal to the
     * pre-collision J(t) in exact arithmetic), J(t+1) on the pre-collision
     * state.  Needs J(t+1), i.e. one step beyond t. */
    LBM_FORCE_DRTT = 2,
    /* Eq. (rtt4) read literally for algorithm A: lost momentum with f_i(x_f, t),
     * gained momentum with the bounced ft_i(x_f, t). Diagnostic. */
    LBM_FORCE_MEA_A_RTT = 3,
    /* Diagnostic, not a force: momentum the collision fails to conserve inside
     * the control volume in the storage arithmetic, sum over its fluid nodes of
     * c.(f - ft) + g; zero in exact arithmetic (BGK conserves momentum). */
    LBM_DIAG_MOMENTUM_DEFECT = 4,
    /* Stress integration, Eq. (stress_int), on the voxelised surface: every
     * axis link (x_f, i), i = 1..4, is a unit face with normal -c_i out of the
     * solid, and adds -c_i . T(x_f, t) with T = -p I + sigma from the
     * pre-collision populations of the fluid node: p = rho theta0 (theta0 = 1/3)
     * and sigma = -(1 - omega/2) sum_k (f_k - feq_k) c_k c_k, the viscous stress
     * rho nu (grad u + grad u^T) (Section IV; the paper writes the factor as
     * 1 - beta, 2 beta = omega). */
    LBM_FORCE_SI = 5
} lbm_scheme;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer (16-byte aligned at least: the kernels'
 * bulk copies and L2 prefetches start on 16-byte boundaries, and creation
 * fails with EINVAL on a pointer that is not) or NULL; stream is the handle's
 * stream.  free releases a pointer from alloc. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lbm_free_fn)(void *ptr, void *user);

typedef struct {
    int kind;             /* lbm_bc_kind */
    int storage;          /* lbm_storage */
    double rho0;          /* reference density: inlet density, deviation base (1.0) */
    double body_force[2]; /* uniform body force g: ft_i += 3 w_i c_i.g (test set-ups) */
    int cv[4];            /* DRTT control volume, inclusive {x0, x1, y0, y1};
                             cv[0] < 0 selects the default box (see lbm_create) */
    int record_series;    /* 1: keep forces of every step; 0: only the last two */
    void *cuda_stream;    /* cudaStream_t for all work of the handle; NULL: the handle
                             creates its own non-blocking stream */
    lbm_alloc_fn alloc;   /* NULL: cudaMalloc / cudaFree */
    lbm_free_fn free;
    void *alloc_user;
    int kernel;           /* collide-stream kernel: 0 direct loads (default);
                             1 staged bulk copies wherever it applies (channel
                             set-up, pulled state).  Both give identical results. */
} lbm_bc;

/* Fill *bc with defaults: channel, FP32, rho0 = 1, no body force, default
 * control volume, record_series = 1, own stream, cudaMalloc, direct kernel. */
void lbm_bc_default(lbm_bc *bc);

/* Create a solver on an nx x ny grid.
 *   mask     uint8 [ny][nx], nonzero = solid node (x_s), zero = fluid (x_f);
 *            the halfway bounce-back wall sits half-way along every
 *            fluid-solid link (Section II, Fig. basicLadd).
 *   tau      lattice relaxation time, > 0.5.
 *   u_in     inlet velocity, n_u_in values: 1 (uniform) or ny (per row y).
 *   bc       boundary set-up, storage, control volume, stream, allocator.
 * Initial state (t = 0): f = feq(rho0, (u_in(y), 0)) on every fluid node.
 * Default control volume: the solid nodes' bounding box widened by
 * max(4, ceil(w/4)) nodes per side (w = box width in x), clipped in x to
 * [1, nx-2] in a channel; a range that would touch a periodic edge becomes the
 * whole period.
 * EINVAL: nx < 4, ny < 3, 8*nx*ny >= 2^31, tau <= 0.5, non-finite input, bad
 * kind/storage/n_u_in, rho0 <= 0, a solid node in columns 0, 1, nx-2, nx-1 of a
 * channel, or a control volume that touches the inlet/outlet column or
 * straddles a periodic edge (it must lie within [1, n-2] or span [0, n-1]),
 * or a population buffer from bc->alloc that is not 16-byte aligned.
 * ENOMEM / ECUDA as named.  On success *out receives the handle. */
lbm_status lbm_create(const uint8_t *mask, int nx, int ny, double tau, const double *u_in,
                      int n_u_in, const lbm_bc *bc, lbm_ctx **out);

/* Advance n >= 0 steps.  Each step t -> t+1 runs, in this order, the fused
 * pull-stream + bounce-back + inlet/outlet + BGK collision kernel (which also
 * accumulates J(t) and the control-volume fluxes), then the link kernel (MEA
 * A, A', B of step t and DRTT of step t-1).  Blocks until the work is done.
 * The call may be split into any sequence of calls with the same total: the
 * state and the force series do not depend on the split.
 * EUNSTABLE if any step produced rho <= 0 or NaN (the state then holds the
 * result after all n steps); ETIMEOUT if a bounded wait of the staged kernel
 * expired; ESTATE if a series row would have fallen outside the series buffer
 * (an internal invariant; the row is dropped rather than written). */
lbm_status lbm_step(lbm_ctx *h, int n);

/* lbm_step without the wait: queues n >= 0 steps on the handle's stream and
 * returns.  The steps' status (EUNSTABLE, ETIMEOUT, ESTATE as for lbm_step,
 * collected over every step queued since the last wait) is returned by the
 * next lbm_sync, lbm_step or any call that reads results, each of which first
 * waits for the queued steps.  The state and the series are those lbm_step
 * gives.  EINVAL for n < 0; ENOMEM/ECUDA when the work cannot be queued. */
lbm_status lbm_step_async(lbm_ctx *h, int n);

/* Wait for the steps queued by lbm_step_async and return their status. */
lbm_status lbm_sync(lbm_ctx *h);

/* Optional: make the next n steps launch-only.  Grows the force series to
 * hold n more steps and builds the captured step graphs for every starting
 * buffer, so that a following lbm_step(m <= n) does no allocation, stream
 * capture or graph instantiation, only launches.  (lbm_step does the same work
 * lazily when it is not called.)  Blocks.  EINVAL for n < 0; ENOMEM, ECUDA. */
lbm_status lbm_prepare(lbm_ctx *h, long n);

/* Force on the body (+x downstream) of the last completed step t = T-1
 * (the transition T-1 -> T) for one lbm_scheme.  ESTATE before the first step. */
lbm_status lbm_force(lbm_ctx *h, int scheme, double *fx, double *fy);

/* Forces of steps [first, first+count) for one lbm_scheme into fx[count], fy[count].
 * EINVAL if the range is not kept (record_series = 0 keeps the last two). */
lbm_status lbm_force_series(lbm_ctx *h, int scheme, long first, long count, double *fx,
                            double *fy);

/* Drag and lift coefficients of one lbm_scheme over steps [first, first+count)
 * (Section V: C_d = 2 F_x / (rho0 U^2 L), C_l = 2 F_y / (rho0 U^2 L), signed,
 * F the force on the body of that step, rho0 the handle's, L = length the
 * reference length (the chord; the diameter for a cylinder, Section VI), U =
 * u_ref the reference speed (u_in)).  Computed on the device from the stored
 * series.  cd[count], cl[count]: per-step values (either may be NULL);
 * stats[4] (may be NULL): the window's mean C_d, mean C_l, and the standard
 * deviations of C_d and C_l (population form, mean removed first), summed in
 * a fixed order.  EINVAL for an empty or unkept range, length <= 0 or
 * u_ref = 0. */
lbm_status lbm_coefficients(lbm_ctx *h, int scheme, long first, long count, double length, double u_ref,
                            double *cd, double *cl, double *stats);

/* Pre-collision populations f(x, T) as double [9][ny][nx]; solid nodes read 0.
 * For deviation storage the base w_i rho0 is added back in FP64. */
lbm_status lbm_populations(lbm_ctx *h, double *out);

/* Replace f(x, T) by in[9][ny][nx] (fluid nodes; solid entries are ignored),
 * rounded to the storage precision.  The step count is kept. */
lbm_status lbm_set_populations(lbm_ctx *h, const double *in);

/* The fluid-solid link list, built on the device: entries n*8 + (i-1) for every
 * fluid node n and direction i = 1..8 whose neighbour n + c_i (y periodic, x
 * periodic only for LBM_BC_PERIODIC) is solid, in ascending order.  Writes at
 * most cap entries to out and the total count to *count. */
lbm_status lbm_links(lbm_ctx *h, int32_t *out, long cap, long *count);

/* The control volume in use, inclusive {x0, x1, y0, y1}. */
lbm_status lbm_control_volume(lbm_ctx *h, int *cv);

/* Voxelise a NACA 4-digit symmetric section on the device.  Half-thickness
 *   y_t(s) = 5 t C [0.2969 sqrt(s) - 0.1260 s - 0.3516 s^2 + 0.2843 s^3 - a4 s^4],
 * s = xi/C, a4 = 0.1015 (closed_te = 0) or 0.1036 (closed_te = 1); mid-chord at
 * (xc, yc); alpha > 0 nose-up:
 *   xi = (x - xc) cos(alpha) - (y - yc) sin(alpha) + C/2,
 *   eta = (x - xc) sin(alpha) + (y - yc) cos(alpha);
 * node solid iff 0 <= xi <= C and |eta| <= y_t(xi/C).  cos and sin are taken on
 * the host of alpha = alpha_deg * pi / 180; the predicate is evaluated on the
 * device in FP64 with round-to-nearest operations in the order written above.
 * (The paper names the NACA0012 section, Section V, but not its formula.)
 * out: uint8 [ny][nx].  EINVAL for non-positive sizes, chord or thickness. */
lbm_status lbm_naca_mask(int nx, int ny, double chord, double thickness, double alpha_deg,
                         double xc, double yc, int closed_te, uint8_t *out);

/* Voxelised circular cylinder of diameter D centred at (xc, yc) (Section VI,
 * flow past a 2-D circular cylinder): out[y][x] = 1 iff
 * (x - xc)^2 + (y - yc)^2 <= (D/2)^2, evaluated as written with separately
 * rounded FP64 operations (bit-for-bit reproducible).  Runs on the device.
 * EINVAL: nx, ny <= 0, D <= 0, non-finite arguments, out NULL. */
lbm_status lbm_cylinder_mask(int nx, int ny, double xc, double yc, double diameter, uint8_t *out);

/* Discrete adjoint (channel set-up, no body force, record_series = 1).
 * From the current state (step T0) run `steps` steps as lbm_step would (the
 * handle ends at T0 + steps with its force series), and return the objective
 *   J = (1/window) sum_{t = T0+steps-window}^{T0+steps-1} (wx Fx(t) + wy Fy(t)),
 * F the algorithm-B force (Eq. rtt5 with bounce-back), with its gradients:
 *   dJ_dtau     dJ/dtau;
 *   dJ_du[ny]   dJ/du_in(y) through the equilibrium inlet of every row;
 *   dJ_df0      [9][ny][nx] dJ/df(x, T0), pre-collision state at T0 (0 on solid
 *               nodes and in the inlet column, which do not enter J); host
 *               memory, or device memory of the handle's device (unified
 *               addressing tells them apart), where it is written in place
 *               without a copy to the host.
 * Every step of the forward map (BGK collision, pull streaming with halfway
 * bounce-back, inlet, outlet) is differentiated exactly and transposed, in the
 * storage's compute precision.  checkpoint_every > 0: states are recomputed
 * from checkpoints taken every checkpoint_every steps.  checkpoint_every <= 0:
 * the forward pass keeps the states of the last L steps in device memory
 * (no recompute for them), L as large as 60 % of the free device memory
 * (or lbm_set_adjoint_budget) allows, and the first steps - L are checkpointed every
 * ceil(sqrt(steps - L)) steps; the results are the same bits either way.
 * Any output may be NULL.
 * Synchronous: every output is complete when the call returns.
 * EINVAL for a periodic domain, a body force, record_series = 0, or
 * window outside [1, steps]. */
lbm_status lbm_adjoint(lbm_ctx *h, int steps, int window, double wx, double wy, int checkpoint_every,
                       double *J, double *dJ_dtau, double *dJ_du, double *dJ_df0);

/* Device memory, in bytes, that lbm_adjoint with checkpoint_every <= 0 may
 * fill with kept states and checkpoints (0, the default: 60 % of the free
 * device memory at the call).  A caller whose allocator holds cached memory
 * that cudaMemGetInfo does not count as free states what it can provide.
 * Host-side only; EINVAL for a negative or non-finite value. */
lbm_status lbm_set_adjoint_budget(lbm_ctx *h, double bytes);

/* Number of completed steps T. */
long lbm_steps_done(const lbm_ctx *h);

/* Number of fluid-solid links. */
long lbm_num_links(const lbm_ctx *h);

/* Choose the collide-stream kernel of later steps: 0 = direct loads, 1 = the
 * staged kernel (bulk tensor copies through an mbarrier pipeline), which needs
 * a handle created with lbm_bc.kernel = 1 (EINVAL otherwise).  Both do the
 * same arithmetic per node.  Waits for the handle's stream. */
lbm_status lbm_set_kernel(lbm_ctx *h, int kernel);

/* Bound, in polls, on each pipeline wait of the staged kernel (default
 * 2^22; polls < 0 restores it).  For testing the timeout path: with 0, every
 * CTA's first wait gives up at once, the CTA waits (with a bound of its own)
 * for the copies it has issued, and lbm_step returns ETIMEOUT; the step's
 * output is then incomplete, and the caller restores a state
 * (lbm_set_populations) before stepping on.  Waits for the handle's stream. */
lbm_status lbm_set_wait_limit(lbm_ctx *h, long polls);

/* Kernel timing for measurements: while on, lbm_step launches each kernel
 * separately (no CUDA graph) between CUDA events on the handle's stream and
 * accumulates device time per kernel.  lbm_kernel_times writes, for
 * k = 0 (collide-stream) and k = 1 (link force), total milliseconds ms[k] and
 * launch counts launches[k] since the last reset; reset = 1 clears them. */
lbm_status lbm_set_kernel_timing(lbm_ctx *h, int on);
lbm_status lbm_kernel_times(lbm_ctx *h, double *ms, long *launches, int reset);

/* Kernel launches made by the handle since creation (all kernels). */
long lbm_launch_count(const lbm_ctx *h);

/* The fluid-solid link list of a mask that already lives in device memory,
 * built without allocating any memory.  The paper has no counterpart: this is
 * a service entry point of this library.  It serves callers that must not
 * allocate device memory themselves or through this library: code that runs
 * inside a host application owning a fixed device-memory budget or its own
 * memory pool, plug-ins whose host forbids cudaMalloc, and latency-sensitive
 * callers that cannot accept the device-wide synchronisation cudaMalloc and
 * cudaFree may cause.  The result equals lbm_links() on a handle created from
 * the same mask and boundary kind (same list, same order).
 *   d_mask      device pointer, uint8 [ny][nx], nonzero = solid; caller-owned.
 *   periodic_x  1: x wraps (LBM_BC_PERIODIC), 0: it does not (LBM_BC_CHANNEL);
 *               y always wraps.
 *   d_links     device pointer to cap int32 entries, caller-owned; receives
 *               n*8 + (i-1) in ascending order (at most cap entries).
 *   count       host pointer; receives the total number of links.
 *   cuda_stream cudaStream_t the work is queued on (NULL: legacy default).
 * The call is synchronous: it reads the total back into host memory and
 * returns after that stream has finished the work.  It therefore cannot be
 * recorded into a CUDA graph, and a stream that is being captured is refused
 * with EINVAL.  If cap < *count, only the first cap links are written and
 * *count still receives the full total.
 * Limit: nx*ny <= 2^26 nodes; larger grids return EINVAL.  Working memory is
 * one fixed static device array of 256 KB, present on every device that loads
 * the library until the process exits.  Every call looks up that array's
 * device address (cudaGetSymbolAddress, with the caller's device current), so
 * a cudaDeviceReset between calls leaves no stale address.  All calls on a
 * device share the array and every call rewrites what it reads, so calls whose
 * GPU work overlaps (other host threads, other streams) race and must be
 * serialised by the caller.  Calls no cudaMalloc, cudaFree or other allocating
 * routine. */
lbm_status lbm_links_noalloc(const uint8_t *d_mask, int nx, int ny, int periodic_x,
                             int32_t *d_links, long cap, long *count, void *cuda_stream);

/* Pressure coefficient at the boundary fluid nodes at the current step
 * (Section VI): cp = (p - p_inf) / q with p = rho theta0 = rho/3 from the
 * pre-collision populations of the node.  The boundary fluid nodes are the
 * distinct fluid nodes of the link list (a fluid node with a solid neighbour
 * in any of the 8 directions), in ascending node index n = y*nx + x.
 *   p_inf   reference pressure (e.g. rho0/3 of the inlet); finite.
 *   q       dynamic pressure (e.g. rho0 u_in^2 / 2); finite, nonzero.
 *   nodes   receives up to cap node indices (NULL: not wanted).
 *   cp      receives up to cap coefficients, same order (NULL: not wanted).
 *   count   receives the number of boundary fluid nodes.
 * EINVAL for p_inf or q out of range. */
lbm_status lbm_pressure_coefficient(lbm_ctx *h, double p_inf, double q, int32_t *nodes, double *cp, long cap,
                                    long *count);

/* Message of the last failed call on h (or of the calling thread when h is NULL). */
const char *lbm_last_error(const lbm_ctx *h);

/* Release the handle and its device memory.  NULL is ignored. */
void lbm_destroy(lbm_ctx *h);

/* ------------------------------------------------------------------------
 * Batches: many independent domains advanced together.
 *
 * A batch holds n domains.  Each is a full problem of its own, as lbm_create
 * defines one: its own grid, body mask, relaxation time, inlet profile and
 * control volume.  They share one boundary kind, storage type and rho0.  One
 * batch step advances every domain by one time step.  It does that in one
 * collide-stream launch over a table of the tiles of all domains, followed
 * by one link launch (one CTA per domain).  Steps are replayed from captured
 * CUDA graphs.  Per domain, the arithmetic and the force rows equal those of
 * a single-domain handle; only the summation order of the DRTT box sums
 * depends on the tile shape.
 * The paper treats one body at a time; the batch serves sweeps of its
 * Section V airfoil study (angle of attack, thickness, Reynolds number) in
 * one launch.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

/* One domain: the arguments of lbm_create for it (all host memory, read
 * during lbm_batch_create only). */
typedef struct {
    const uint8_t *mask;  /* uint8 [ny][nx], nonzero = solid */
    int nx, ny;
    double tau;           /* > 0.5 */
    const double *u_in;   /* n_u_in values: 1 (uniform) or ny (per row) */
    int n_u_in;
    int cv[4];            /* control volume x0, x1, y0, y1 inclusive; cv[0] < 0: default */
} lbm_domain;

/* Create a batch of n >= 1 domains.  bc gives the boundary kind, storage,
 * rho0, stream and allocator of all domains (bc->cv is ignored: each domain
 * has its own).  The body force must be zero and bc->kernel 0.  The force
 * series is always kept in full when bc->record_series is 1; otherwise only
 * the last two steps are kept.  Initial state as lbm_create.  The launch
 * configuration starts at tile shape 0 with one CTA per tile;
 * lbm_batch_autotune picks a faster one.
 * EINVAL: n < 1, any domain failing lbm_create's checks (the message names
 * the domain), a nonzero body force, bc->kernel != 0, a population arena from
 * bc->alloc that is not 16-byte aligned.  ENOMEM / ECUDA as named. */
lbm_status lbm_batch_create(const lbm_domain *domains, int n, const lbm_bc *bc, lbm_batch **out);

/* Advance every domain n >= 0 steps (as lbm_step, for each domain).
 * Blocks until the work is done.  EUNSTABLE when any domain's instability
 * flag is set (the flags are sticky; lbm_batch_status names the domains);
 * every domain has still taken all n steps.  ESTATE if a series row would
 * have fallen outside the series buffer (an internal invariant). */
lbm_status lbm_batch_step(lbm_batch *b, int n);

/* Forces of every domain at one step (0 <= step < steps done), for a scheme
 * of lbm_scheme: fx[n], fy[n].  As lbm_force_series for each domain. */
lbm_status lbm_batch_forces(lbm_batch *b, int scheme, long step, double *fx, double *fy);

/* Force series of one domain, steps [first, first+count): as lbm_force_series. */
lbm_status lbm_batch_force_series(lbm_batch *b, int domain, int scheme, long first, long count,
                                  double *fx, double *fy);

/* Drag and lift coefficients of one domain over steps [first, first+count): as
 * lbm_coefficients, with that domain's force series. */
lbm_status lbm_batch_coefficients(lbm_batch *b, int domain, int scheme, long first, long count, double length,
                                  double u_ref, double *cd, double *cl, double *stats);

/* Optional: make the next n batch steps launch-only (as lbm_prepare): grows
 * the series and builds the captured step graphs of both starting buffers for
 * the current launch configuration (a later lbm_batch_set_launch or
 * lbm_batch_autotune that changes it drops them again). */
lbm_status lbm_batch_prepare(lbm_batch *b, long n);

/* Pre-collision populations of one domain at the current step: out is double
 * [9][ny][nx] of that domain (0 at solid nodes), as lbm_populations. */
lbm_status lbm_batch_populations(lbm_batch *b, int domain, double *out);

/* Set the pre-collision populations of one domain, before the first step
 * only (ESTATE afterwards): in is double [9][ny][nx], finite. */
lbm_status lbm_batch_set_populations(lbm_batch *b, int domain, const double *in);

/* Pressure coefficient at the boundary fluid nodes of one domain: as
 * lbm_pressure_coefficient, node indices n = y*nx + x of that domain. */
lbm_status lbm_batch_pressure_coefficient(lbm_batch *b, int domain, double p_inf, double q, int32_t *nodes,
                                          double *cp, long cap, long *count);

/* Per-domain instability flags: unstable[d] = 1 when domain d produced
 * rho <= 0 or NaN in some step, and first_bad_step[d] = that step (-1 when
 * the flag is clear).  Either pointer may be NULL. */
lbm_status lbm_batch_status(lbm_batch *b, int *unstable, long *first_bad_step);

/* Launch configuration of the batched collide-stream kernel.
 * shape: a tile shape index (0 .. lbm_batch_num_shapes()-1).
 * ctas_per_sm: 0 for one CTA per tile, k > 0 for a persistent grid of
 * k * (SM count) CTAs walking the tile table.  Shapes and grids differ only
 * in speed and in the summation order of the DRTT box sums.
 * EINVAL: an unknown shape, or k above what the SM can hold of that kernel. */
lbm_status lbm_batch_set_launch(lbm_batch *b, int shape, int ctas_per_sm);
lbm_status lbm_batch_get_launch(const lbm_batch *b, int *shape, int *ctas_per_sm);

/* Tile shape k: width tile_w nodes along x by tile_h rows, for the batch's
 * storage type (EINVAL for an unknown k). */
int lbm_batch_num_shapes(void);
lbm_status lbm_batch_shape(const lbm_batch *b, int k, int *tile_w, int *tile_h);

/* Time every tile shape with every grid the SM can hold (one CTA per tile,
 * or 1, 2, 3, 4, 6, 8 CTAs per SM), trials launches each after one warm-up,
 * and keep the fastest.  The trials run the collide-stream kernel alone,
 * from the current state into the spare buffer.  Their partial sums and
 * flags go to scratch memory, so the simulation state and its results do
 * not change.  On return *shape and *ctas_per_sm (either may be NULL) hold
 * the choice, and *best_ms its time per launch. */
lbm_status lbm_batch_autotune(lbm_batch *b, int trials, int *shape, int *ctas_per_sm,
                              double *best_ms);

long lbm_batch_steps_done(const lbm_batch *b);
int lbm_batch_num_domains(const lbm_batch *b);
/* Total nodes of all domains (the unit of the batch's MLUPS). */
long long lbm_batch_nodes(const lbm_batch *b);
/* Kernel launches issued by the batch so far (set-up included). */
long long lbm_batch_launch_count(const lbm_batch *b);
/* Message of the last failed call on b (or of the calling thread when b is NULL). */
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* GBLBM_H */
