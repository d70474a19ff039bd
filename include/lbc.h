/*
 * lbc.h -- C ABI of the GB300 half-range lattice Boltzmann Couette solver.
 *
 * The solver integrates the reduced Shakhov-model Boltzmann equation for planar
 * Couette flow (Ambrus, Sharipov & Sofonea, arXiv:1810.07803, Sec. II,
 * Eq. boltz_red) with the mixed-quadrature lattice Boltzmann model
 * HHLB(Nx;Qx) x HLB(Ny;Qy) of Sec. III: half-range Gauss-Hermite abscissas on
 * p_x (each half-space separately), full-range Gauss-Hermite on p_y, the
 * equilibrium replaced by its Hermite truncations (Eqs. gx, gy), diffuse walls
 * with the zero-mass-flux density (Eqs. diffuse, diffuse_nw), relaxation time
 * from the viscosity law (Eqs. mu, tau), WENO-5 advection on the
 * tanh-stretched grid (Eq. stretch) and TVD RK-3 in time.
 *
 * Units: m = k_B = 1; lengths in L (walls at x = -1/2, +1/2); temperatures in
 * T_ref; velocities and momenta in v_ref = sqrt(k_B T_ref / m); times in
 * L / v_ref; densities in n_ref (the initial, and mean, density).
 *
 * Velocity set: index v = a * Qy + j with a in [0, 2Qx), j in [0, Qy).
 * a < Qx: p_x = +p0 z_a; a >= Qx: p_x = -p0 z_{a-Qx} (the paper's
 * p_{x,i+Qx} = -p_{x,i}); p_y = p0 y_j; quadrature weight w_a w_j, where z, w
 * is the half-range rule of order Qx and y, w the full-range rule of order Qy.
 *
 * State: the reduced distributions phi and chi (Sec. II) divided by the
 * quadrature weights, ft = phi_v / (w_a w_j), so that an equilibrium is O(1)
 * at every velocity. Host-side state arrays are float64, row-major
 * [2][V][Nx] (field 0 = phi, field 1 = chi; V = 2 Qx Qy).
 *
 * Errors: every call returns an lbc_status; nothing throws across the ABI.
 * lbc_last_error() gives a thread-local message for the last failure. A failed
 * call leaves the solver unchanged, except LBC_ENONFINITE (the state held a
 * NaN or Inf), LBC_ETIMEOUT and LBC_EBOUNDS, after which the solver refuses
 * further steps until a state is installed.
 *
 * Threads and streams: a solver may be used from one host thread at a time.
 * All device work is enqueued on the CUDA stream given at creation; calls
 * that return host data synchronise that stream.
 *
 * Ownership: the solver owns all of its device memory (allocated with
 * cudaMallocAsync on its stream at lbc_create, freed by lbc_destroy). The
 * caller owns every host array passed in; lbc_params is copied at creation.
 */
#ifndef LBC_H
#define LBC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbc_solver lbc_solver;

typedef enum {
    LBC_OK = 0,
    LBC_EINVAL = 1,      /* invalid argument (message says which) */
    LBC_ENOMEM = 2,      /* device allocation failed */
    LBC_ECUDA = 3,       /* a CUDA runtime call failed */
    LBC_ENOTCONV = 4,    /* lbc_run_to_steady hit max_steps */
    LBC_ENONFINITE = 5,  /* NaN/Inf in the state; the solver is poisoned */
    LBC_ETIMEOUT = 6,    /* a bounded device wait gave up */
    LBC_EBOUNDS = 7,     /* range-checked build only: a device index check failed (message names it) */
    LBC_ESTALLED = 8     /* run to steady: a residual stopped falling above the threshold (stall window) */
} lbc_status;

typedef enum { LBC_MU_POWER = 0, LBC_MU_TABLE = 1 } lbc_mu_law;
typedef enum { LBC_FP64 = 0, LBC_FP32_STATE = 1 } lbc_precision;

#define LBC_NMOM 10
/* Rows of lbc_moments' output: */
enum { LBC_M_N = 0, LBC_M_UX, LBC_M_UY, LBC_M_T, LBC_M_PXX, LBC_M_PYY, LBC_M_PZZ,
       LBC_M_PXY, LBC_M_QX, LBC_M_QY };

typedef struct {
    double delta;            /* rarefaction parameter (Eq. delta); 0 = collisionless */
    double u_left, u_right;  /* wall velocities along y (v_ref units) */
    double T_left, T_right;  /* wall temperatures (T_ref units), > 0 */
    double Pr;               /* Prandtl number of the Shakhov model (Sec. II) */
    lbc_mu_law mu_law;       /* LBC_MU_POWER: mu = T^omega (Eq. mu), Pr constant;
                                LBC_MU_TABLE: Eqs. mun, interp (below) */
    double omega;            /* viscosity index of the power law */
    /* LBC_MU_TABLE: tab_n in [2, 256] entries (copied at creation) of temperatures
     * tab_T (T_ref units, > 0, strictly increasing), viscosities tab_mu (> 0, any
     * unit) and Prandtl numbers tab_Pr (> 0). On [T_n, T_{n+1}) mu is the power
     * law through both points, the first and last intervals extend below T_2 and
     * above T_{N-1}; Pr = Pr_1 below T_2, Pr_n on [T_n, T_{n+1}), Pr_N from T_N on.
     * delta refers to mu(T_ref = 1) of this law: 1/tau = n T delta sqrt(2) / (mu(T)/mu(1)). */
    const double *tab_T, *tab_mu, *tab_Pr;
    int tab_n;
    int Nx;                  /* grid nodes across the full channel, >= 8 */
    double stretch_A;        /* Eq. stretch parameter A in [0, 1); 0 = uniform grid */
    int Qx;                  /* half-range quadrature order per half (2 Qx values of p_x) */
    int Qy;                  /* full-range quadrature order */
    int Nexp_x, Nexp_y;      /* expansion orders N < Q of Eqs. gx, gy; 0 = Q - 1 */
    double p0;               /* momentum scale of both quadratures; 0 = 1 */
    double cfl;              /* CFL number of the time step; 0 = 0.5 */
    double dt;               /* explicit time step; 0 = automatic (see lbc_create) */
    lbc_precision precision; /* LBC_FP64, or LBC_FP32_STATE (below) */
    int local_dt;            /* 0: one time step for every node (time-accurate);
                                1: local pseudo-time steps for steady states (below) */
    int half_channel;        /* 0: the full channel -1/2 < x < 1/2 with Nx nodes;
                                1: the half channel 0 < x < 1/2 with Nx nodes (below) */
    int compensated;         /* LBC_FP32_STATE only: 1 carries each state value's rounding
                                remainder from step to step (below); 0: plain FP32 state */
} lbc_params;

/*
 * FP32 state (precision LBC_FP32_STATE): the state and the stage arithmetic
 * (WENO-5, targets, relaxation, RK combination) are float32. Accumulations are
 * compensated: each node's raw moment sums are float32 partials over the 4 rows a
 * thread takes from each 32-row block of velocities, added into running sums with
 * Kahan's compensation, and the partials of warps and of velocity chunks with TwoSum;
 * the Hermite coefficients of the equilibrium are compensated dot products (Dot2);
 * the wall densities n_w are accumulated in float64. The steady-state residual takes
 * each value's increment in float32 (exact to one rounding) and reduces in float64.
 *
 * Compensated FP32 state (compensated = 1, precision LBC_FP32_STATE; LBC_EINVAL
 * otherwise). Each value of the state is held as an FP32 value d plus an FP32
 * remainder c, and each stage adds its dt L to a per-value FP32 accumulator of the
 * step's increment; the third stage adds Delta = dt (L0 + L1)/6 + (2/3) dt L2 to
 * d + c with the rounding error kept (TwoSum), so increments below half an ulp of d
 * still move the state and the increment is never rounded at the size of the state.
 * Without it an FP32 iteration stalls at a steady state biased by about
 * eps_32 |f| tau / dt (~1e-3 relative at delta = 0.1 on stretched grids); with it
 * the steady state is within 1e-5 of the FP64 one, although the residual itself
 * stays above ~1e-9 (the stage inputs are rounded to FP32). The stage arithmetic
 * stays FP32. lbc_get_state returns d + c and lbc_set_state stores the FP64 input
 * as d + c. lbc_step_noalloc rejects it.
 *
 * Local pseudo-time steps (local_dt = 1; dt must be 0). Only the steady state
 * is meaningful: node s advances by dt_s = min(cfl * J_s deta / max|p_x|,
 * tau_min / 2), the automatic step below with the CFL bound taken at each node,
 * so nodes in the coarse centre of a stretched grid take larger steps. The
 * fluxes then no longer telescope, so after each step the state is multiplied
 * by M_ref / M(f^n), where M(f) = sum_s J_s deta n_s is the mass of the step's
 * input and M_ref the mass at creation or at the last set_state. The fixed
 * point is the steady state of the global step with mass M_ref. The residual
 * is that of the pseudo-time iteration. lbc_step_noalloc rejects local_dt.
 *
 * Half channel (half_channel = 1): walls of equal temperature moving at -u_w
 * and +u_w (T_left = T_right, u_left = -u_right, else LBC_EINVAL). The flow
 * then has the symmetry phi(-x, -p_x, -p_y) = phi(x, p_x, p_y) (Sec. II), and
 * the solver integrates 0 < x < 1/2 only: Nx nodes, the right half of the
 * full-channel grid of 2 Nx nodes (the paper's S = Nx), with the ghost nodes
 * left of x = 0 taken from nodes 0, 1, 2 at the opposite velocity. States,
 * moments, node positions and masses refer to those Nx nodes.
 */

/*
 * Creates a solver for one Couette problem and sets the rest Maxwellian
 * n = 1, u = 0, T = 1 at every node.
 *   params: copied. Requires 1 <= Qx <= 64, 1 <= Qy <= 64, 2 Qx Qy <= 4096,
 *           0 <= N < Q (and N >= 2 on both axes, so the equilibrium has a
 *           temperature), Nx >= 8, delta >= 0, T_w > 0, 0 <= stretch_A < 1,
 *           p0 > 0; the largest orders must also fit one CTA's shared memory.
 *   Automatic time step: dt = min(cfl * min_s(J_s deta) / max|p_x|, tau_min / 2),
 *   with tau_min the smallest relaxation time (Eq. tau, with the problem's
 *   viscosity law) of the initial state and of the two walls at n = 1.
 *   cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 *   out: receives the handle; unchanged on failure.
 * Errors: LBC_EINVAL, LBC_ENOMEM, LBC_ECUDA.
 */
lbc_status lbc_create(const lbc_params *params, void *cuda_stream, lbc_solver **out);

/* Advances nsteps >= 0 RK-3 steps (three fused advect+collide stages each).
 * Enqueued only; returns before the GPU finishes. */
lbc_status lbc_step(lbc_solver *s, long nsteps);

/*
 * Steps until the per-step residual r_n = max_{field,v,s} w_v |ft^{n+1} - ft^n|
 * falls below `residual` (the paper states no criterion; this is the reading),
 * or max_steps more steps were taken. The state is left at the first step with
 * r < residual. steps_done / final_residual (either may be NULL) receive the
 * number of steps taken by this call and the last step's residual.
 * Errors: LBC_ENOTCONV (max_steps reached; state advanced by max_steps),
 * LBC_ESTALLED (the stall rule below ended the run), LBC_ENONFINITE, LBC_ECUDA,
 * LBC_EINVAL.
 */
lbc_status lbc_run_to_steady(lbc_solver *s, double residual, long max_steps,
                             long *steps_done, double *final_residual);

/*
 * Stall rule of lbc_run_to_steady / lbc_batch_run_to_steady (no counterpart in the
 * paper, which runs to a fixed residual; off by default). window > 0 steps: the
 * residual is sampled every 64 steps, and an instance none of whose samples over
 * its last `window` steps is below 0.99 times its lowest sample before them has
 * stalled: its residual has stopped setting new lows (an FP32 state's residual
 * wanders near 1e-9, the rounding noise of its stage inputs). It stops at the
 * sample, its state and steps_done are those of that sample, and final_residual
 * is its residual there (>= the threshold). A residual that still contracts sets
 * new lows however slowly (rate^window < 0.99); one that oscillates with a period
 * longer than the window, or rises for a whole window, is taken for stalled, so
 * the window is the caller's bound on such stretches. window = 0: off.
 * Errors: LBC_EINVAL (NULL handle, window < 0).
 */
lbc_status lbc_set_stall_window(lbc_solver *s, long window);

/*
 * Moments of the current state (Sec. II definitions), FP64, per node:
 *   out: caller-owned [LBC_NMOM][Nx], rows n, u_x, u_y, T, P_xx, P_yy, P_zz,
 *        P_xy, q_x, q_y (the paper's T_ij is the pressure tensor P_ij).
 *   x:   caller-owned [Nx] node positions, or NULL.
 * Synchronises the solver's stream. Errors: LBC_ECUDA, LBC_EINVAL.
 */
lbc_status lbc_moments(lbc_solver *s, double *out, double *x);

/* Copies the weight-divided state to / from caller-owned host memory
 * [2][V][Nx] float64. set_state converts to the solver's precision and
 * recomputes the stage moments. Synchronise the solver's stream. */
lbc_status lbc_get_state(lbc_solver *s, double *state);
lbc_status lbc_set_state(lbc_solver *s, const double *state);

/* Sizes and constants of a created solver (any pointer may be NULL); dt is the
 * global time step (with local_dt, the smallest node step). */
lbc_status lbc_info(const lbc_solver *s, int *Nx, int *V, double *dt, long *steps_taken);

/* Frees all device memory of the solver (stream-ordered). NULL is a no-op. */
void lbc_destroy(lbc_solver *s);

/* Thread-local description of the last error ("" if none). */
const char *lbc_last_error(void);

/*
 * Host-side building blocks (no GPU needed), for users that prepare inputs:
 *
 * lbc_quadrature: the Q-point Gauss rule of Sec. III in FP64.
 *   half_range != 0: weight exp(-z^2/2)/sqrt(2 pi) on [0, inf) (nodes > 0,
 *   weights sum to 1/2); else the full-range rule on the real line (weights sum
 *   to 1). nodes/weights: caller-owned [Q], ascending nodes. 1 <= Q <= 64.
 *
 * lbc_equilibrium: the weight-divided discrete equilibrium factors of Eqs. gx
 *   and gy at (u_x, u_y, T) for the orders and p0 of `params`:
 *   gx[2 Qx] (indexed like a), gy[Qy]; phi_eq/(w_a w_j) = n gx[a] gy[j],
 *   chi_eq = T phi_eq. Same algorithm as the device path, in FP64.
 */
lbc_status lbc_quadrature(int Q, int half_range, double *nodes, double *weights);
lbc_status lbc_equilibrium(const lbc_params *params, double ux, double uy, double T,
                           double *gx, double *gy);

/*
 * Batches: many independent Couette problems ("instances") stepped together,
 * one stage kernel launch per RK stage for the whole batch (no counterpart in
 * the paper, which solves one problem at a time; the discretisation of every
 * instance is exactly that of lbc_create).
 *
 * Each tile of 31 nodes of each instance is one work item; its velocity set is
 * split over `cluster` chunk CTAs (one thread-block cluster in the cluster
 * form, see below). Work items are scheduled longest first; instances of any
 * size, order and parameters mix freely. All instances of a batch share one
 * precision.
 *
 * lbc_batch_create: params[n] (copied), n >= 1; cluster = chunk CTAs per tile
 *   in [1, 16], or 0 to choose by a wave model of the whole batch.
 *   Errors: LBC_EINVAL (message names the instance), LBC_ENOMEM, LBC_ECUDA.
 * lbc_batch_step: nsteps RK-3 steps of every instance (enqueued only).
 *   LBC_ENONFINITE if an instance is poisoned (lbc_batch_set_state clears it).
 * lbc_batch_run_to_steady: every instance steps until its own residual (as in
 *   lbc_run_to_steady) falls below `residual`, or max_steps more steps; an
 *   instance that converged stops while the others go on. steps_done[n] and
 *   final_residual[n] (caller-owned, either may be NULL) receive each
 *   instance's steps taken by this call and its last step's residual.
 *   LBC_ENOTCONV if any instance reached max_steps (the others' results hold);
 *   else LBC_ESTALLED if the stall rule (lbc_set_stall_window; per batch:
 *   lbc_batch_set_stall_window) stopped any instance, the others converged.
 * lbc_batch_moments / get_state / set_state / info: as the single-solver calls,
 *   for instance i in [0, n).
 * lbc_batch_set_states: states[i] (caller-owned host [2][V_i][Nx_i] float64, or
 *   NULL to leave instance i as it is) for every instance in one call: all copies
 *   and conversions are enqueued back to back and checked once; if any state
 *   holds a NaN or Inf, no instance changes (LBC_EINVAL). Synchronises the
 *   stream twice, where n calls of lbc_batch_set_state synchronise 2n times.
 * lbc_batch_moments_all: the moments of every instance, the blocks
 *   [LBC_NMOM][Nx_i] of instances 0 .. n-1 back to back in `out` (caller-owned,
 *   sum_i LBC_NMOM Nx_i doubles); one synchronisation.
 * lbc_batch_shape: the launch shape (cluster size, work items, dynamic shared
 *   memory bytes of one stage CTA).
 * lbc_batch_autotune: for a batch whose instances have taken no step, times
 *   trial_steps steps for every feasible cluster size in the three kernel
 *   forms (below), and the solo and split forms with chunks of 256 velocity
 *   rows (each instance's last chunk shorter), and keeps the fastest; the instances are at their initial (rest)
 *   state afterwards. *cluster (may be NULL) receives the choice. Synchronises
 *   the stream.
 * Kernel forms of the batched stage launch (same arithmetic in the same order,
 * identical results): in the cluster form the chunk CTAs of a tile form one
 * thread-block cluster, exchange their moment partials through distributed
 * shared memory and each builds the next-stage data (moments, relaxation data,
 * equilibrium factors) of a share of the tile's nodes; in the solo form the
 * chunk CTAs are independent, write their partials to device memory and the
 * tile's last CTA to finish builds the data of all its nodes while the others
 * have left. lbc_batch_create picks the solo form when its work list fills the
 * device at least once, else the cluster form.
 * A third form, split, runs the solo form's independent chunk CTAs without the
 * node step and builds every tile's next-stage data in a second launch per
 * stage, spread over the whole GPU (same arithmetic, identical results).
 * lbc_batch_form: *solo = 0 cluster form (also for a single-instance batch),
 *   1 solo, 2 solo with 256-row chunks, 3 split, 4 split with 256-row chunks.
 *   Errors: LBC_EINVAL (NULL argument).
 * lbc_batch_set_form: forces the form of the per-stage launches (the persistent
 *   form below always runs the cluster form), with the codes of lbc_batch_form:
 *   0, 1 and 3 keep the cluster size; 2 and 4 use chunks of 256 velocity rows
 *   (each instance's last chunk shorter; the cluster size follows).
 *   Synchronises the stream. Errors: LBC_EINVAL (single-instance batch, form
 *   outside 0-4, a shape that does not fit), LBC_ECUDA.
 */
typedef struct lbc_batch lbc_batch;
lbc_status lbc_batch_create(const lbc_params *params, int n, int cluster, void *cuda_stream, lbc_batch **out);
lbc_status lbc_batch_step(lbc_batch *b, long nsteps);
lbc_status lbc_batch_run_to_steady(lbc_batch *b, double residual, long max_steps, long *steps_done,
                                   double *final_residual);
lbc_status lbc_batch_moments(lbc_batch *b, int i, double *out, double *x);
lbc_status lbc_batch_get_state(lbc_batch *b, int i, double *state);
lbc_status lbc_batch_set_state(lbc_batch *b, int i, const double *state);
lbc_status lbc_batch_set_states(lbc_batch *b, const double *const *states);
lbc_status lbc_batch_moments_all(lbc_batch *b, double *out);
lbc_status lbc_batch_info(const lbc_batch *b, int i, int *Nx, int *V, double *dt, long *steps_taken);
lbc_status lbc_batch_shape(const lbc_batch *b, int *cluster, int *nwork, size_t *smem_bytes);
lbc_status lbc_batch_autotune(lbc_batch *b, int trial_steps, int *cluster);
lbc_status lbc_batch_form(const lbc_batch *b, int *solo);
lbc_status lbc_batch_set_form(lbc_batch *b, int solo);
/* The stall rule of lbc_set_stall_window for every instance of the batch. */
lbc_status lbc_batch_set_stall_window(lbc_batch *b, long window);
/* As lbc_batch_step with eager launches, timing each stage launch with CUDA
 * events on the batch's stream; *stage_ms receives the sum of the 3 nsteps
 * stage-kernel durations (for roofline reports). Synchronises the stream. */
lbc_status lbc_batch_step_timed(lbc_batch *b, long nsteps, double *stage_ms);
/*
 * Persistent form (on != 0; no counterpart in the paper): each group of steps of the
 * whole batch runs as ONE cooperative launch whose thread-block clusters (as many as
 * can be resident, at most one per work item) take (step, stage, tile) items in order
 * from a device counter. An item starts when its tile and the two neighbouring tiles
 * (the WENO-5 stencil's halo) finished the previous stage; an instance with early stop
 * (lbc_batch_run_to_steady) or local steps also waits, at the first stage of a step,
 * for its whole previous step. Every wait is bounded (2 s): on timeout the launch
 * aborts and the instance reports LBC_ETIMEOUT. Results are bit-identical to the
 * per-stage launches. on = 0 returns to one launch per RK stage. Not available with
 * lbc_batch_step_timed (LBC_EINVAL). Errors: LBC_EINVAL (the launch shape does not fit
 * the device), LBC_ECUDA.
 */
lbc_status lbc_batch_set_persistent(lbc_batch *b, int on);
void lbc_batch_destroy(lbc_batch *b);

/*
 * Instance pool: problems that join and leave while others run, stepped
 * together by the batched stage kernel (continuous batching; no counterpart
 * in the paper). Each admitted instance gets its own stream-ordered device
 * allocation; admission is by device footprint against the pool's budget.
 *
 * lbc_pool_create: cluster = chunk CTAs per tile for every instance, in
 *   [1, 16] (instances whose velocity set needs more rows per CTA than 256 or
 *   more shared memory than one CTA has are rejected; for instances of at most
 *   256 velocities, 1 gives the most solves per second under load, larger
 *   clusters the lower latency at light load); precision of every
 *   instance; budget_bytes = device bytes the instances (tables and state, as
 *   lbc_pool_footprint) may use in total -- the pool adds a fixed part (slots,
 *   work list) and one staging buffer for state transfers of the largest
 *   instance admitted;
 *   max_instances slots; max_tiles = capacity of the work list (31-node tiles
 *   over all instances).
 * lbc_pool_footprint: device bytes an instance of `params` takes in a pool's budget.
 * lbc_pool_add: admits an instance at the rest state (as lbc_create); *slot
 *   receives its slot. LBC_ENOMEM when the budget, the slots or the work list
 *   are exhausted (nothing changes: the caller queues and retries later).
 *   Synchronises the stream.
 * lbc_pool_remove: frees the slot (stream-ordered).
 * lbc_pool_run: advances every instance up to nsteps steps; an instance stops
 *   at its first step whose residual (as lbc_run_to_steady) is below
 *   `residual`, and one that does not converge takes exactly nsteps steps (a
 *   caller may count those itself). finished[] (caller-owned, max_instances entries, may be NULL)
 *   receives the slots that converged and were not reported before,
 *   *nfinished their count; a reported instance left in the pool takes no
 *   further steps. Synchronises the stream.
 * lbc_pool_info / moments / get_state: as the single-solver calls for a slot;
 *   info also gives the last step's residual.
 * lbc_pool_usage: device bytes in use, instances, work items.
 */
typedef struct lbc_pool lbc_pool;
lbc_status lbc_pool_create(int cluster, lbc_precision precision, size_t budget_bytes, int max_instances,
                           int max_tiles, void *cuda_stream, lbc_pool **out);
lbc_status lbc_pool_footprint(const lbc_params *params, int cluster, size_t *bytes);
lbc_status lbc_pool_add(lbc_pool *pool, const lbc_params *params, int *slot);
lbc_status lbc_pool_remove(lbc_pool *pool, int slot);
lbc_status lbc_pool_run(lbc_pool *pool, double residual, long nsteps, int *finished, int *nfinished);
lbc_status lbc_pool_info(const lbc_pool *pool, int slot, int *Nx, int *V, double *dt, long *steps_taken,
                         double *last_residual);
lbc_status lbc_pool_usage(const lbc_pool *pool, size_t *used_bytes, int *instances, int *work_items);
lbc_status lbc_pool_moments(lbc_pool *pool, int slot, double *out, double *x);
lbc_status lbc_pool_get_state(lbc_pool *pool, int slot, double *state);
void lbc_pool_destroy(lbc_pool *pool);

/*
 * Allocation-free stepping (the paper has no counterpart: this serves callers
 * that cannot allocate device memory, e.g. code embedded in an application
 * whose own allocator owns the GPU memory, or latency-critical loops where the
 * implicit synchronisation of an allocation is not acceptable).
 *
 * Advances nsteps >= 0 RK-3 steps of the problem `params` (same validation and
 * discretisation as lbc_create) on a state the caller owns:
 *   d_state: DEVICE pointer to the weight-divided state, float64 [2][V][Nx]
 *            (the layout of lbc_get_state), read at entry and overwritten with
 *            the result. It is not aligned beyond 8 bytes by requirement.
 *   cuda_stream: a cudaStream_t or NULL (legacy default stream).
 * All other working memory (tables, RK buffers, moment partials, control
 * block) lives in one static device array of 8 MiB inside the library, which
 * every GPU that loads the library holds until the process exits. Problems
 * whose working set does not fit return LBC_EINVAL with the size needed.
 * Calls no cudaMalloc/cudaFree or other allocating routine. The first call on
 * each device resolves the array's device address (cudaGetSymbolAddress) and
 * sets kernel attributes; make that first call before any stream capture on
 * that device. Every call shares the array and clears what must start at zero;
 * calls whose GPU work overlaps (other streams or threads) race on it and must
 * be serialised by the caller. Returns after the work has finished
 * (synchronises the stream).
 * Errors: LBC_EINVAL, LBC_ECUDA, LBC_ENONFINITE, LBC_ETIMEOUT.
 */
lbc_status lbc_step_noalloc(const lbc_params *params, double *d_state, long nsteps, void *cuda_stream);

/*
 * Measurement helper (no counterpart in the paper): the device's FP64 FMA rate in
 * TFLOP/s, measured by timing independent FMA chains on every SM with CUDA events
 * (best of three launches after a warm-up), for the roofline of the FP64 path.
 * Uses the current device; changes no device setting. Errors: LBC_EINVAL, LBC_ECUDA.
 */
lbc_status lbc_measure_fp64_peak(double *tflops);

/*
 * Build variant (no counterpart in the paper): 1 if this library is the
 * range-checked build (liblbc_checked.so, kernels compiled with LBC_CHECKED),
 * else 0. In that build the stage, equilibrium and persistent kernels check
 * their computed indices (TMA box alignment, bulk-copy extents, stencil and
 * ghost columns, factor-table indices, state stores, symmetry partners,
 * cluster exchange slots, persistent work neighbours) before each access; a
 * failed check skips the access, records its site in the instance's control
 * block, and the next call that reads the control blocks returns LBC_EBOUNDS
 * naming the site; stepping is then refused until a state is installed.
 * Never fails.
 */
int lbc_checked_build(void);

#ifdef __cplusplus
}
#endif
#endif /* LBC_H */
