/*
 * plan.h -- C ABI of the GB300 three-weight ADMM (TWA) multi-agent trajectory
 * planner.
 *
 * The method is the message-passing planner of Bento, Derbinsky, Alonso-Mora
 * and Yedidia, "A message-passing algorithm for multi-agent trajectory
 * planning" (NIPS 2013).  The problem (Section 1): p disk agents with radii
 * r_i move in the plane from start x_i(0) to goal x_i(T) along piecewise
 * linear paths with eta segments and shared break-points s = 0..eta; the
 * paths must not collide (Eq. basic_opt_prob) and minimise the kinetic energy
 * (Eq. velo_cost_pair_wise), optionally avoiding wall segments
 * (Eq. wall_minimizer).  One iteration (Appendix B, steps 1-7) updates every
 * collision, kinetic, wall and position factor of the graph of Section 3.3,
 * then the consensus z per break-point and the dual u per edge.
 *
 * Conventions for every entry point:
 *  - every call returns a plan_status; nothing throws across the ABI; the
 *    message of the last failure on the calling thread is plan_last_error();
 *  - arrays are float32, row-major, 2-D points stored as (x, y) pairs;
 *  - "host" pointers are ordinary CPU memory (pinned memory is faster);
 *    "device" pointers are CUDA global memory on the plan's device;
 *  - the library never keeps a caller pointer past the call, except the
 *    workspace handed to plan_create, which the caller keeps alive until
 *    plan_destroy;
 *  - work is enqueued on the stream given to plan_create; only calls that
 *    return a number to the host (residual, iteration count, host copies)
 *    synchronise that stream.
 */
#ifndef PLAN_H
#define PLAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct plan_s* plan_t;

typedef enum {
  PLAN_OK = 0,
  PLAN_EINVAL = 1,             /* bad argument (null pointer, size, flag) */
  PLAN_ENOMEM = 2,             /* allocation failed or workspace too small */
  PLAN_ECUDA = 3,              /* a CUDA call failed; see plan_last_error() */
  PLAN_ENOTCONV = 4,           /* plan_solve hit max_iter before tol */
  PLAN_ENUMERIC = 5,           /* a non-finite value appeared in the iterate */
  PLAN_EINFEASIBLE_INPUT = 6,  /* overlapping starts/goals, endpoint in a wall */
  PLAN_EUNSUPPORTED = 7        /* a mode this build does not implement */
} plan_status;

/* flags of plan_config.flags */
#define PLAN_U_KEEP            (1u << 0) /* inactive edges keep u instead of resetting it to 0 */
#define PLAN_COST_UNNORM       (1u << 1) /* kinetic coefficient C_{i,s} instead of C_{i,s}/(p eta) */
#define PLAN_COST_PER_SEGMENT  (1u << 2) /* cost_w holds p x eta values C_{i,s} (else p values C_i) */
#define PLAN_DENSE_STATE       (1u << 3) /* stream the u record of every collision factor each
                                            iteration, zeros included (else only active ones) */
#define PLAN_ADMM              (1u << 4) /* standard ADMM (App. B): every factor always sends
                                            rho0; implies the dense state */
#define PLAN_NO_ENERGY         (1u << 5) /* no kinetic factors: the feasibility problem of
                                            Eq. basic_opt_prob (Section 4); break-points
                                            can then receive only zero weights */
#define PLAN_VMAX              (1u << 6) /* a maximum-velocity factor per agent segment,
                                            |x(s+1) - x(s)| <= vmax (Eq. max_vel_min, App. F) */
#define PLAN_VMIN              (1u << 7) /* a minimum-velocity factor per agent segment,
                                            |x(s+1) - x(s)| >= vmin (the reversed Eq.
                                            max_vel_min, App. G) */
#define PLAN_VO                (1u << 8) /* one velocity-obstacle epoch (Section 5, App. H):
                                            eta = 2, start = x(0), goal = x_ref; collision,
                                            wall and velocity factors on segment 0 only, the
                                            kinetic factor C'_i |x - x_ref|^2 (cost_w,
                                            unnormalised) on segment 1 only */
#define PLAN_U_LITERAL         (1u << 9) /* dual step u += (alpha / rho) (x - z) as printed in
                                            App. B step 7, rho the value in force in that
                                            iteration (warm_rho during the warm-up); without
                                            it u += alpha (x - z) (the scaled-dual form, the
                                            same when rho = 1) */

typedef struct {
  int p;              /* agents, >= 1 */
  int eta;            /* segments, >= 1; break-points s = 0..eta */
  float T;            /* horizon; kept for the caller, the cost does not use it */
  float rho0;         /* rho0 of the three weights {0, rho0, inf} (Section 2), > 0 */
  float alpha;        /* dual step of Appendix B step 7 (the paper uses 0.1), > 0 */
  int warm_iters;     /* iterations at rho = warm_rho before rho0 (Section 4); 0 = off */
  float warm_rho;
  float tol;          /* plan_solve stops when the residual falls below tol */
  int max_iter;       /* plan_solve gives up after this many iterations */
  int check_every;    /* plan_solve reads the residual back every this many iterations (>=1) */
  int n_walls;        /* wall segments, >= 0 */
  unsigned flags;     /* PLAN_* flags above */
} plan_config;

/* Bytes of device workspace plan_create needs for cfg (cfg->p, eta, n_walls,
 * flags).  Errors: PLAN_EINVAL for a null pointer or sizes out of range. */
plan_status plan_workspace_size(const plan_config* cfg, size_t* bytes);

/*
 * Build a planner for one problem (Section 1) and set the initial state of
 * Section 4: z = start at every break-point except the goal node, u = 0.
 *
 *   start, goal : host, p x 2          fixed positions at s = 0 and s = eta
 *   radius      : host, p              agent radii r_i > 0
 *   cost_w      : host, p (or p x eta with PLAN_COST_PER_SEGMENT), >= 0,
 *                 the C_{i,s} of Eq. velo_cost_pair_wise
 *   walls       : host, n_walls x 4    rows [xL.x, xL.y, xR.x, xR.y]
 *                 (Eq. wall_minimizer); may be NULL when n_walls == 0
 *   workspace   : device memory of plan_workspace_size() bytes, 256-byte
 *                 aligned, owned by the caller; NULL makes the library
 *                 allocate (and free) its own
 *   cuda_stream : cudaStream_t to enqueue on (NULL = legacy default stream)
 *
 * Errors: PLAN_EINVAL (null pointers, non-finite values, sizes),
 * PLAN_EINFEASIBLE_INPUT (two starts or two goals closer than r_i + r_j, or an
 * endpoint closer than r_i to a wall), PLAN_ENOMEM, PLAN_ECUDA.
 */
plan_status plan_create(const plan_config* cfg, const float* start, const float* goal,
                        const float* radius, const float* cost_w, const float* walls,
                        void* workspace, size_t workspace_bytes, void* cuda_stream,
                        plan_t* out);

/* Back to the initial state (iteration counter 0).  Enqueued, no sync. */
plan_status plan_reset(plan_t plan);

/* Replace the fixed start and goal positions (host, p x 2 each) and keep the
 * current iterate as the warm start (the re-planning use of Appendix J).  The
 * new endpoints are checked like in plan_create (on the device for
 * p <= 8192, on the host above); a failed check leaves the plan unchanged.
 * Copies are enqueued on the plan's stream; the call returns once the host
 * buffers may be reused.  Errors: PLAN_EINVAL (null pointers, a non-finite
 * coordinate), PLAN_EINFEASIBLE_INPUT (overlapping starts or goals, an
 * endpoint within its radius of a wall), PLAN_ECUDA. */
plan_status plan_set_endpoints(plan_t plan, const float* start, const float* goal);

/* plan_set_endpoints without waiting for the check (p <= 8192, where the
 * check runs on the device; else PLAN_EUNSUPPORTED): the new endpoints are
 * checked and, only if they pass, applied on the device in stream order
 * before any work enqueued later; the call returns once the host buffers may
 * be reused.  A failed check is reported as PLAN_EINFEASIBLE_INPUT (or
 * PLAN_EINVAL for a non-finite coordinate) by the
 * next call on this plan that synchronises its stream (plan_iterate with a
 * residual, plan_solve, plan_get_trajectory to the host, plan_check,
 * plan_get_info, plan_get_endpoints, plan_set_params, plan_set_endpoints, or
 * the next plan_set_endpoints_async, which then takes no new endpoints); the
 * plan keeps its previous endpoints, and the iterations enqueued in between
 * ran with them.  Errors returned directly: PLAN_EINVAL (null input),
 * PLAN_EUNSUPPORTED, PLAN_ECUDA. */
plan_status plan_set_endpoints_async(plan_t plan, const float* start, const float* goal);

/* Run k_iters TWA iterations (Appendix B steps 1-7 over every factor).  When
 * max_residual is non-NULL the call synchronises and stores the residual of
 * the last iteration: max over weighted edges of |x - z|_inf and over nodes
 * of |z_new - z_old|_inf.  Errors: PLAN_EINVAL, PLAN_ECUDA. */
plan_status plan_iterate(plan_t plan, int k_iters, float* max_residual);

/* Iterate until the residual falls below cfg.tol (checked every
 * cfg.check_every iterations) or cfg.max_iter iterations have run.  Returns
 * PLAN_OK on convergence, PLAN_ENOTCONV at max_iter, PLAN_ENUMERIC on a
 * non-finite residual.  iters_done / max_residual may be NULL. */
plan_status plan_solve(plan_t plan, int* iters_done, float* max_residual);

/* Copy the break-points z (p x (eta+1) x 2) to z; on_device selects a device
 * or host destination.  A host copy synchronises. */
plan_status plan_get_trajectory(plan_t plan, float* z, int on_device);

/*
 * State exchange in the paper's variables (Appendix B), all DEVICE pointers
 * (any of them may be NULL to skip that array):
 *   z       : p x (eta+1) x 2
 *   u_coll  : eta x P x 4 x 2, P = p(p-1)/2 pairs (i < j) in lexicographic
 *             order; edges (i,s), (i,s+1), (j,s), (j,s+1)
 *   u_kin   : eta x p x 2 x 2, edges (i,s), (i,s+1)
 *   u_wall  : n_walls x eta x p x 2 x 2
 *   act_coll: eta x P bytes, 1 where the factor sent rho0 in the last
 *             iteration (export only)
 *   act_wall: n_walls x eta x p bytes (export only)
 * plan_export_state writes the state at the start of the next iteration;
 * plan_import_state replaces it (k = iteration counter to resume from); it
 * needs z and u_kin, u_coll when p > 1 and u_wall when n_walls > 0.
 */
plan_status plan_export_state(plan_t plan, float* z, float* u_coll, float* u_kin, float* u_wall,
                              uint8_t* act_coll, uint8_t* act_wall, int* k);
plan_status plan_import_state(plan_t plan, const float* z, const float* u_coll,
                              const float* u_kin, const float* u_wall, int k);

typedef struct {
  long long n_coll;          /* collision factors eta p (p-1)/2 */
  long long n_kin;           /* kinetic factors eta p */
  long long n_wall;          /* wall factors n_walls eta p */
  long long n_pos;           /* position factors 2 p */
  long long active_coll;     /* collision factors active in the last iteration */
  long long active_wall;     /* wall factors active in the last iteration */
  int k;                     /* iterations done */
  int tile;                  /* agents per tile of the collision kernel */
  size_t workspace_bytes;
} plan_info;

/* Sizes and counters (synchronises to count the active factors). */
plan_status plan_get_info(plan_t plan, plan_info* info);

/*
 * Final feasibility and cost check of the current break-points z, in FP64 on
 * the device (the FP32 z promoted exactly):
 *   total_cost         : sum over agents and kinetic segments of
 *                        c_{i,s} |z_i(s+1) - z_i(s)|^2, the cost of Eq.
 *                        velo_cost_pair_wise (c_{i,s} = C_{i,s} / (p eta), or
 *                        C_{i,s} with PLAN_COST_UNNORM);
 *   min_pair_clearance : min over pairs i < j and segments s of the smallest
 *                        distance between the two agents along the segment
 *                        (linear motion between break-points) divided by
 *                        r_i + r_j; Eq. basic_opt_prob holds when it is >= 1
 *                        (+inf when p = 1);
 *   min_wall_clearance : min over walls, agents and segments of the distance
 *                        between the agent's segment and the wall segment
 *                        divided by r_i (+inf without walls);
 *   max_endpoint_error : max over agents of |z_i(0) - start_i|_inf and
 *                        |z_i(eta) - goal_i|_inf.
 * For a PLAN_VO plan the clearances cover segment 0 and the cost segment 1
 * (the local planner's graph).  All pointers are HOST doubles and may be
 * NULL.  Synchronises.  Errors: PLAN_EINVAL (null plan), PLAN_ECUDA.
 */
plan_status plan_check(plan_t plan, double* total_cost, double* min_pair_clearance,
                       double* min_wall_clearance, double* max_endpoint_error);

/* Per-kernel timing of the next iterations (CUDA events on the plan's
 * stream).  enable = 1 starts collecting (and synchronises once per
 * iteration, so timings are taken without overlap between iterations);
 * enable = 0 stops and writes the average milliseconds per iteration of the
 * three kernels to ms[0..3] = {pass 1: collision tests, with the kinetic
 * factors and wall tests in the same launch; pass 2: wall and collision
 * minimizers; 0 (no separate kinetic / wall launch); consensus} and their
 * count to *iterations (either may be NULL).  Errors: PLAN_EINVAL (a batch
 * member), PLAN_ECUDA. */
plan_status plan_profile(plan_t plan, int enable, float* ms, int* iterations);

/*
 * Batches: n independent problems (uneven p, eta, walls) advanced together.
 * Every pass of an iteration is one launch over all members' blocks, and
 * iterations are replayed from CUDA graphs (the spec batching form; the
 * paper solves one problem at a time).  Members must share the state-mode
 * flags (PLAN_DENSE_STATE, PLAN_U_KEEP, PLAN_ADMM).  Arguments are arrays of
 * n host pointers laid out as for plan_create; walls may be NULL (no member
 * has walls) or hold NULL entries.  workspace: plan_batch_workspace_size()
 * bytes of device memory, 256-byte aligned, or NULL to let the library
 * allocate.  Errors as for plan_create, with the member index in the message.
 */
typedef struct plan_batch_s* plan_batch_t;
plan_status plan_batch_workspace_size(int n, const plan_config* cfgs, size_t* bytes);
plan_status plan_batch_create(int n, const plan_config* cfgs, const float* const* start,
                              const float* const* goal, const float* const* radius,
                              const float* const* cost_w, const float* const* walls,
                              void* workspace, size_t workspace_bytes, void* cuda_stream,
                              plan_batch_t* out);
/* k_iters iterations of every member not yet converged (enqueued, no sync). */
plan_status plan_batch_iterate(plan_batch_t batch, int k_iters);
/* Iterate until every member's residual is below its tol or it reached its
 * max_iter (checked every min check_every iterations, rounded up to even);
 * converged members are frozen.  iters_done / residual: n host values (may be
 * NULL): the iteration at which each member converged (or the last one run)
 * and its last residual.  n_converged: how many converged.  PLAN_ENUMERIC on
 * a non-finite residual. */
plan_status plan_batch_solve(plan_batch_t batch, int* iters_done, float* residual,
                             int* n_converged);
/* Break-points of one member, as plan_get_trajectory. */
plan_status plan_batch_get_trajectory(plan_batch_t batch, int member, float* z, int on_device);
/* One member's state in the paper's variables, as plan_import_state /
 * plan_export_state (DEVICE pointers, the same layouts).  An imported state
 * becomes the member's state at the batch's current iteration (members
 * advance together) and unfreezes the member.  Both synchronise the batch's
 * stream.  Errors: PLAN_EINVAL (null batch or pointers, member out of
 * range), PLAN_ECUDA. */
plan_status plan_batch_import_state(plan_batch_t batch, int member, const float* z,
                                    const float* u_coll, const float* u_kin, const float* u_wall);
plan_status plan_batch_export_state(plan_batch_t batch, int member, float* z, float* u_coll,
                                    float* u_kin, float* u_wall, uint8_t* act_coll,
                                    uint8_t* act_wall);
/* Time the launch-shape candidates (rows per warp of the collision test
 * {4, 8, 16}, or 32: one warp per tile with lane = row agent, gated state
 * only; minimizer CTAs per SM {1, 2, 4} x the base grid; iterations per
 * graph {2, 8}) on this batch, iters_per_candidate iterations each (they are
 * real iterations: results do not depend on the shape), and keep the fastest.
 * choice: 3 host ints receiving the chosen values (may be NULL). */
plan_status plan_batch_autotune(plan_batch_t batch, int iters_per_candidate, int* choice);
/* Set the launch shape directly (for example one found by the autotuner on
 * another batch of the same instances): rows_per_warp in {4, 8, 16, 32},
 * prox_ctas_per_sm in 1..8, iterations_per_graph even and >= 2. */
plan_status plan_batch_set_shape(plan_batch_t batch, int rows_per_warp, int prox_ctas_per_sm,
                                 int iterations_per_graph);
void plan_batch_destroy(plan_batch_t batch);

/*
 * Velocity limits and the feasibility problem (Section 3.3 "minimum energy
 * and maximum (minimum) velocity minimizer", Appendices F and G, Section 4).
 *
 * plan_set_velocity_limits: host arrays p x eta of the per-segment limits on
 * |x_i(s+1) - x_i(s)| (distance per segment); vmax needs PLAN_VMAX (values
 * > 0, +inf allowed), vmin needs PLAN_VMIN (finite, >= 0); either may be NULL
 * to keep the current values.  Until set, maxima are +inf and minima 0 (no
 * factor ever activates).  Each factor sends rho0 while the n-messages
 * violate its limit and 0 otherwise.
 *
 * plan_export_velocity_state / plan_import_velocity_state: the velocity
 * factors' u (DEVICE, eta x p x 2 x 2, edges (i,s), (i,s+1)) and activity
 * (eta x p bytes, export only); any pointer may be NULL.  plan_import_state
 * resets these to 0, so import them after it.
 *
 * plan_set_energy(plan, 0) switches the kinetic factors off from the next
 * iteration (the feasibility problem from the current state: the paper's
 * recovery of collision-free paths from a solve stopped early); 1 switches
 * them back on with their u restarted at 0.  Without kinetic factors a
 * break-point whose factors all sent 0 gets back weight 0 (App. B step 6),
 * and the minimizers take the limit of that weight -> 0+.
 *
 * Not combined with PLAN_ADMM; batches, plan_iterate_static and the adjoint
 * return PLAN_EUNSUPPORTED for these modes.
 */
plan_status plan_set_velocity_limits(plan_t plan, const float* vmax, const float* vmin);
plan_status plan_export_velocity_state(plan_t plan, float* u_vmax, float* u_vmin,
                                       uint8_t* act_vmax, uint8_t* act_vmin);
plan_status plan_import_velocity_state(plan_t plan, const float* u_vmax, const float* u_vmin);
plan_status plan_set_energy(plan_t plan, int on);
/* Copy the current fixed positions (start, goal; host, p x 2 each, either may
 * be NULL).  Synchronises. */
plan_status plan_get_endpoints(plan_t plan, float* start, float* goal);
/* One epoch of the velocity-obstacle local planner (Section 5) on a PLAN_VO
 * plan: set x_ref = x(0) + (dest - x(0)) clipped to length step (the
 * preferred velocity times the horizon), reset to the initial state, solve
 * (cfg.tol / max_iter / check_every), then move x(0) a fraction advance in
 * (0, 1] of the way to the planned x.  dest: DEVICE p x 2.  iters / residual
 * (may be NULL): the solve's iterations and last residual; max_dist: the
 * largest remaining distance to dest.  Returns PLAN_ENOTCONV when the solve
 * hit max_iter (x(0) still advances), else as plan_solve.  Synchronises. */
plan_status plan_vo_epoch(plan_t plan, const float* dest, float step, float advance, int* iters,
                          float* residual, float* max_dist);
/* Back-weight class of every break-point (App. B step 6), DEVICE p x (eta+1)
 * bytes: 0 zero, 1 rho0, 2 infinite (the fixed ends).  Export works in every
 * mode; import (feasibility problem only; fixed ends ignored) replaces the
 * classes that plan_import_state / plan_import_velocity_state otherwise infer
 * from which imported u are nonzero. */
plan_status plan_export_back_weights(plan_t plan, uint8_t* classes);
plan_status plan_import_back_weights(plan_t plan, const uint8_t* classes);
/* Replace the radii (host, p) and/or the kinetic cost weights (host, laid
 * out as cost_w of plan_create) and keep the current iterate; either pointer
 * may be NULL.  New radii are checked against the endpoints like in
 * plan_create.  Returns once the host buffers may be reused. */
plan_status plan_set_params(plan_t plan, const float* radius, const float* cost_w);
/*
 * Differentiation through K unrolled iterations (the paper differentiates
 * nothing; this serves callers that fit starts, goals, radii or cost weights
 * to a loss on the planned trajectory).
 *
 * plan_unroll resets the plan to the initial state of Section 4 for its
 * current inputs and runs K iterations of Appendix B, keeping a copy of the
 * device state every checkpoint_every iterations (0 = ceil(sqrt(K))) and at
 * iteration K; afterwards the trajectory is z^K (plan_get_trajectory).  The
 * copies live in device memory that the library allocates on first use and
 * frees in plan_destroy: about ceil(K / C) + 1 copies of the iteration state
 * plus C recorded iterations, C = checkpoint_every.
 *
 * plan_backward returns the gradient of a loss L(z^K) given dL_dz = dL/dz^K
 * (DEVICE, p x (eta+1) x 2), with every branch choice of the forward run held
 * fixed: which collision factors were active in each iteration and which
 * candidate direction each minimizer took (Appendix C).  It replays the
 * iterations segment by segment from the checkpoints and runs the adjoint of
 * each iteration in reverse.  Outputs are DEVICE arrays: d_start, d_goal
 * (p x 2), d_radius (p), d_cost_w (laid out as cost_w).  K must be the K of
 * the last plan_unroll, with no state change in between (else PLAN_EINVAL);
 * the plan is left at iteration K, and plan_backward may be called again
 * with another dL_dz.  Wall and velocity-limit factors are differentiated
 * like collision factors, and a PLAN_VO plan gives the gradient of one
 * local-planner epoch (start = x(0), goal = x_ref, cost_w = C'); the
 * feasibility problem (PLAN_NO_ENERGY or plan_set_energy(plan, 0)),
 * PLAN_ADMM, PLAN_U_KEEP and a rho warm-up give PLAN_EUNSUPPORTED.
 * Enqueued on the plan's stream.
 */
plan_status plan_unroll(plan_t plan, int K, int checkpoint_every);
plan_status plan_backward(plan_t plan, int K, const float* dL_dz, float* d_start, float* d_goal,
                          float* d_radius, float* d_cost_w);

/*
 * One iteration without any allocation, for callers that cannot allocate GPU
 * memory: code whose device memory is owned by a host framework or a memory
 * pool it may not bypass, real-time control loops where cudaMalloc is banned
 * because it can synchronise the device and take unbounded time, and plugins
 * loaded into processes whose allocator belongs to someone else.  The paper
 * has no counterpart; this is a packaging of plan_iterate for those callers.
 *
 * It runs the same kernels as plan_iterate on one iteration of the paper's
 * variables: (z_in, u_*_in) at iteration k -> (z_out, u_*_out) at k + 1,
 * with the layouts of plan_export_state.  Every pointer is DEVICE memory on
 * the current device: the problem arrays (start, goal, radius, cost_w,
 * walls, laid out as for plan_create; walls may be NULL when n_walls == 0,
 * u_coll_* when p == 1, u_wall_* when n_walls == 0, act_* may be NULL) and
 * the state in and out (in and out must not overlap).  The endpoints are not
 * checked for overlap: that check needs host copies.
 *
 * All temporaries live in one file-scope device array of
 * PLAN_STATIC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * holds until the process exits.  Problems whose workspace
 * (plan_workspace_size) exceeds it are rejected with PLAN_ENOMEM.  The first
 * call on a device looks the array's address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call reuses the same array, so calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * Work is enqueued on cuda_stream; the call does not synchronise, so a
 * numeric failure cannot be returned as a status: when a message of the
 * iteration is non-finite or beyond the fixed-point range of the consensus
 * sums (the case plan_iterate reports as PLAN_ENUMERIC), every entry of z_out
 * is set to NaN.  Errors returned: PLAN_EINVAL (null pointers, sizes, flags,
 * rho0 / alpha / warm_rho not positive), PLAN_EUNSUPPORTED, PLAN_ENOMEM
 * (problem too large for the array), PLAN_ECUDA.
 */
#define PLAN_STATIC_SCRATCH_BYTES (16u << 20)
plan_status plan_iterate_static(const plan_config* cfg, const float* start, const float* goal,
                                const float* radius, const float* cost_w, const float* walls,
                                const float* z_in, const float* u_coll_in, const float* u_kin_in,
                                const float* u_wall_in, float* z_out, float* u_coll_out,
                                float* u_kin_out, float* u_wall_out, uint8_t* act_coll_out,
                                uint8_t* act_wall_out, int k, void* cuda_stream);

void plan_destroy(plan_t plan);
const char* plan_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PLAN_H */
