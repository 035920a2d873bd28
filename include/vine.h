/*
 * vine.h -- C ABI of the GB300 library for the batched quasi-static growth
 * step of planar vine robots, "Parallel Simulation of Contact and Actuation
 * for Soft Growing Robots" (arXiv 2509.15180).
 *
 * What one growth step computes (Sec. 3-4 of the paper):
 *   - a link is added at the tip (Sec. 4.1: only the distal length l_last
 *     changes; every other link keeps length l_seg),
 *   - per joint, the wrinkling-based restoring moment of the inflated body
 *     (Sec. 3.2, Eq. wrinkling_model) and the moment of every sPAM actuator
 *     covering the joint (Sec. 3.1, Eq. sPAM_model; Sec. 3.3,
 *     Eq. restoring_moment) are summed,
 *   - every link is tested against the robot's obstacles for penetration,
 *   - the cost of Eq. (pbd) (weights w_a, w_b, w_c of Sec. 4.1, used in
 *     potential form so that its stationary point is the moment balance with
 *     contact forces) is brought to equilibrium from the previous state
 *     (Algorithm 1, read as "the equilibrium reached from the warm start").
 *
 * Conventions for every entry point:
 *   - Return value: vine_status.  No C++ exception crosses this boundary.
 *     On failure vine_last_error() returns a thread-local message.
 *   - Per-instance failures do not fail a call; they are reported in the
 *     per-instance status (vine_inst_status).
 *   - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default
 *     stream).  Calls that only enqueue device work are asynchronous on that
 *     stream.  Calls that read or write HOST memory synchronise the stream
 *     before returning.
 *   - Ownership: inputs are caller-owned and are copied during the call;
 *     the caller may free them afterwards.  Outputs go to caller buffers.
 *     Opaque handles are library-owned and released by the matching
 *     *_destroy call.
 *   - Units: SI (m, Pa, N, rad).  Link indices and actuator spans are in
 *     link units (link k covers [k, k+1)).
 */
#ifndef VINE_H_
#define VINE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VINE_OK = 0,
  VINE_EINVAL = 1,         /* malformed argument or descriptor */
  VINE_ENOMEM = 2,         /* device allocation failed */
  VINE_ECUDA = 3,          /* CUDA runtime error (message in vine_last_error) */
  VINE_ETIMEOUT = 4,       /* a bounded wait ran out */
  VINE_EBUSY = 5,          /* admission refused, retry later */
  VINE_ENOTCONVERGED = 6   /* reserved */
} vine_status;

typedef enum {
  VINE_INST_OK = 0,        /* every step converged */
  VINE_INST_MAXITER = 1,   /* a step did not reach the tolerance (max_iter, or no
                              acceptable line-search trial); the instance stopped
                              there: later steps would start from a state that is
                              not an equilibrium */
  VINE_INST_NONFINITE = 2, /* the state became NaN/Inf; the instance stopped */
  VINE_INST_BADINPUT = 3   /* invalid design or obstacle values; never stepped */
} vine_inst_status;

/* Model and solver constants.  Fill with vine_params_default().
 * w_a, w_b, w_c: weights of Eq. (pbd), Sec. 4.1 (160, 15, 1).
 * eps_crit: critical wrinkling strain of Sec. 3.2 (fitted in the paper, value
 *   not printed; default 0.01).
 * R_c, R_act, a_spam: sPAM constants of Sec. 3.1 / 4.2 (5 mm, 17.18 mm, 1e-4).
 * m_lo: lower end of the contraction parameter range of the force table (0.002).
 * pen_frac: contact stiffness k_c = w_a pi P R^3 / (2 pen_frac R l_seg) (0.01).
 * tol, tol_link: a growth step has converged when the Newton step predicts
 *   no displacement of a link end point (nor l_seg times a joint step)
 *   larger than tol times the robot length N l_seg (1e-6) and no larger
 *   than tol_link link lengths (default 2.5e-5; <= 0 drops this bound).
 *   The second bound keeps converged states within 1e-4 link lengths of
 *   the equilibrium at any chain length.  The displacement sums are
 *   float-float, the test is decided in FP64.
 * fval_eps, armijo_c1: every step is line-searched on the projected path
 *   (at most max_halvings halvings): accepted when the cost decreases by
 *   armijo_c1 times the predicted decrease (Armijo), or, when the cost change
 *   is within fval_eps times the sum of the magnitudes of the cost's terms
 *   (each contact counted at w_c k_c (pen^2 + 2 R pen)) -- the rounding
 *   level of the FP32 evaluation -- when the directional slope
 *   there is at most (2 armijo_c1 - 1) times the initial slope (approximate
 *   Wolfe condition of Hager and Zhang, 2005).  Defaults 1e-6, 1e-4.
 * max_iter: Gauss-Newton iterations per growth step (100).
 * discs_per_link: contact discs K_s of radius R at fractions k/K_s of each
 *   link (2; 1..4 supported).
 * mode: 0 = each step solved to equilibrium (default); 1 = Algorithm 1 of
 *   Sec. 4.1 read literally: the actuator forces are evaluated once per step
 *   at the step's initial joint strains and held, then gd_steps steps of
 *   gradient descent on the cost (no convergence test; every completed step
 *   counts in robot_link_steps).  The printed learning rate is not given and
 *   would mix units, so the joint angles step by gd_alpha 2 theta_c /
 *   (w_a pi P R^3) times their gradient (gd_alpha times the inverse slope of
 *   the moment ramp below wrinkling onset) and the distal length by
 *   gd_alpha / (2 w_b k_g) times its gradient, kept in [0, l_seg].
 * gd_alpha, gd_steps: mode 1 step fraction (0.005) and steps (50).
 * exact_hessian: 1 = Newton steps with the exact Hessian of the cost when it
 *   is positive definite, else with the Gauss-Newton matrix (contact second
 *   derivatives dropped); 0 = always Gauss-Newton (default 1).
 * threads_per_robot: 32 = one warp grows a robot (several robots per CTA);
 *   64 or 128 = two or four warps of one CTA share a robot's link loops,
 *   which shortens each robot's evaluation at the cost of fewer robots per
 *   SM.  0 (default) chooses by the batch's longest robot: 32 up to 64
 *   links, 64 up to 200, else 128 (measured on the design, robustness and
 *   uneven batches).  Team sizes agree to rounding (sums over different
 *   thread counts round differently), not bitwise.  The serving loop takes
 *   the same rule with its slot capacity in links.
 * broad_phase: 1 = each link tests only the obstacles on a list built when
 *   it last moved by more than 0.4 body radii (the result is the same as
 *   with 0, which tests every obstacle at every evaluation; default 1). */
typedef struct {
  double w_a, w_b, w_c;
  double eps_crit;
  double R_c, R_act, a_spam;
  double m_lo;
  double pen_frac;
  double tol;
  double fval_eps;
  double armijo_c1;
  int32_t max_iter;
  int32_t discs_per_link;
  int32_t max_halvings;
  int32_t mode;
  double gd_alpha;
  int32_t gd_steps;
  int32_t exact_hessian;
  int32_t broad_phase;
  int32_t threads_per_robot;
  double tol_link;
} vine_params;

/* Batch of independent robot instances, structure-of-arrays with CSR
 * offsets.  All pointers are caller-owned; mem_is_device = 0 means host
 * memory, 1 means device memory of the current device.
 *   n_links[n]      target link count (>= 1); one link grows per step
 *   l_seg[n]        segment length (m, > 0)
 *   radius[n]       body radius R_vine (m, > 0)
 *   pressure[n]     body pressure P_vine (Pa, > 0)
 *   base[3n]        base x, y (m) and heading (rad)
 *   act_ptr[n+1]    actuators of instance i are act_ptr[i] .. act_ptr[i+1]-1
 *   act_begin/end   span [begin, end) in link units, 0 <= begin < end
 *   act_side        +1 / -1: side the actuator pulls toward
 *   act_pressure    actuation pressure P_act (Pa, >= 0)
 *   act_l0          sPAM cell length l_0 (m, > 0)
 *   obs_ptr[n+1]    obstacles of instance i are obs_ptr[i] .. obs_ptr[i+1]-1
 *   obs_kind        0 circle (obs_a = radius), 1 axis-aligned box (obs_a,
 *                   obs_b = half-width, half-height)
 *   obs_cx, obs_cy  centre (m)
 * Limits: n_links <= 1024, at most 1024 obstacles and 64 actuators per
 * instance.  Values outside their ranges mark the instance BADINPUT. */
typedef struct {
  int32_t n_inst;
  int32_t mem_is_device;
  const int32_t* n_links;
  const float* l_seg;
  const float* radius;
  const float* pressure;
  const float* base;
  const int32_t* act_ptr;
  const float* act_begin;
  const float* act_end;
  const int8_t* act_side;
  const float* act_pressure;
  const float* act_l0;
  const int32_t* obs_ptr;
  const uint8_t* obs_kind;
  const float* obs_cx;
  const float* obs_cy;
  const float* obs_a;
  const float* obs_b;
} vine_batch_desc;

typedef struct vine_batch vine_batch;

/* Per-batch counters (all instances), filled by vine_get_stats. */
typedef struct {
  int64_t robot_link_steps;  /* sum over converged steps of the links present */
  int64_t steps_converged;
  int64_t steps_total;
  int64_t iterations;        /* Gauss-Newton iterations */
  int64_t evaluations;       /* cost/gradient evaluations (incl. line search) */
  int64_t link_evaluations;  /* sum over evaluations of the links present */
  int64_t pair_tests;        /* all-pairs disc-obstacle count: sum over evaluations of N K_s n_obs */
  int64_t circle_pair_tests; /* the part of pair_tests against circles */
  int64_t gn_fallbacks;      /* Newton steps that used the Gauss-Newton matrix */
  int32_t n_maxiter, n_nonfinite, n_badinput, reserved;
  int64_t pair_tests_executed; /* disc-obstacle tests actually run (the broad phase skips the
                                  obstacles that cannot reach a link) */
} vine_stats;

/* Defaults listed above. */
vine_status vine_params_default(vine_params* out);

/* Copies the descriptor to the device, validates every instance, builds the
 * sPAM force tables (one per distinct l_0: FP64 solves of Eq. sPAM_1/sPAM_2
 * on 256 uniform strain knots) and the wrinkling-energy table, and leaves
 * every instance with zero links.  Synchronises `cuda_stream`. */
vine_status vine_batch_create(const vine_batch_desc* desc, const vine_params* params, void* cuda_stream,
                              vine_batch** out);

/* Back to zero links for every instance (statistics cleared).  Async. */
vine_status vine_batch_reset(vine_batch* b, void* cuda_stream);

/* Grows every instance by up to n_steps links (capped at its n_links), each
 * step solved to equilibrium, in one persistent launch per length class
 * (see vine_autotune).  An instance whose step does not converge stops
 * there (status VINE_INST_MAXITER).  Async. */
vine_status vine_grow_step(vine_batch* b, int32_t n_steps, void* cuda_stream);

/* Re-solves every instance's equilibrium at its present links without
 * adding one: the same solver as a growth step (or, in mode 1, the same
 * descent), from the present state and with the present actuators.  With
 * fix_length = 1 the distal length is held fixed, so the robot does not
 * grow while its actuation changes: the tip-steering of the paper's
 * supplement, where growth is stunted by penalising changes in length and
 * an actuator at the tip is pressurised.  fix_length = 0 leaves it free in
 * [0, l_seg].  Instances with no links or a status other than OK (a failed
 * step, non-finite or bad input; vine_batch_reset and vine_set_state
 * restore it) are skipped.  Counted in the statistics like a growth step.  (vine_grad
 * treats the distal length as free unless it sits at a bound.)  Async. */
vine_status vine_relax(vine_batch* b, int32_t fix_length, void* cuda_stream);

/* Grows every instance to its n_links: one persistent launch per length
 * class over its longest-first work queue (the classes on parallel
 * branches), replayed from a CUDA graph.  Async. */
vine_status vine_simulate(vine_batch* b, void* cuda_stream);

/* Launch autotuner.  A batch grows in length classes (robots of up to 64
 * links, 65-200, more: each class one persistent launch of its own team
 * size, the classes on parallel branches of the CUDA graph, the longest
 * robots' class first; with threads_per_robot set, one class).  The tuner
 * grows a sample of every class (`sample` robots in all, 0: 4096; at least
 * 64 per class; spread over each class's longest-first order) from reset
 * to full length per candidate and times each launch with CUDA events:
 *   - per class alone: threads per robot 32 (with 4, 2 or 1 robots per
 *     CTA), 64 or 128 (warps per robot);
 *   - all classes together with the chosen teams: the broad-phase margin
 *     0.5, 1 or 2 body radii (list length against rebuild frequency).
 * The result is adopted for later vine_grow_step / vine_simulate calls when
 * the sample grows faster than with the configuration chosen at creation
 * (timed first).  The margin never changes a result; the team size changes
 * results at rounding level (sums over other thread counts), each within
 * the parity bar.  Leaves the batch reset.  Synchronises the stream. */
typedef struct {
  int32_t warps_per_cta;   /* warps per CTA of the first (longest) class */
  float list_margin;       /* chosen, body radii */
  double best_ms;          /* sample growth time with the adopted configuration */
  double default_ms;       /* with the configuration chosen at creation */
  int32_t candidates;      /* configurations timed */
  int32_t sample;          /* instances grown per candidate */
  int32_t n_class;         /* length classes */
  int32_t adopted;         /* 1 if the tuned configuration replaced the default */
  int32_t class_threads[3];        /* threads per robot per class */
  int32_t class_robots_per_cta[3]; /* robots per CTA per class */
  double class_ms[3];      /* best sample time of each class alone */
} vine_tune_result;
vine_status vine_autotune(vine_batch* b, int32_t sample, void* cuda_stream, vine_tune_result* out);

/* Same result as vine_simulate, computed with one launch per instance in
 * sequence (the comparison form).  Async. */
vine_status vine_simulate_plain(vine_batch* b, void* cuda_stream);

/* Current state.  Any output pointer may be NULL.  Layouts:
 *   theta[sum n_links] (CSR by n_links; entries past the present links are 0)
 *   l_last[n], n_present[n], iterations[n] (summed over steps),
 *   residual[n] (largest final residual of any step, FP64),
 *   inst_status[n] (vine_inst_status),
 *   link_pose[3 * sum n_links]: start point x, y and heading of each link,
 *   tip[2n]: distal end point.
 * out_is_device = 1: outputs are device pointers (async);
 * 0: host pointers (the stream is synchronised). */
vine_status vine_get_state(const vine_batch* b, float* theta, float* l_last, float* link_pose, float* tip,
                           int32_t* n_present, int32_t* iterations, double* residual, int32_t* inst_status,
                           int32_t out_is_device, void* cuda_stream);

/* Contact set at the current state: pairs (link k, obstacle o) with o the
 * index within the instance's obstacles, such that some disc of link k
 * penetrates obstacle o.  counts[n] receives the number of pairs of each
 * instance (possibly more than max_pairs); pairs[n][max_pairs][2] receives
 * the first max_pairs of them in (link, obstacle) order.  Memory flag and
 * synchronisation as for vine_get_state. */
vine_status vine_get_contacts(const vine_batch* b, int32_t* counts, int32_t* pairs, int32_t max_pairs,
                              int32_t out_is_device, void* cuda_stream);

/* Replaces every actuator's pressure and span (arrays [sum n_act] in the
 * descriptor's actuator order; Pa and link units), keeping its side and cell
 * length.  Takes effect at the next launch that reads the design
 * (vine_grow_step, vine_simulate, vine_relax, vine_grad): the design update
 * of an optimisation loop without rebuilding the batch or its tables, or a
 * change of actuation in the middle of a growth (tip-steering).  Values that
 * fail the create-time checks (finite, 0 <= begin < end, pressure >= 0) mark
 * the instance VINE_INST_BADINPUT until the batch is recreated.
 * ptrs_are_device as for vine_grad (host pointers: the stream is
 * synchronised; device pointers: async). */
vine_status vine_set_actuators(vine_batch* b, const float* pressure, const float* begin, const float* end,
                               int32_t ptrs_are_device, void* cuda_stream);

/* Sets every instance's present state, so that the next vine_grow_step or
 * vine_simulate continues growth from it (Sec. 4.1: a growth step starts
 * from the previous step's joint angles; Algorithm 2 propagates tree nodes
 * from their stored states).  Arrays in the layouts vine_get_state returns:
 *   n_present[n]     links present, 0 <= n_present[i] <= n_links[i]
 *   theta[sum n_links] joint angles (rad), CSR by n_links; entries at or
 *                    past n_present are ignored (NULL allowed when every
 *                    instance has zero target links)
 *   l_last[n]        distal link length (m), 0 <= l_last <= l_seg (ignored
 *                    when n_present = 0)
 * Counters and statistics are cleared as by vine_batch_reset.  A state
 * outside these ranges (or non-finite) marks the instance
 * VINE_INST_BADINPUT with zero links until the next reset or
 * vine_set_state.  Continuing from a state read by vine_get_state gives
 * bitwise the same result as continuing in place.  ptrs_are_device as for
 * vine_grad (host pointers: the stream is synchronised). */
vine_status vine_set_state(vine_batch* b, const int32_t* n_present, const float* theta, const float* l_last,
                           int32_t ptrs_are_device, void* cuda_stream);

/* Adjoint of the equilibrium (implicit differentiation; the gradient a
 * design optimisation over the models of Sec. 3 needs).  For every instance,
 * at its current state taken as the equilibrium of its last growth step:
 *   cost[n] = |p_tip - goal|, goal_xy[2n] absolute goal points (m);
 *   d_pressure, d_begin, d_end [sum n_act] (CSR by act_ptr, the descriptor's
 *     actuator order): d cost / d P_a (per Pa), d cost / d b_a and
 *     d cost / d e_a (per link unit; right derivatives at integer ends);
 *   grad_status[n]: 0 ok; 1 the exact Hessian of the cost of Eq. (pbd) is
 *     not positive definite at the state (derivatives NaN); 2 the instance
 *     has no valid state (bad input or non-finite; cost and derivatives NaN).
 * lambda = H^-1 d cost / d x (x = joint angles and the distal length, the
 * distal length dropped when its bound is active, as in the solver), then
 * d cost / d q = -lambda . d(grad J)/dq: grad J depends on an actuator's
 * pressure and span only through its moment c_aj s_a P_a f_a(eps_aj) d
 * (Eq. restoring_moment).  An instance with no links has cost |base - goal|
 * and zero derivatives.
 * ptrs_are_device = 1: every pointer is a device pointer (async on
 * cuda_stream); 0: host pointers (staged through a library-owned device
 * buffer; the stream is synchronised).  The batch state is not changed. */
vine_status vine_grad(const vine_batch* b, const float* goal_xy, double* cost, double* d_pressure, double* d_begin,
                      double* d_end, int32_t* grad_status, int32_t ptrs_are_device, void* cuda_stream);

/* Adjoint of a path cost (the benchmark spec (3); the path the planner of Sec. 5
 * grows along, as target points of the link ends):
 *   cost[n] = (1/N) sum_{k=1..N} |p_k - q_k|^2, p_k the end point of link
 *     k-1 (p_N the tip) at the current state, q_k = path_xy[2 (o_i + k - 1)
 *     .. + 1] the targets (m, absolute), o_i the robot's offset in the
 *     joint-angle layout (sum of the earlier robots' n_links), so path_xy
 *     holds 2 sum n_links floats; a robot with N < n_links links uses its
 *     first N targets;
 *   derivatives and grad_status as vine_grad.
 * d cost / d theta_j = (2/N) sum_{k > j} (p_k - q_k) . (z x (p_k - p_j)),
 * d cost / d l_last = (2/N) (p_N - q_N) . u_{N-1}; the adjoint as
 * vine_grad.  An instance with no links has cost 0.  ptrs_are_device as
 * vine_grad. */
vine_status vine_grad_path(const vine_batch* b, const float* path_xy, double* cost, double* d_pressure,
                           double* d_begin, double* d_end, int32_t* grad_status, int32_t ptrs_are_device,
                           void* cuda_stream);

/* Batch counters (host struct; synchronises the stream). */
vine_status vine_get_stats(const vine_batch* b, vine_stats* out, void* cuda_stream);

/* The prologue tables as used by the kernels (synchronous):
 *   n_tab: number of sPAM force tables (one per distinct actuator l_0, in
 *     order of first appearance among the actuators);
 *   hdr[4 n_tab]: eps_lo, knot spacing h, 1/h, G(0) per table;
 *   knots[2 * 256 n_tab]: (f_k, G_k): force per unit actuation pressure
 *     (Eq. sPAM_force / P_act, m^2) at strain eps_lo + k h, and its integral
 *     from eps_lo;
 *   utab[2 * 1025]: (Uhat, mhat) of the wrinkling moment (Eq. wrinkling_model,
 *     per unit pi P R^3) and its integral from 0, at theta_c + k h_u;
 *   consts[4]: Uhat(pi), mhat(pi), theta_c, h_u.
 * Any output pointer may be NULL. */
vine_status vine_get_tables(const vine_batch* b, int32_t* n_tab, float* hdr, float* knots, float* utab,
                            double* consts);

/* Introspection of one robot at a caller-given state (synchronous; host
 * buffers; allocates a small device buffer): with n_links links present,
 * joint angles theta[n_links] and distal length l_last, returns the cost of
 * Eq. (pbd) in potential form (FP64 sum of FP32 terms), its gradient
 * grad[n_links + 1] (the last entry is d/d l_last), the Gauss-Newton step
 * step[n_links + 1] the solver would take there (the last entry is 0 when
 * the bound on l_last is active, reported in *l_fixed), and that step's
 * predicted-displacement residual.  Does not change the batch state. */
vine_status vine_probe_state(const vine_batch* b, int32_t inst, int32_t n_links, const float* theta, float l_last,
                             double* cost, float* grad, float* step, double* residual, int32_t* l_fixed);

/* Per-robot counters since the last reset (host arrays of n; any may be
 * NULL; synchronises the stream): converged growth steps, cost
 * evaluations, and SM clock cycles its warp spent on it. */
vine_status vine_get_robot_counters(const vine_batch* b, int32_t* steps_converged, int64_t* evaluations,
                                    int64_t* cycles, void* cuda_stream);

/* Number of instances and total link capacity (sum of n_links). */
vine_status vine_batch_info(const vine_batch* b, int32_t* n_inst, int64_t* total_links);

/* The growth launch of the first (longest robots') length class, chosen at
 * creation or by vine_autotune: threads per robot, robots per CTA and CTAs.
 * Any output may be NULL. */
vine_status vine_batch_launch(const vine_batch* b, int32_t* threads_per_robot, int32_t* robots_per_cta,
                              int32_t* grid);

/* The length classes of the batch's growth launch (see vine_autotune), the
 * longest robots' first: *n_class (1..3) and per class (arrays of 3, any
 * may be NULL) threads per robot, robots, robots per CTA, CTAs and the
 * longest robot's links. */
vine_status vine_batch_classes(const vine_batch* b, int32_t* n_class, int32_t* threads_per_robot, int32_t* robots,
                               int32_t* robots_per_cta, int32_t* grid, int32_t* max_links);

/* Releases the batch (device memory freed after synchronising the device). */
vine_status vine_batch_destroy(vine_batch* b);

/* ---------------------------------------------------------------------------
 * Allocation-free table build.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- for example a
 * process whose device memory is entirely handed to another framework's
 * pool, or a latency-critical loop in which the device synchronisation that
 * cudaMalloc/cudaFree imply is not acceptable.
 *
 * Builds the sPAM force-per-pressure tables (the same kernels and results as
 * the tables vine_batch_create builds and vine_get_tables returns) for n_tab
 * cell lengths l0[n_tab] (device, metres), writing hdr[4 n_tab] (device,
 * 16-byte aligned) and knots[2 * 256 n_tab] (device, 8-byte aligned) in the
 * vine_get_tables layout.  Only R_c, R_act, a_spam and m_lo of *params are
 * used.  Asynchronous on cuda_stream.
 *
 * The FP64 working space is a file-scope device array sized for
 * VINE_NOALLOC_MAX_TABLES tables (133 KB), held by every GPU that loads the
 * library until the process exits.  n_tab beyond that maximum is rejected
 * with VINE_EINVAL and nothing is launched.  The call allocates no memory
 * (no cudaMalloc, cudaFree or allocating library routine).  Its first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call shares the one array: calls whose work overlaps on the GPU
 * (other streams, or other host threads on the same device) race on it and
 * must be serialised by the caller.  No entry of the array needs to start at
 * zero: each entry a call reads is written earlier by that call. */
#define VINE_NOALLOC_MAX_TABLES 64
vine_status vine_spam_tables_noalloc(const double* l0, int32_t n_tab, const vine_params* params, float* hdr,
                                     float* knots, void* cuda_stream);

/* Actuator design synthesis (Sec. 4.2): for every target angle per joint
 * theta_target[q] (rad), the sPAM design -- a pressure from the caller's
 * discrete set and a cell length on the caller's grid -- whose actuator holds
 * a free joint of the body (no contact) at theta_target within tol.
 *   A design (P, l0) holds the joint at theta_eq(P, l0) in (0, pi], where the
 *   wrinkling moment (Eq. wrinkling_model) equals the actuator moment
 *   (Eq. sPAM_force per pressure times P times the arm 2 R + R_act of
 *   Sec. 3.3) at the actuator strain (2 R + R_act) theta / l_seg, the force
 *   per pressure from the cell length's sPAM table (the growth step's table,
 *   built here in FP64); pi when the actuator still wins at pi.
 *   Among the designs with |theta_eq - theta_target| <= tol: the highest
 *   pressure (the paper's rule), then the closest angle, then the shorter
 *   cell, then the lower pressure index.  None: indices -1, theta_eq NaN.
 * A per-joint target times the number of covered joints is the segment's
 * turning angle.  spec: body radius R (m), body pressure P_vine (Pa),
 * segment length l_seg (m), pressures[n_p] (Pa, > 0), cell lengths
 * l0_min + k l0_step (m), k < n_l0, tol (rad, >= 0); n_p, n_l0 in [1, 4096],
 * n_p n_l0 <= 2^20.  params: sPAM constants and eps_crit (NULL: defaults).
 * Outputs (host): p_index[n_targets], l0_index[n_targets],
 * theta_eq[n_targets], and theta_pairs[n_p][n_l0] (may be NULL).  Host
 * pointers; the stream is synchronised.  The FP64 sPAM tables of a grid of
 * cell lengths (with its sPAM constants) are kept for later calls on the
 * same device, up to 8 grids per process; a later call copies them instead
 * of building them again (bitwise the same tables). */
typedef struct {
  double R, P_vine, l_seg;
  const double* pressures;
  int32_t n_p;
  double l0_min, l0_step;
  int32_t n_l0;
  double tol;
} vine_synth_spec;
vine_status vine_synthesize(const vine_synth_spec* spec, const vine_params* params, const double* theta_target,
                            int32_t n_targets, int32_t* p_index, int32_t* l0_index, double* theta_eq,
                            double* theta_pairs, void* cuda_stream);

/* sPAM neural surrogate (Sec. 4.3).  The paper replaces the numerical
 * solution of Eq. sPAM_1/sPAM_2 inside its simulator by a 2-32-2 network
 * (ReLU hidden units, He initialisation) from (strain, cell length) to
 * (m, phi_Rc), trained on 40k samples of the exact model by mean squared
 * error on normalised outputs.
 *
 * vine_spam_samples: the exact model at given (m[i] in (0, 0.5], l0[i] > 0)
 * -- strain eps (Eq. sPAM_1), phi_Rc (the smallest root of Eq. sPAM_2 in
 * (0, acos(R_c / R_act)], else that bound: the saturated branch), force per
 * pressure f (Eq. sPAM_force), saturated flag -- in FP64, one warp per
 * sample.  params: sPAM constants (NULL: defaults).  Host pointers; the
 * stream is synchronised.
 *
 * vine_surrogate: the network's 162 parameters, W1[32][2] (hidden, input),
 * b1[32], W2[2][32] (output, hidden), b2[2], and its normalisation:
 * x_i = (input_i - in_lo_i) in_scale_i, output_k = y_k / out_scale_k.
 *
 * vine_surrogate_train: full-batch Adam (beta 0.9 / 0.999, eps 1e-8) for
 * `steps` steps of learning rate lr on the loss (1 / 2n) sum |y - t|^2,
 * t the normalised targets (m, phi) times out_scale; inputs[n][2] =
 * (strain, cell length), targets[n][2] = (m, phi).  net holds the initial
 * parameters on entry and the trained ones on return; loss_history[steps]
 * (may be NULL) the loss before each step.  The gradient sums run in a
 * fixed order: the result does not depend on scheduling.  Host pointers;
 * the stream is synchronised.
 *
 * vine_surrogate_eval: outputs[n][2] = (m, phi) of the network at
 * inputs[n][2]; ptrs_are_device as for vine_grad (net itself is a host
 * struct). */
typedef struct {
  float theta[162];
  float in_lo[2], in_scale[2], out_scale[2];
} vine_surrogate;
vine_status vine_spam_samples(const double* m, const double* l0, int32_t n, const vine_params* params, double* eps,
                              double* phi, double* f, int32_t* saturated, void* cuda_stream);
vine_status vine_surrogate_train(vine_surrogate* net, const double* inputs, const double* targets, int32_t n,
                                 int32_t steps, float lr, float* loss_history, void* cuda_stream);
vine_status vine_surrogate_eval(const vine_surrogate* net, const double* inputs, int32_t n, double* outputs,
                                int32_t ptrs_are_device, void* cuda_stream);

/* Tree operations of the batched SST* planner (Sec. 5.2, Algorithm 2).
 * Tip poses are (x, y, phi) triples, float32 [3 n], headings in [-pi, pi],
 * positions in any length unit; rho converts radians to that unit, so that
 *   d^2 = dx^2 + dy^2 + (rho * dphi)^2,  dphi wrapped to [-pi, pi],
 * evaluated in float32 with every product and sum rounded on its own (no
 * fused multiply-add).  Two states overlap when d < r (strictly).  Costs
 * are float64 and should be finite.  States are ordered by the key
 * (cost, id): ties go to the lower id, tree nodes (ids 0 .. n_old-1)
 * before new states (ids n_old ..).
 * ptrs_are_device = 1: every array is a device pointer (async on the
 * stream); 0: host pointers (the stream is synchronised).  Device scratch
 * is taken from the stream-ordered allocator for the call.  Counts up to
 * 2^31 - 1 in total. */

/* Pruning of overlapping states (Algorithm 2, prune).  new_keep[j] = 1
 * exactly when no overlapping state -- an active tree node or another new
 * state of finite cost -- has a smaller key (a new state of non-finite cost
 * is never kept); old_deactivate[i] = 1 exactly when tree node i is active
 * and a kept new state of smaller key overlaps it.  radius, rho >= 0. */
vine_status vine_sst_prune(int32_t n_old, const float* old_pose, const double* old_cost, const uint8_t* old_active,
                           int32_t n_new, const float* new_pose, const double* new_cost, float radius, float rho,
                           uint8_t* new_keep, uint8_t* old_deactivate, int32_t ptrs_are_device, void* cuda_stream);

/* Best-near selection of the nodes to expand (Algorithm 2, sample: lowest
 * cost first).  For every sample pose: among the active nodes within delta
 * of it, the one of smallest key; if none is within delta, the nearest
 * active node (ties to the lower index); -1 when no node is active.
 * delta, rho >= 0. */
vine_status vine_sst_select(int32_t n_nodes, const float* pose, const double* cost, const uint8_t* active,
                            int32_t n_samples, const float* sample_pose, float delta, float rho, int32_t* chosen,
                            int32_t ptrs_are_device, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving loop: continuous batching of growth requests on one GPU.  The
 * paper's planners (Sec. 5) issue many small simulation requests; a server
 * keeps every admitted robot's state on the device between growth launches
 * and mixes robots of different requests in each launch.
 *
 * A server owns a fixed arena of robot slots (design, obstacles, joint
 * angles and counters of one robot each, capacities below), the sPAM force
 * tables of every cell length seen so far and the wrinkling-energy table, and
 * one worker thread that owns its CUDA streams.  The worker admits waiting
 * requests into free slots (copy in, validate, encode, build missing tables)
 * and assigns each to one of `lanes` launch lanes.  Each lane repeatedly
 * launches the persistent growth kernel over up to `window` robots of its
 * requests, oldest requests first, for up to steps_per_tick links each, on
 * its own stream; lanes overlap on the GPU, so one lane's launch finishing
 * its slowest robots leaves the SMs to the other.  After each launch the
 * lane reads back links present and status, and retires the requests whose
 * robots are all done (reached n_links, or stopped non-finite / bad input).
 * A robot's result does not depend on the requests it shared launches with.
 * ------------------------------------------------------------------------- */
typedef struct vine_server vine_server;

typedef struct {
  size_t device_mem_budget; /* bytes the server may hold on the device (0: 1 GiB) */
  int32_t max_slots;        /* robot slots (0: as many as the budget holds) */
  int32_t max_links;        /* per slot: links (0: 320) */
  int32_t max_obs;          /* per slot: obstacles (0: 256) */
  int32_t max_act;          /* per slot: actuators (0: 16) */
  int32_t max_request;      /* robots per request (0: 256) */
  int32_t steps_per_tick;   /* growth steps per robot per launch (0: max_links, i.e. to completion) */
  int32_t max_tables;       /* distinct sPAM cell lengths live at one time (0: 256): a table entry is
                               held while an admitted request uses its cell length and reused after */
  int32_t lanes;            /* concurrent launch lanes, 1..8 (0: 4) */
  int32_t window;           /* robots per launch and lane (0: twice the resident warps) */
} vine_server_config;

typedef struct {
  int32_t n_inst;             /* robots of the request */
  int32_t reserved;
  int64_t total_links;        /* sum of n_links */
  int64_t robot_link_steps;   /* links present summed over converged steps */
  double t_submit, t_admit, t_done; /* vine_serve_clock seconds */
} vine_request_info;

typedef struct {
  int64_t ticks;              /* growth launches */
  int64_t requests_done;
  int64_t robot_link_steps;   /* of retired requests */
  int32_t active_robots, waiting_requests;
  int32_t free_slots, max_slots;
  double busy_s;              /* wall time of ticks with active robots */
} vine_server_stats;

/* The defaults listed above (a zero field in a config passed to
 * vine_server_create also selects its default). */
vine_status vine_server_config_default(vine_server_config* out);

/* Allocates the slot arena and tables (one cudaMalloc within the budget),
 * builds the wrinkling table and starts the worker on the current device.
 * VINE_EINVAL when the budget cannot hold one slot per robot of a maximal
 * request or the slot does not fit in shared memory. */
vine_status vine_server_create(const vine_params* params, const vine_server_config* config, vine_server** out);

/* Copies a request (host memory: desc->mem_is_device must be 0) and queues
 * it; *request_id identifies it.  VINE_EBUSY when the free slots (less those
 * promised to requests still waiting) cannot hold its robots: nothing is
 * kept and the client retries later; VINE_EBUSY too when its cell lengths,
 * with those held by admitted requests and those of waiting requests, are
 * more than max_tables (entries free up as requests finish).  VINE_EINVAL
 * for a malformed request, more robots than max_request, a robot beyond the
 * slot capacities, or more distinct cell lengths in the request itself than
 * max_tables.  Thread-safe. */
vine_status vine_serve_submit(vine_server* s, const vine_batch_desc* desc, uint64_t* request_id);

/* Waits up to timeout_us (0: do not wait) for request_id to finish.  Done:
 * fills *info (may be NULL) and the host outputs (any may be NULL), in the
 * layouts of vine_get_state -- theta[sum n_links], l_last[n], tip[2n],
 * n_present[n], inst_status[n], iterations[n] -- and releases the request
 * (its id is then unknown).  Not done: VINE_ETIMEOUT (info filled with the
 * request's size and submit time).  Unknown id: VINE_EINVAL.  A worker
 * failure: VINE_ECUDA.  Thread-safe. */
vine_status vine_serve_poll(vine_server* s, uint64_t request_id, int32_t timeout_us, vine_request_info* info,
                            float* theta, float* l_last, float* tip, int32_t* n_present, int32_t* inst_status,
                            int32_t* iterations);

/* Counters of the server (host struct). */
vine_status vine_server_get_stats(vine_server* s, vine_server_stats* out);

/* The clock of t_submit / t_admit / t_done (seconds, monotonic). */
vine_status vine_serve_clock(double* seconds);

/* Stops the worker after its current tick, drops unfinished and unpolled
 * requests and frees the server. */
vine_status vine_server_destroy(vine_server* s);

/* Message of the last failed call on this thread ("" if none). */
const char* vine_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VINE_H_ */
