/*
 * mppi.h -- C ABI of libmppi: GPU (sm_103a) sampling-based optimisation of
 * bimanual ball manipulation with a parallel rigid-body contact simulator.
 *
 * The optimiser is the MPPI loop of the paper's Algorithm 1 (sample control
 * sequences from N(nu, Sigma), roll each out through the world model, sum the
 * stage costs, weight the samples with s_j = exp(-c_j / beta) and move the
 * mean to the weighted average, Eq. 8a and 8d) with the learning rate
 * eta = 1, the elite set equal to all K samples, beta = lambda and a fixed
 * diagonal Sigma = diag(sigma^2).  The world model is a MuJoCo-style
 * simulator of two revolute arms with capsule links, a free ball, static
 * boxes and a floor (Sec. III, Eq. 1b; joint-space dynamics, soft frictional
 * contact by projected Gauss-Seidel, semi-implicit Euler).
 *
 * Conventions
 *  - Every tensor argument is a caller-owned DEVICE pointer to float32 in
 *    row-major order (last index fastest) unless stated otherwise.  The
 *    library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work and return without synchronising, except
 *    where stated.
 *  - Return codes are the MPPI_* values below; no exception crosses the ABI.
 *    Errors detected on the device (non-finite costs, a failed Cholesky
 *    pivot, a bounded wait that ran out) are recorded in the handle's error
 *    word and returned by mppi_sync() / mppi_batch_sync().
 *  - One handle per stream; a handle is not thread-safe.
 *  - Dimensions for a model with n_a joints per arm: nq = 2 n_a + 7
 *    (left arm, right arm, ball position, ball quaternion w-first),
 *    nv = 2 n_a + 6 (arm joint rates, ball linear and angular velocity in
 *    world axes), nu = 2 n_a (one control per arm joint), state
 *    x = (q, qdot) of nx = nq + nv floats.  Supported n_a: 3 and 7.
 */
#ifndef MPPI_H
#define MPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MPPI_OK = 0,
    MPPI_ERR_INVALID_ARG = 1, /* bad pointer, size or blob                   */
    MPPI_ERR_OOM = 2,         /* device or host allocation failed            */
    MPPI_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed        */
    MPPI_ERR_NONFINITE = 4,   /* every sample cost was NaN/inf, or a state
                                 went non-finite; u_nom was left unchanged   */
    MPPI_ERR_TIMEOUT = 5,     /* a bounded device wait gave up               */
    MPPI_ERR_ADMISSION = 6,   /* server: request does not fit the budget     */
    MPPI_ERR_CHOLESKY = 7,    /* (M + dt D) lost positive definiteness       */
    MPPI_ERR_UNSUPPORTED = 8  /* model outside the compiled variants         */
};

typedef struct mppi_model mppi_model;
typedef struct mppi_ctx mppi_ctx;

/* Human-readable name of a return code (static string). */
const char *mppi_strerror(int code);

/* ---------------------------------------------------------------- model */
/* The world model f of Eq. 1b (Sec. III): the simulator that maps a state
 * and one control to the next state.  Parse a scene blob (host memory,
 * `len` bytes; layout: u32 magic 0x4950504D, u32 version 1, u32 count,
 * u32 0, then `count` float64 values
 * -- kinematics, inertias, capsule geometry, contact constants, boxes, cost
 * weights, home state) and upload it to the current device.  The blob is
 * copied; the caller keeps ownership of it.  *out receives an immutable
 * model that may be shared by many handles. */
int mppi_model_load(const void *blob, size_t len, mppi_model **out);
void mppi_model_free(mppi_model *m);
/* Dimensions of a loaded model (any output pointer may be NULL). */
int mppi_model_dims(const mppi_model *m, int *nq, int *nv, int *nu, int *n_boxes);
/* Home state x0 of the scene into host memory (nx floats). */
int mppi_model_home(const mppi_model *m, float *x0_host);

/* ------------------------------------------------------------- controller */
/* One MPPI controller (paper Alg. 1, Eq. 8).  K samples per iteration,
 * horizon H steps, temperature lambda > 0, sigma = nu per-control standard
 * deviations (HOST pointer, copied), 64-bit Philox key `seed`.  Allocates
 * the handle's device workspace (K costs, error word, iteration counter).
 * 1 <= K <= 1<<20, 1 <= H <= 1024. */
int mppi_create(const mppi_model *m, int K, int H, float lambda, const float *sigma, uint64_t seed,
                mppi_ctx **out);
int mppi_destroy(mppi_ctx *c);

/* One optimisation iteration (Alg. 1 loop body without the QP projection):
 *   eps[k,h,j] = sigma_j N(0,1) from Philox4x32-10, key = seed, counter =
 *                (j/4, h, k, iteration), Box-Muller on the word pairs;
 *   U_k = clamp(u_nom + eps_k, u_lo, u_hi) per control;
 *   c_k = sum_h stage cost along the rollout of U_k from `state`;
 *   w_k = exp(-(c_k - min c)/lambda) (non-finite c_k -> 0);
 *   u_nom_out = sum_k w_k U_k / sum_k w_k        (Eq. 8a, 8d).
 * state: nx floats; u_nom, u_nom_out: H x nu, may alias.  Advances the
 * handle's iteration counter (on the device) by one. */
int mppi_step(mppi_ctx *c, const float *state, const float *u_nom, float *u_nom_out, void *stream);

/* The same iteration with HOST buffers (state: nx floats, u_nom and
 * u_nom_out: H x nu floats, may alias): one copy of (state, u_nom) to the
 * device through a pinned staging buffer the handle owns (allocated on the
 * first call), the iteration, one copy of u_nom' back; returns after the
 * stream has synchronised.  Not capturable. */
int mppi_step_host(mppi_ctx *c, const float *state, const float *u_nom, float *u_nom_out, void *stream);

/* `iters` iterations of mppi_step in place on u_nom_inout (Alg. 1, M =
 * iters).  best_cost_out (optional, 2 floats): lowest sample cost of the
 * last iteration and its sample index (as float).  After the first call
 * with a given (state, u_nom_inout, iters, stream), the iterations are
 * replayed from a captured CUDA graph. */
int mppi_solve(mppi_ctx *c, const float *state, float *u_nom_inout, int iters, float *best_cost_out,
               void *stream);

/* Weighted-mean update alone (Eq. 8a, 8d) for host- or test-supplied
 * costs: costs (K), u_nom, u_out (H x nu, may alias).  The samples are the
 * Philox samples of the handle's current iteration counter.  Does not
 * advance the counter. */
int mppi_update(mppi_ctx *c, const float *costs, const float *u_nom, float *u_out, void *stream);

/* The world model f of Eq. 1b (Sec. III) applied H times per sequence, with
 * the stage costs summed as in Alg. 1's rollout and cost step.
 * Roll out n explicit control sequences: states (n x nx), U (n x H x nu),
 * costs (n) -- the same simulator and stage costs as mppi_step with the
 * controls given instead of sampled.  states_out (optional, n x nx): the
 * state after the last step.  n <= K of the handle. */
int rollout_batch(mppi_ctx *c, int n, const float *states, const float *U, float *costs,
                  float *states_out, void *stream);

/* One application of the world model f of Eq. 1b (Sec. III): x' = f(x, u).
 * One simulator step for n states in place: states_inout (n x nx), U1
 * (n x nu).  n <= K. */
int sim_step(mppi_ctx *c, int n, float *states_inout, const float *U1, void *stream);

/* Alg. 1's sampling step (control perturbations drawn from N(0, Sigma)).
 * Materialise the Philox noise of iteration `iteration`: eps_out
 * (K x H x nu).  For tests. */
int mppi_debug_noise(mppi_ctx *c, uint64_t iteration, float *eps_out, void *stream);

/* Raw Philox4x32-10 words for n counters (tests of the integer stream):
 * ctr (device, n x 4 uint32), key = the 64-bit key, out (device, n x 4). */
int mppi_debug_philox(int n, const uint32_t *ctr, uint64_t key, uint32_t *out, void *stream);

/* Bounds check.  In a library compiled with -DMPPI_BOUNDS_CHECK every index
 * the rollout, update, elite-set and QP kernels use into shared memory, the
 * staged model and the device buffers is compared with its extent; a failed
 * check sets a bit in a device word (1: shared/workspace index, 2: device
 * buffer index) and the access is diverted, with no trap.  This call
 * synchronises the device, returns the word of every translation unit ORed
 * (and clears it) and sets *checked to 1 in such a build, 0 (word 0)
 * otherwise.  Either pointer may be NULL.  A stand-in for a memory checker
 * on small cases. */
int mppi_debug_bounds(unsigned *word, int *checked);

/* Iteration counter (checkpoint / resume).  get synchronises `stream`. */
int mppi_get_iteration(mppi_ctx *c, uint64_t *iteration, void *stream);
int mppi_set_iteration(mppi_ctx *c, uint64_t iteration, void *stream);

/* Synchronise `stream`, then return and clear the handle's device error
 * word: MPPI_OK, MPPI_ERR_NONFINITE, MPPI_ERR_CHOLESKY or MPPI_ERR_TIMEOUT. */
int mppi_sync(mppi_ctx *c, void *stream);

/* Profiling.  mppi_profile(c, n) records CUDA events around the rollout
 * and update kernels of the next n iterations (mppi_step / mppi_solve
 * eager path) on the launching stream and counts, on the device, the active
 * contacts and the capsule-box pairs that pass the separating-axis cull;
 * n = 0 turns it off.  mppi_profile_read synchronises the recorded events
 * and returns: iterations recorded, total rollout and update kernel time
 * (ms), mean active contacts per sample-step and mean exact capsule-box
 * tests per sample-step.  Any output pointer may be NULL. */
int mppi_profile(mppi_ctx *c, int n);
int mppi_profile_read(mppi_ctx *c, int *n, float *rollout_ms, float *update_ms, double *contacts_per_step,
                      double *box_tests_per_step);
/* Of the recorded sample-steps, the fraction whose only contact is the
 * ball against static geometry (floor or box): the Delassus block of such a
 * contact is diagonal (its point lies on the normal through the ball's
 * centre), so projected Gauss-Seidel is at its fixed point after one sweep
 * and the rollout solves it directly.  Counted on the device with the
 * statistics of mppi_profile; synchronous.  Errors: MPPI_ERR_INVALID_ARG for
 * a NULL handle or output. */
int mppi_profile_lone_contacts(mppi_ctx *c, double *lone_per_step);
/* Total time (ms) of the QP projection launches over the recorded
 * iterations (0 when the projection is off); synchronises the events. */
int mppi_profile_projection(mppi_ctx *c, float *qp_ms);

/* The paper's full update (Eq. 8a-8d): the elite set is the n_elite
 * samples of lowest cost (ties -> lower index; non-finite costs never
 * elite), s_j = exp(-(c_j - c_min)/lambda) over the elite set,
 *   nu'      = (1 - eta) nu + eta sum_j s_j U_j / sum_j s_j,
 * and with update_cov = 1
 *   Sigma'_h = (1 - eta) Sigma_h + eta sum_j s_j (U_j[h] - nu'_h)(...)^T /
 *              sum_j s_j + cov_floor I
 * for one nu x nu block per horizon step h (a reading: the paper does not
 * fix the covariance structure); later iterations then sample
 * U = clamp(nu + L_h z) with L_h the block's Cholesky factor.  Defaults:
 * n_elite = K, eta = 1, update_cov = 0 (the plain update).  n_elite < K
 * needs K <= 8192; update_cov needs the controller's sample buffer
 * (K H nu floats <= 256 MB). */
int mppi_set_update(mppi_ctx *c, int n_elite, float eta, int update_cov, float cov_floor);
/* Covariance blocks Sigma_h (device, H x nu x nu).  set: each block must be
 * positive definite (factored on the host); sampling then uses them. */
int mppi_get_covariance(mppi_ctx *c, float *Sigma, void *stream);
int mppi_set_covariance(mppi_ctx *c, const float *Sigma, void *stream);
/* Controls of the lowest-cost sample of the last elite update (device,
 * H x nu): the optimiser's output besides nu and Sigma (Alg. 1). */
int mppi_best_controls(mppi_ctx *c, float *U_best, void *stream);

/* ------------------------------------------------ QP smoothing projection */
/* Eq. 5a-5b (Alg. 1, the step between sampling and rollout): a joint's H
 * commanded velocities vt are replaced by
 *   v = argmin 1/2 |v - vt|^2  subject to, for r = 0..3 (Sec. III),
 *   position      b0 <= q + dt sum_{i<=t} v_i              <= b1, t = 0..H-1
 *   velocity      b2 <= v_t                                <= b3, t = 0..H-1
 *   acceleration  b4 <= (v_t - v_{t-1}) / dt               <= b5, t = 0..H-1
 *   jerk          b6 <= (v_t - 2 v_{t-1} + v_{t-2}) / dt^2 <= b7, t = 1..H-1
 * with q, qd the joint's present position and velocity (v_{-1} = qd).  A
 * group whose two bounds are -inf and +inf is left out.  The paper names no
 * solver: this library runs `iters` iterations of ADMM (scaled form, penalty
 * rho, row groups scaled by `scales` = position/dt, velocity, acceleration*dt
 * and jerk*dt^2 weights) from v = vt, so a feasible vt is returned
 * unchanged (up to FP32 rounding), and returns the last iterate: after 30
 * iterations white-noise samples that broke the jerk bound 40-fold keep
 * every derivative within about 5% of its bound, after 100 within 0.3%.  An
 * infeasible problem (a present state the bounds cannot hold) returns a
 * compromise.  Every sequence runs the same iteration count. */
#define MPPI_QP_MAX_H 256
#define MPPI_QP_SCALE_POSITION 0.1f
#define MPPI_QP_SCALE_VELOCITY 1.0f
#define MPPI_QP_SCALE_ACCELERATION 2.0f
#define MPPI_QP_SCALE_JERK 4.0f
/* Projection of n independent sequences sharing one set of bounds.
 *   bounds   HOST, 8 floats (lo, hi) x (position, velocity, acceleration,
 *            jerk); lo <= hi, no NaN
 *   scales   HOST, 4 floats > 0, or NULL for the MPPI_QP_SCALE_* defaults
 *   q0, qd0  device, n floats: each sequence's present position, velocity
 *   v_in     device, n x H; v_out device, n x H (may alias v_in)
 * 1 <= H <= MPPI_QP_MAX_H, iters >= 0, rho > 0, dt > 0.  Allocates a small
 * stream-ordered scratch block (cudaMallocAsync) per call. */
int mppi_qp_project(int n, int H, float dt, const float *bounds, int iters, float rho, const float *scales,
                    const float *q0, const float *qd0, const float *v_in, float *v_out, void *stream);
/* Turn the projection on inside the controller's iteration (iters > 0) or
 * off (iters = 0).  bounds: HOST, nu x 8 floats, one row per joint as
 * above; q, qd come from the state passed to each step.  While on, the
 * samples are drawn unclamped (nu + sigma z, or nu + L_h z), projected, and
 * the projected sequences are what the rollout simulates and the update
 * averages (Eq. 8 uses the projected samples).  Needs the controller's
 * sample buffer (K H nu floats <= 256 MB) and H <= MPPI_QP_MAX_H. */
int mppi_set_projection(mppi_ctx *c, const float *bounds, int iters, float rho, const float *scales);
/* The samples of the last iteration as the rollout used them (device,
 * H x K x nu, h-major): projected when the projection is on, else the
 * clamped samples.  Needs the sample buffer. */
int mppi_get_samples(mppi_ctx *c, float *U, void *stream);

/* --------------------------------------------------- ball-task cost suite */
/* The paper's cost for lifting and transporting the ball (Sec. IV-B), in
 * place of the scene's stage cost for every rollout of the handle
 * (mppi_step, mppi_solve, rollout_batch):
 *   C = w_pick (w_c C_c + w_eo C_eef-obj) + w_move (w_c C_c + w_ot C_obj-targ)
 *       + w_theta C_theta + w_yz C_yz + w_v C_v + w_r C_r + w_l C_l,
 * w_pick = 1, w_move = 0 in the pick phase and the reverse in the move
 * phase.  With x_0 the present state and x_1..x_H the states the controls
 * produce, p_i the distal end of arm i's last capsule, q_i its last link
 * frame as a quaternion and c = (p_1 + p_2)/2:
 *   C_c       = sum over the H transitions and every pair b of
 *               max(-d_{k+1,b} + (1 - gamma) d_{k,b}, 0)  +  the number of
 *               (state k >= 1, pair) with d_{k,b} < 0; pairs: every link x
 *               every box, every link x the ball (pick phase only), every
 *               left link x every right link (signed distances)
 *   C_theta   = sum_k |theta_k - theta_home|
 *   C_yz      = sum_k |(p_1 - p_2) in y and z|
 *   C_v       = sqrt(sum_k ((p_1 - p_2) . (pdot_1 - pdot_2))^2)
 *   C_r       = sum_k (acos|<q_1, q_1*>| + acos|<q_2, q_2*>|)
 *   C_l       = sum_k (|p_1 - p_2| - l_ball)^2
 *   C_eef-obj = sum_k |c - (p_ball0 - (0, 0, eps))|
 *   C_obj-targ= sum_k |c + (0, 0, eps) - p_target|
 * params (HOST, MPPI_TASK_N + nu floats): [0] phase (0 pick, 1 move),
 * [1] w_c, [2] gamma in [0, 1), [3] w_theta, [4] w_yz, [5] w_v, [6] w_r,
 * [7] w_l, [8] l_ball, [9] w_eo, [10] w_ot, [11] eps, [12..14] p_ball0,
 * [15..17] p_target, [18..21] q_1*, [22..25] q_2* (unit, w first),
 * [26..26+nu) theta_home.  params = NULL turns the suite off. */
#define MPPI_TASK_N 26
int mppi_set_task_cost(mppi_ctx *c, const float *params, int n);

/* ------------------------------------------------ closed-loop episodes */
/* Receding-horizon control as the paper runs it (Sec. III-A, Alg. 1 and
 * the text after Eq. 8; metrics of Sec. IV-A): the simulator itself stands
 * in for the robot ("world").  Each planning step
 *   1. runs cfg->iters optimiser iterations (mppi_solve) from the world
 *      state on the warm-started nominal sequence;
 *   2. takes the lowest-cost sequence of the last iteration (the elite
 *      update's best sequence, or the lowest-cost sample of the plain
 *      update) and averages its first cfg->n_avg steps;
 *   3. applies that average for cfg->n_avg world steps;
 *   4. shifts the nominal sequence (and the covariance blocks, when the
 *      full Eq. 8 update is on) by cfg->n_avg steps, repeating the last.
 * After every world step the state is checked: success when the ball
 * centre is within cfg->goal_tol of the goal (the task's target when the
 * ball-task cost suite is on, else the scene's goal); failure on a
 * collision (a link penetrating a box or a link of the other arm), on the
 * ball falling (its centre more than cfg->drop_dz below the highest point
 * it reached once it was cfg->lift_dz above its start) or on reaching
 * cfg->max_steps world steps.  With the task suite on and cfg->pick_tol > 0
 * the pick phase switches to the move phase once the end effectors'
 * midpoint is within pick_tol of the pick point.  Synchronises the stream
 * at every planning step. */
typedef struct {
    int iters;       /* optimiser iterations per planning step, >= 1 */
    int n_avg;       /* steps averaged and executed per planning step, 1..H */
    int max_steps;   /* world steps before a timeout, >= 1 */
    float goal_tol;  /* m */
    float lift_dz;   /* m */
    float drop_dz;   /* m */
    float pick_tol;  /* m; 0 = never switch */
} mppi_episode_config;
enum { MPPI_EP_SUCCESS = 0, MPPI_EP_TIMEOUT = 1, MPPI_EP_COLLISION = 2, MPPI_EP_DROPPED = 3 };
typedef struct {
    int outcome;           /* MPPI_EP_* */
    int plans;             /* planning steps (N_steps) */
    int steps;             /* world steps executed */
    int switch_step;       /* world step of the pick -> move switch, -1 if none */
    double task_time_s;    /* steps x dt */
    double comp_mean_ms;   /* mean and standard deviation of the planning */
    double comp_std_ms;    /* steps' compute time (steps 1-2, CUDA events) */
} mppi_episode_result;
/* x0: HOST, nx floats (the world's start).  u_nom: device, H x nu, the
 * warm start on entry, the last nominal sequence on return.  Optional HOST
 * outputs: traj ((max_steps + 1) x nx world states), u_exec (max_steps x nu
 * executed controls), comp_ms (per planning step, up to max_steps). */
int mppi_run_episode(mppi_ctx *c, const float *x0, float *u_nom, const mppi_episode_config *cfg, float *traj,
                     float *u_exec, float *comp_ms, mppi_episode_result *res, void *stream);

/* Launch shape: samples per CTA for the rollout kernels, 1..32, rounded up
 * to whole warps, at most 512 threads (0 = the library default: the shape
 * that puts the K samples on the SMs in the fewest waves of CTAs with the
 * least load on the busiest SM, from the kernel's occupancy; it follows
 * later layout changes).  A shape whose per-sample workspaces do not fit
 * one CTA's shared memory makes the stepping calls return
 * MPPI_ERR_INVALID_ARG.  Used by the autotuner. */
int mppi_set_launch(mppi_ctx *c, int samples_per_cta);

/* Layout of the rollout kernels.  lanes_per_sample: 32 (one sample per
 * warp), 16 (two) or 8 (four; 3-link arms only); 0 = 32.  The default of a
 * new controller is 16 when K exceeds 16 x the SM count (32-lane groups'
 * registers then cannot hold all samples at once), else 32.  placement of the
 * solve of a lone ball contact with static geometry: 0 = fused with the
 * arms' factorisation (every lane runs both chains), 1 = after it.  Every
 * layout gives bitwise the same samples, costs and updates.  The ball-task
 * cost suite always runs on 32 lanes per sample.  Errors:
 * MPPI_ERR_INVALID_ARG for other values or more than 512 threads per CTA,
 * MPPI_ERR_UNSUPPORTED for 8 lanes with 7-link arms. */
int mppi_set_layout(mppi_ctx *c, int lanes_per_sample, int placement);
int mppi_get_layout(const mppi_ctx *c, int *lanes_per_sample, int *placement, int *samples_per_cta);

/* ---------------------------------------------------------------- batch */
/* Many independent controllers advanced together (the paper runs one
 * optimiser; batching them is this library's serving pattern).  Every
 * instance has its own model, K, H, lambda, sigma and Philox key; all must
 * share the arm size n_a.  One iteration of every instance is one
 * persistent rollout launch -- CTAs take (instance, tile of samples) work
 * items from a device counter, longest instances first -- and one update
 * launch with a CTA per (instance, horizon step).  Each instance's result
 * is bitwise the one mppi_step gives it alone: a sample's rollout is one
 * lane group's work, reduced in a layout-independent order, and the update
 * reduces in a fixed order. */
typedef struct mppi_batch mppi_batch;
typedef struct {
    const mppi_model *model; /* kept alive by the caller for the batch's lifetime */
    int K, H;
    float lambda;
    const float *sigma; /* host, nu floats (copied) */
    uint64_t seed;
} mppi_batch_desc;

int mppi_batch_create(const mppi_batch_desc *desc, int n, mppi_batch **out);
int mppi_batch_destroy(mppi_batch *b);
/* One iteration of every instance: states (host array of n device pointers
 * to nx floats), u (host array of n device pointers to H_i x nu floats,
 * updated in place).  Advances each instance's iteration counter. */
int mppi_batch_step(mppi_batch *b, const float *const *states, float *const *u, void *stream);
/* The same iteration replayed from a CUDA graph (descriptor copy from a
 * pinned table, rollout, update) captured on the first call for `stream`
 * (not the legacy stream).  Passing different pointers than the previous
 * call synchronises `stream` before the table is rewritten. */
int mppi_batch_step_graph(mppi_batch *b, const float *const *states, float *const *u, void *stream);
/* Synchronise; per-instance device status into errors (host, n; optional);
 * returns the first non-OK status. */
int mppi_batch_sync(mppi_batch *b, int *errors, void *stream);
/* Iteration counter of instance i (i = -1 in set: all instances). */
int mppi_batch_iteration(mppi_batch *b, int i, uint64_t *iteration, void *stream);
int mppi_batch_set_iteration(mppi_batch *b, int i, uint64_t iteration, void *stream);
/* Device pointer to instance i's K sample costs of the last iteration. */
const float *mppi_batch_costs(const mppi_batch *b, int i);
/* Launch shape: samples per tile (CTA) 1..32, rounded up to whole warps,
 * at most 256 threads; order 0 = as given, 1 = longest instances first. */
int mppi_batch_set_launch(mppi_batch *b, int samples_per_cta, int order);
int mppi_batch_get_launch(const mppi_batch *b, int *samples_per_cta, int *order);
/* Layout: lanes per sample (32, 16, or 8 for 3-link arms; 0 = 32) and the
 * placement of the lone ball contact's solve (as mppi_set_layout). */
int mppi_batch_set_layout(mppi_batch *b, int lanes_per_sample, int placement);
int mppi_batch_get_layout(const mppi_batch *b, int *lanes_per_sample, int *placement);
/* Autotuner: times `reps` iterations of every shape -- lanes per sample
 * {32, 16, and 8 for 3-link arms} x placement {fused, after} x samples per
 * CTA {1, 2, 4, 8} warps' worth x both orders -- on the given buffers (u is
 * modified: pass scratch copies), keeps the fastest, restores the iteration
 * counters and appends the choice to the tuning table under a key of (nv,
 * box-count bucket, instances, total K, longest H); mppi_batch_create
 * applies a stored choice for its key.  best_ms (optional): time of one
 * iteration. */
int mppi_batch_autotune(mppi_batch *b, const float *const *states, float *const *u, int reps, void *stream,
                        float *best_ms);
/* The paper's full Eq. 8 for instance i (i = -1: every instance), as
 * mppi_set_update does for one controller: elite set of n_elite samples
 * (0 = all), learning rate eta, the covariance blocks updated (and sampled
 * from) when update_cov, diagonal floor cov_floor.  Results stay bitwise
 * those of a single controller with the same settings.  Errors as
 * mppi_set_update. */
int mppi_batch_set_update(mppi_batch *b, int i, int n_elite, float eta, int update_cov, float cov_floor);
/* The QP smoothing projection (Eq. 5) of every instance's samples before its
 * rollouts, as mppi_set_projection: bounds = n x nu x 8 floats (host; per
 * instance and joint lo/hi of position, velocity, acceleration, jerk), the
 * ADMM iterations (0 turns the projection off for the batch), rho and the
 * row scales (NULL = defaults).  Allocates each instance's H x K x nu sample
 * buffer.  MPPI_ERR_INVALID_ARG for bad bounds or instances of different
 * time steps, MPPI_ERR_UNSUPPORTED for H above MPPI_QP_MAX_H. */
int mppi_batch_set_projection(mppi_batch *b, const float *bounds, int iters, float rho, const float *scales);
/* Tuning table: text file of "key spc order lps placement ms" lines at
 * $MPPI_TUNE_FILE (default ~/.cache/mppi_tune.txt); the last entry of a
 * key wins.  Host only; no GPU needed. */
int mppi_tune_store(const char *key, int samples_per_cta, int order, int lanes_per_sample, int placement,
                    float ms);
int mppi_tune_lookup(const char *key, int *samples_per_cta, int *order, int *lanes_per_sample, int *placement);

/* --------------------------------------------------------------- server */
/* Replanning with continuous batching.  Registered scenes keep their
 * simulator state, warm-started nominal sequence and Philox counter on the
 * device (receding horizon with warm start, paper §III-A).  A request asks
 * for one replan of one scene: `iters_per_request` MPPI iterations (Alg. 1
 * with M = iters_per_request).  Waiting requests are admitted while there
 * are free slots (max_active), the scene has no request in flight and the
 * request's workspace (K sample costs) fits the device-memory budget.
 * Admitted requests join the size class of their work per iteration; each
 * class runs on its own stream, one batched iteration of all its requests
 * at a time, and takes newly admitted requests at its next iteration
 * boundary, so classes overlap on the device and short requests do not wait
 * for long ones.  A request that reached M iterations retires: the plan is
 * copied out, the scene's state advances one simulator step under
 * u_nom[0] and u_nom shifts by one step (last step kept).  Latency =
 * retirement time - submission time.  max_active = 1 serves one request at
 * a time (no batching). */
typedef struct mppi_server mppi_server;
typedef struct {
    size_t mem_budget_bytes; /* device arena for active requests' workspaces */
    int max_active;          /* 1..4096 */
    int iters_per_request;   /* M >= 1 */
    int samples_per_cta;     /* launch shape, 0 = default */
    int lanes_per_sample;    /* rollout layout: 32, 16 (0 = 16 for 7-link
                                arms, 32 for 3-link arms) */
    int size_classes;        /* 1..8 streams of requests grouped by work per
                                iteration (K x H in powers of two); 1 = one
                                batch of every active request; 0 = 6 */
    int qp_iters;            /* QP projection (Eq. 5) of every request's
                                samples, ADMM iterations; 0 = off.  Every
                                scene then needs srv_set_scene_projection and
                                a request's workspace holds its H x K x nu
                                projected samples besides the K costs */
} mppi_server_config;
typedef struct {
    long long completed, iterations, waiting, active, admission_waits;
    double p50_ms, p99_ms, mean_ms, mean_active, sample_steps_per_s;
} srv_stats_t;

int srv_create(const mppi_server_config *cfg, mppi_server **out);
int srv_destroy(mppi_server *s);
/* Register a scene before srv_start: model (kept alive by the caller), K,
 * H, lambda, sigma (host, nu), Philox key, initial state (host nx; NULL =
 * the model's home state).  MPPI_ERR_ADMISSION if one request of it can
 * never fit the budget. */
int srv_add_scene(mppi_server *s, const mppi_model *m, int K, int H, float lambda, const float *sigma, uint64_t seed,
                  const float *x0, int *scene_id);
int srv_start(mppi_server *s);
/* Stop the scheduler thread (requests in flight are abandoned); returns the
 * first device or CUDA error the scheduler met. */
int srv_stop(mppi_server *s);
/* Before srv_start: the full Eq. 8 for a scene (as mppi_set_update; its
 * covariance blocks stay resident and carry over to its next request, the
 * warm start of Sigma of Sec. III-A), and a scene's projection bounds (nu x
 * 8 floats, host; rho and scales as mppi_set_projection). */
int srv_set_scene_update(mppi_server *s, int scene_id, int n_elite, float eta, int update_cov, float cov_floor);
int srv_set_scene_projection(mppi_server *s, int scene_id, const float *bounds, float rho, const float *scales);
int srv_submit(mppi_server *s, int scene_id, uint64_t *ticket);
/* Withdraw a request that has not been admitted yet. */
int srv_cancel(mppi_server *s, uint64_t ticket);
/* done = 1 when the request is finished: u_out (host, up to u_len floats of
 * the H x nu plan), latency_ms; the ticket is then released.  Waits up to
 * wait_ms for completion.  Returns the request's status. */
int srv_poll(mppi_server *s, uint64_t ticket, float *u_out, int u_len, double *latency_ms, int *done, int wait_ms);
/* Resident state of a scene (host nx); fails while a request of it is active. */
int srv_get_state(mppi_server *s, int scene_id, float *x_host);
int srv_stats(mppi_server *s, srv_stats_t *out);
/* Poisson load: arrivals at rate_hz for duration_s over the registered
 * scenes (uniform), then wait up to drain_ms for all of them. */
int srv_run_load(mppi_server *s, double rate_hz, double duration_s, uint64_t seed, int drain_ms);

/* --------------------------------------------------------------- no-alloc */
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they plan -- a real-time control
 * loop that must not call cudaMalloc/cudaFree once it runs (those calls can
 * synchronise the device and take unbounded time), or code running inside a
 * host framework that owns the GPU's memory budget.
 *
 * mppi_step_noalloc runs one MPPI iteration exactly like mppi_step (same
 * kernels, same samples for the same seed and iteration) without a model
 * handle or a controller handle and without allocating anything: the scene
 * model, sigma, the control bounds, the error word and the K sample costs go
 * to one static device array of about 36 KB that every GPU loading the
 * library holds until the process exits.
 *   blob, len   scene blob in host memory (as for mppi_model_load), parsed
 *               on every call
 *   K, H        samples and horizon; 1 <= K <= MPPI_NOALLOC_MAX_K and
 *               1 <= H <= 1024, else MPPI_ERR_INVALID_ARG
 *   lambda      temperature > 0;  sigma: nu host floats
 *   seed, iteration   Philox key and counter (the caller keeps the count)
 *   state (device, nx), u_nom, u_nom_out (device, H x nu; may alias)
 *   status_out  optional host int: when non-NULL the call synchronises
 *               `stream` and stores the device status (MPPI_OK,
 *               MPPI_ERR_NONFINITE, MPPI_ERR_CHOLESKY); when NULL the call
 *               only enqueues work and does not wait for the stream
 * The model and parameters reach the device as a kernel parameter of the
 * call's first launch, so no host buffer is read after the call returns.
 * The first call on a device looks up the array's device address with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use this entry point after a
 * cudaDeviceReset on that device (the kept address would be stale).  Every
 * call shares the array and it keeps the last call's contents (the error
 * word is cleared at the start of each call): calls that overlap on the GPU
 * -- on different streams, or from different host threads -- race. */
#define MPPI_NOALLOC_MAX_K 8192
int mppi_step_noalloc(const void *blob, size_t len, int K, int H, float lambda, const float *sigma, uint64_t seed,
                      uint64_t iteration, const float *state, const float *u_nom, float *u_nom_out, int *status_out,
                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MPPI_H */
