/*
 * exact_mppi.h -- C ABI of the GB300 (sm_103a) EXACT-MPPI hot path.
 *
 * EXACT-MPPI (arXiv 2605.29663) scores K sampled control sequences over a
 * horizon T by rolling them out through a kinematic model (Sec. III-D),
 * moving all N obstacle points into every predicted body frame (Sec. IV-C.1)
 * and taking each point's exact signed distance to the robot footprint
 * (simple polygon: Sec. IV-C.3; rectangle cover: Sec. IV-C.2).  The per-step
 * minima feed the collision / clearance cost and the unsafe flag (Sec. IV-E),
 * and the cycle ends with the softmax-weighted update, the validation of the
 * updated nominal and the shift or reset (Sec. III-E, Algorithm 1).
 *
 * Conventions for every entry point below:
 *  - Array arguments marked "device" are caller-owned device memory of the
 *    current CUDA device; the library never frees or retains them.  Arrays
 *    are dense, row-major, float32 unless stated.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream; results are valid once
 *    the stream has been synchronised.
 *  - The return value reports argument and launch errors (exact_status).
 *    Errors found on the device (exact_ctx_get_error) are reported later.
 *  - No C++ exception crosses this boundary.  Thread-compatible: objects may
 *    be used from several host threads only with external synchronisation.
 */
#ifndef EXACT_MPPI_H
#define EXACT_MPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EXACT_OK = 0,
    EXACT_EINVAL = 1,       /* bad argument (NULL, negative size, non-finite value) */
    EXACT_ENOTSIMPLE = 2,   /* polygon is not simple (self-intersection, repeated vertex, zero area) */
    EXACT_ECAPACITY = 3,    /* size beyond a documented maximum */
    EXACT_ECUDA = 4,        /* a CUDA runtime call failed */
    EXACT_ETIMEOUT = 5      /* a bounded device-side wait gave up: the bulk copy that stages a
                               block's obstacle points did not complete (no kernel of this library
                               waits on another block; phases end with atomic tickets) */
} exact_status;

typedef enum { EXACT_FP_POLYGON = 0, EXACT_FP_RECTS = 1 } exact_fp_kind;

/* Motion models of Sec. III-D and their control vectors:
 * DIFF (v, omega), ACKERMANN (v, delta), OMNI (vx, vy, omega),
 * SPIN (omega), PARALLEL (v_para). */
typedef enum {
    EXACT_MM_DIFF = 0, EXACT_MM_ACKERMANN = 1, EXACT_MM_OMNI = 2,
    EXACT_MM_SPIN = 3, EXACT_MM_PARALLEL = 4
} exact_motion;

#define EXACT_MAX_POLY_VERTICES 64
#define EXACT_MAX_RECTS 8
#define EXACT_MAX_HORIZON 128
#define EXACT_MAX_SAMPLES 65536

/* Human-readable name of an exact_status value (static string). */
const char *exact_status_string(int status);

/* ------------------------------------------------------------------ footprint
 * Effective footprint B_eff (Sec. III-B, IV-B), fixed in the body frame.
 * kind = EXACT_FP_POLYGON: host_data = n cyclic vertices (x, y), 3 <= n <= 64,
 *   either orientation (Sec. IV-B.2).  Rejected with EXACT_ENOTSIMPLE when
 *   the boundary self-intersects (O(n^2) host check), repeats a vertex or
 *   encloses zero area.
 * kind = EXACT_FP_RECTS: host_data = n boxes (cx, cy, sx, sy) with half
 *   extents sx, sy > 0, 1 <= n <= 8 (Sec. IV-B.1).
 * The library copies host_data; *out is owned by the caller and released
 * with exact_footprint_destroy.  Changing the footprint means creating a new
 * object: no recompilation and no device allocation is involved. */
typedef struct exact_footprint exact_footprint;
int exact_footprint_create(int kind, const float *host_data, int n, exact_footprint **out);
void exact_footprint_destroy(exact_footprint *fp);
/* Kind and number of vertices / boxes of a footprint. */
int exact_footprint_info(const exact_footprint *fp, int *kind, int *n);

/* ------------------------------------------------------------------ context
 * A context owns the device scratch of mppi_step and of the multi-block
 * exact_sdf_batch reduction, plus a device error word.  It is bound to the
 * device that is current at creation.  Scratch grows on demand (a call with
 * larger sizes than any before may allocate, which must not happen during
 * stream capture); exact_ctx_reserve allocates ahead of time. */
typedef struct exact_ctx exact_ctx;
int exact_ctx_create(exact_ctx **out);
void exact_ctx_destroy(exact_ctx *ctx);
/* Make sure scratch for sdf batches of up to max_poses poses and MPPI steps
 * of up to max_K samples and max_T steps exists (synchronous). */
int exact_ctx_reserve(exact_ctx *ctx, int max_poses, int max_K, int max_T);
/* The same, also for clouds of up to max_points points: an MPPI step without
 * a d_min output keeps a spatially ordered copy of clouds of 1,024 points or
 * more in the context (it makes the pruning of far points effective whatever
 * the input order), so a step with a larger cloud than any before may
 * allocate -- reserve ahead of stream capture. */
int exact_ctx_reserve_cloud(exact_ctx *ctx, int max_poses, int max_K, int max_T, int max_points);
/* Device-side error word of the context (an exact_status, 0 = none): the
 * first error a kernel launched with this context recorded.  Kernels record
 *   EXACT_EINVAL    non-finite device data the host cannot check: the start
 *                   state, the nominal U or the noise of mppi_step, a pose of
 *                   exact_sdf_batch (the call still runs; its results are
 *                   not meaningful);
 *   EXACT_ETIMEOUT  a staging copy that did not complete within its bounded
 *                   wait;
 *   EXACT_ECAPACITY an index out of range, in the debug build only
 *                   (compiled with -DEXACT_DEBUG_CHECKS: every checked access
 *                   is skipped instead of made).
 * The word is read and cleared in the order of `stream` (the stream of the
 * calls whose errors are wanted), which is then synchronised; other streams
 * and the rest of the device are not waited for. */
int exact_ctx_get_error(exact_ctx *ctx, void *stream);

/* Cycle statistics of the MPPI steps run with a context (Sec. III-E weights;
 * diagnostics, the paper reports none): after exact_ctx_enable_stats(ctx, 1)
 * every mppi_step / mppi_step_predicted on ctx also launches one small
 * kernel that records, for that cycle, the effective sample size
 * ESS = 1 / sum_r omega_r^2 of the normalised weights, the minimum and mean
 * of J~, whether the updated nominal passed validation, and counts the
 * cycles and the validation failures since the counters were last read.
 * exact_ctx_get_stats reads (and zeroes the counters) in the order of
 * `stream`, which is then synchronised.  Statistics are off by default
 * (enabling allocates nothing; the record lives in the context). */
typedef struct {
    long long cycles;                /* cycles recorded since the last read */
    long long validation_failures;   /* of which failed validation */
    float ess;                       /* last cycle: 1 / sum omega^2, in [1, K] */
    float cost_min, cost_mean;       /* last cycle: min and mean of J~ */
    int last_valid;                  /* last cycle: 1 if the updated nominal passed */
} exact_cycle_stats;
int exact_ctx_enable_stats(exact_ctx *ctx, int enable);
int exact_ctx_get_stats(exact_ctx *ctx, exact_cycle_stats *out, void *stream);

/* ------------------------------------------------------------------ SDF batch
 * Batched exact signed distance (Sec. IV-C, IV-D; the evaluator of
 * Experiment 1).  For pose p = (x, y, theta) and point o_i every point is
 * moved into the body frame, p_i = R(theta)^T (o_i - (x, y)), and its signed
 * distance to the footprint is taken (negative inside).
 *   points  device, n_points x 2 (x, y) in the planning frame
 *   mask    device, n_points uint8 (0 = padding) or NULL (all valid)
 *   poses   device, n_poses x 3 (x, y, theta)
 *   dist    device, n_poses x n_points, or NULL: signed distances; padded
 *           points get +inf
 *   dmin    device, n_poses, or NULL: masked minimum (+inf if no valid point)
 *   argmin  device, n_poses int32, or NULL: index of the minimum (lowest
 *           index among equal float32 keys; -1 if no valid point)
 * n_points, n_poses >= 0 (0 is a no-op); n_points * n_poses < 2^62.  ctx
 * supplies scratch when many blocks share one pose; it may be NULL, in which
 * case each pose is reduced by a single block. */
int exact_sdf_batch(exact_ctx *ctx, const float *points, const uint8_t *mask, int n_points,
                    const float *poses, int n_poses, const exact_footprint *fp,
                    float *dist, float *dmin, int *argmin, void *stream);

/* ------------------------------------------------------------------ MPPI step
 * Parameters of one control cycle (Algorithm 1 "Params" plus the task /
 * control cost of Sec. III-E, which the paper leaves open):
 *   J = sum_h [ w_goal * dist(s_h, guidance) + w_ctrl * |u_h|^2 + phi_obs(d_h) ]
 *       + w_term * dist(q_T, guidance),
 *   phi_obs(d) = w_coll * I(d < 0) + w_rep * max(d_safe - d, 0)^2,
 *   chi = OR_h (d_h < d_safe),  J~ = J + w_inf * I(chi),
 * where s_h = q_{h+1} (state_offset = 1) or q_h (state_offset = 0, the
 * printed indexing).  clamp != 0 clips every sampled control to
 * [u_min, u_max] and uses the clipped perturbation in the update. */
typedef struct {
    int K, T, n_u, model;             /* samples, horizon, control dim, exact_motion */
    float dt, lambda, d_safe;
    float w_coll, w_rep, w_inf, w_goal, w_term, w_ctrl;
    float wheelbase;                  /* Ackermann L */
    float u_min[3], u_max[3];
    int clamp, state_offset;
} exact_mppi_params;

/* One batched EXACT-MPPI control cycle (Algorithm 1) for one robot.
 *   state     device, 3: q_0 = (x, y, theta)
 *   cloud     device, n_points x 2 obstacle points; mask device n_points or NULL
 *   waypoints device, n_wp x 2: a goal point (n_wp = 1) or a polyline
 *   U         device, T x n_u, in/out: the nominal sequence; on return the
 *             shifted sequence (last entry repeated) if validation passed,
 *             all zeros otherwise
 *   noise     device, K x T x n_u perturbations eps (Sec. III-E)
 *   u_star    device, n_u: the executed command (zero on validation failure)
 *   costs     device, K, or NULL: J~ per sample
 *   weights   device, K, or NULL: omega per sample
 *   valid     device, 1 int32, or NULL: 1 if the updated nominal passed
 *   U_upd     device, T x n_u, or NULL: the updated nominal before shift/reset
 *   dmin      device, K x T, or NULL: d_min of every scored rollout state.
 *             Without it the sample phase skips the points that provably
 *             cannot come within d_safe of the footprint at a step (bounding
 *             circles of point sub-chunks, then the footprint's bounding box
 *             for the points or 16-point fine sub-chunks of the kept ones;
 *             below 1,024 points, bounding circles per point): every cost
 *             term and the validation test are the same for any d >= d_safe,
 *             so costs, weights and U are identical either way
 * Limits: 1 <= K <= 65536, 1 <= T <= 128, n_points >= 0, n_wp >= 1,
 * n_u must match the model.  Scratch comes from ctx (grown on demand). */
int mppi_step(exact_ctx *ctx, const float *state, const float *cloud, const uint8_t *mask,
              int n_points, const float *waypoints, int n_wp, float *U, const float *noise,
              const exact_footprint *fp, const exact_mppi_params *params,
              float *u_star, float *costs, float *weights, int *valid, float *U_upd,
              float *dmin, void *stream);

/* mppi_step with time-indexed obstacle predictions (the extension named in
 * Sec. V-F: signed-distance costs against predicted obstacle positions along
 * the horizon instead of the current observation only).  Every point i has a
 * velocity v_i and at horizon step h it is evaluated at the constant-velocity
 * prediction o_i + t_h v_i, t_h = (h + state_offset) dt being the time of the
 * scored state (the validation of the updated nominal uses the same
 * predictions).  velocity: device, n_points x 2 (m/s), 8-byte aligned,
 * required when n_points > 0; a point whose predicted position is not finite
 * is ignored like a masked one.  Everything else as mppi_step; zero
 * velocities give mppi_step's results. */
int mppi_step_predicted(exact_ctx *ctx, const float *state, const float *cloud, const float *velocity,
                        const uint8_t *mask, int n_points, const float *waypoints, int n_wp, float *U,
                        const float *noise, const exact_footprint *fp, const exact_mppi_params *params,
                        float *u_star, float *costs, float *weights, int *valid, float *U_upd,
                        float *dmin, void *stream);

/* ------------------------------------------------------------------ learned proposal
 * Project extension (the paper has no learned component): a small network
 * shifts the sampling mean of MPPI; plain MPPI on the same noise remains the
 * fallback whenever the shifted candidate's best J~ is not lower.
 *
 * Network: y = W3 g(W2 g(W1 x + b1) + b2) + b3, g = exact GELU
 * (z Phi(z)); W1 hidden x d_in, W2 hidden x hidden, W3 d_out x hidden,
 * row-major.  BF16 x BF16 -> FP32 tensor-core products, FP32 master
 * parameters and Adam moments (beta1 0.9, beta2 0.999, eps 1e-8), loss =
 * mean squared error over batch and outputs.  Parameters are exchanged as
 * one packed FP32 vector [W1, b1, W2, b2, W3, b3] of exact_mlp_num_params
 * floats.  d_in <= 128, hidden <= 1024, d_out <= 256, batch <= max_batch.
 * exact_mlp_create allocates device memory; the other calls do not. */
typedef struct exact_mlp exact_mlp;
int exact_mlp_create(int d_in, int hidden, int d_out, int max_batch, exact_mlp **out);
void exact_mlp_destroy(exact_mlp *m);
long long exact_mlp_num_params(const exact_mlp *m);
/* host packed parameters in / out (synchronous); set resets Adam */
int exact_mlp_set_params(exact_mlp *m, const float *host_params);
int exact_mlp_get_params(const exact_mlp *m, float *host_params);
/* The whole training state for a checkpoint (synchronous): parameters and
 * Adam's first and second moments (host, exact_mlp_num_params floats each)
 * and the Adam step count.  Setting a state got from another object of the
 * same shape resumes training exactly: the next steps give the same bits as
 * the uninterrupted run (every kernel reduces in a fixed order). */
int exact_mlp_get_state(const exact_mlp *m, float *host_params, float *host_m, float *host_v, long long *step);
int exact_mlp_set_state(exact_mlp *m, const float *host_params, const float *host_m, const float *host_v,
                        long long step);
/* x device B x d_in -> y device B x d_out */
int exact_mlp_forward(exact_mlp *m, const float *x, int B, float *y, void *stream);
/* loss (device 1 float, or NULL) and gradients (device packed vector, or
 * NULL) of the mean squared error against target (device B x d_out) */
int exact_mlp_loss_grad(exact_mlp *m, const float *x, const float *target, int B, float *loss, float *grads,
                        void *stream);
/* one Adam step with learning rate lr on (x, target); loss as above */
int exact_mlp_train_step(exact_mlp *m, const float *x, const float *target, int B, float lr, float *loss,
                         void *stream);

/* Polar nearest-range histogram of B robots: clouds device B x N x 2,
 * masks device B x N or NULL, poses device B x 3.  Each valid point is moved
 * into its robot's body frame; bin = floor((atan2(p_y, p_x) + pi) / (2 pi)
 * nbins) clamped to nbins - 1; out (device B x nbins) = min(r_max, nearest
 * range in the bin). */
int exact_polar_hist(const float *clouds, const uint8_t *masks, int B, int N, const float *poses, int nbins,
                     float r_max, float *out, void *stream);
/* Network input of B robots, x (device B x (nbins + 7 + 2T)) =
 * [hist / r_max, goal in the body frame / r_max, previous command (v, w),
 *  |goal| / r_max, cos and sin of the goal bearing, previous nominal U (T x 2)];
 * poses B x 3, goals B x 2 (planning frame), prev_cmd B x 2, U_prev B x T x 2. */
int exact_proposal_features(const float *hist, int nbins, float r_max, const float *poses, const float *goals,
                            const float *prev_cmd, const float *U_prev, int T, int B, float *x, void *stream);
/* U_prop = U_prev + shift, U_plain = U_prev (n floats each, device). */
int exact_proposal_prepare(const float *U_prev, const float *shift, long long n, float *U_prop, float *U_plain,
                           void *stream);
/* Per robot b: keep the proposal candidate when min_r costs_prop[b] <
 * min_r costs_plain[b] (device B x K each): copy its nominal (B x T x nu)
 * and command (B x nu) to U_out / u_out; chose_prop (device B, or NULL)
 * records the choice. */
int exact_proposal_select(const float *costs_prop, const float *costs_plain, int B, int K, const float *U_prop,
                          const float *U_plain, const float *u_prop, const float *u_plain, int T, int nu,
                          float *U_out, float *u_out, int *chose_prop, void *stream);

/* ------------------------------------------------------------------ no allocation
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory (a control loop that must not call
 * cudaMalloc after start-up, code running during stream capture, a program
 * whose device memory belongs to another allocator).
 *
 * mppi_step_noalloc computes what mppi_step computes (the same kernels, the
 * same output bits) without a context: its scratch is a file-scope device
 * array of EXACT_NOALLOC_ARENA_BYTES that every GPU loading the library
 * holds until the process exits.  One difference in cost, not in results:
 * without a d_min output and with 1,024 points or more, mppi_step prunes far
 * point chunks on a spatially ordered copy of the cloud kept in its context,
 * while this call prunes on the cloud in the order given, which skips fewer
 * chunks (and so runs slower) when consecutive points are not close together.  It allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call); it clears the parts of the array
 * that must start at zero with stream-ordered memsets on `stream`.
 *  - The first call on a device looks the array's device address up (once,
 *    with that device current); make that first call before any stream
 *    capture.
 *  - Every call shares the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and give wrong results.
 *  - Sizes whose scratch does not fit the array return EXACT_ECAPACITY
 *    (4 MiB holds, e.g., K = 16384 samples with T = 128 and n_u = 3).
 * Arguments, layouts and the remaining errors are those of mppi_step. */
#define EXACT_NOALLOC_ARENA_BYTES (4u << 20)
int mppi_step_noalloc(const float *state, const float *cloud, const uint8_t *mask, int n_points,
                      const float *waypoints, int n_wp, float *U, const float *noise,
                      const exact_footprint *fp, const exact_mppi_params *params,
                      float *u_star, float *costs, float *weights, int *valid, float *U_upd,
                      float *dmin, void *stream);

/* ------------------------------------------------------------------ batches
 * Many independent scenes (robots) with different K, T, N, footprints and
 * motion models advanced by one control cycle each in a single persistent
 * launch (plus two small table-driven launches for the update and the
 * validation).  A scene is Algorithm 1 exactly as in mppi_step; only the
 * scheduling differs.  Every pointer in exact_scene refers to caller-owned
 * device memory laid out as for mppi_step (optional outputs may be NULL);
 * fp is a footprint object (its constants are copied into the batch). */
typedef struct {
    const float *state;          /* device, 3 */
    const float *cloud;          /* device, n_points x 2 */
    const uint8_t *mask;         /* device, n_points, or NULL */
    int n_points;
    const float *waypoints;      /* device, n_wp x 2 */
    int n_wp;
    float *U;                    /* device, T x n_u, in/out */
    const float *noise;          /* device, K x T x n_u */
    const exact_footprint *fp;
    exact_mppi_params params;
    float *u_star;               /* device, n_u */
    float *costs;                /* device, K, or NULL */
    float *weights;              /* device, K, or NULL */
    int *valid;                  /* device, 1, or NULL */
    float *U_upd;                /* device, T x n_u, or NULL */
    float *dmin;                 /* device, K x T, or NULL */
    float *nom_cost;             /* device, 1, or NULL: cost J of the updated nominal,
                                    scored like a sample (the J_m of Algorithm 2) */
} exact_scene;

/* A batch plan: validates the scenes, uploads a device scene table, the
 * work-item list (one item per (scene, sample), or per two samples of a
 * scene when the batch holds at least four samples per SM and T <= 64;
 * heaviest scenes first) and the
 * per-scene scratch (synchronous; allocates device memory).  The scene
 * pointers are fixed for the life of the plan; their contents may change
 * between steps.  1 <= n_scenes <= 4096; each scene obeys the mppi_step
 * limits.  *out is released with exact_batch_destroy. */
typedef struct exact_batch exact_batch;
int exact_batch_create(int n_scenes, const exact_scene *scenes, exact_batch **out);
void exact_batch_destroy(exact_batch *batch);

/* One control cycle of every scene of the batch: a queue reset, the
 * persistent sample kernel, the update kernel and the validation kernel on
 * `stream` (no allocation, no host synchronisation: capturable in a CUDA
 * graph).  Calls on one batch must not overlap on the GPU. */
int mppi_step_batched(exact_batch *batch, void *stream);

/* Tile autotuner: times the batch's sample phase (which writes only batch
 * scratch, never the scenes' U or outputs) for each candidate tile shape
 * (threads per block x point pairs per lane: the sample phase cuts the
 * staged cloud into sub-chunks of 64 x pairs_per_lane points, the unit it
 * skips when a sub-chunk cannot come within d_safe of the footprint at a
 * step; scenes without a d_min output only), `iters` runs
 * each, keeps the fastest for later steps and, when json_out is non-NULL,
 * writes the timings as JSON text (at most json_cap bytes, NUL-terminated).
 * Synchronises `stream`. */
int exact_batch_autotune(exact_batch *batch, int iters, char *json_out, int json_cap, void *stream);
/* The batch's device error word (as exact_ctx_get_error: first error of
 * any of its kernels, read and cleared in the order of `stream`, which is
 * then synchronised).  A hybrid object reports through its batch
 * (exact_hybrid_batch). */
int exact_batch_get_error(exact_batch *batch, void *stream);
/* Current tile shape of the batch. */
int exact_batch_get_tiles(const exact_batch *batch, int *threads, int *pairs_per_lane);
/* Set the tile shape (threads in {64, 128, 256, 512}, pairs_per_lane in 1..8). */
int exact_batch_set_tiles(exact_batch *batch, int threads, int pairs_per_lane);

/* ------------------------------------------------------------------ hybrid modes
 * Hybrid-mode EXACT-MPPI (Sec. IV-F, Algorithm 2, steps 1-2) for platforms
 * with several non-skidding motion modes (e.g. Ackermann, parallel, spin).
 * Each mode m is a scene (exact_scene) of the same robot: it shares the
 * caller's state, cloud and footprint as the caller chooses and has its own
 * motion model, nominal sequence U_m, noise and parameters.  One step runs
 * Algorithm 1 for every mode (one batched launch set, as mppi_step_batched:
 * each U_m is updated and shifted or reset), then one selection kernel:
 *   Jbar_m = J_m + lambda_switch * I(m != m_prev) if mode m's nominal passed
 *            validation, else +inf, J_m = cost of mode m's updated nominal;
 *   all +inf: safe stop (zero command, m_prev and tau_cool unchanged);
 *   m* = argmin Jbar_m (lowest mode index on ties); while tau_cool > 0 a
 *   switch away from m_prev is refused (m* = m_prev; m_prev = -1 means no
 *   mode yet and is never kept);
 *   tau_cool = cool_max after a switch, else max(tau_cool - 1, 0).
 * The command is the chosen mode's first command (Algorithm 1's u*: zero if
 * that mode failed validation).  The actuator post-processing of Algorithm 2
 * (deadzone scaling) is hardware-specific and not part of the library. */
#define EXACT_MAX_MODES 8
typedef struct {
    float lambda_switch;   /* switching penalty, >= 0 */
    int cool_max;          /* tau_cool^max, >= 0: cycles after a switch that refuse another */
} exact_hybrid_params;

typedef struct exact_hybrid exact_hybrid;
/* 1 <= n_modes <= EXACT_MAX_MODES; each mode obeys the exact_batch_create
 * rules (its valid and nom_cost outputs may be NULL: the object then keeps
 * its own).  Synchronous; allocates device memory; *out is released with
 * exact_hybrid_destroy. */
int exact_hybrid_create(int n_modes, const exact_scene *modes, const exact_hybrid_params *hp,
                        exact_hybrid **out);
void exact_hybrid_destroy(exact_hybrid *hybrid);
/* One hybrid cycle on `stream` (no allocation, no host synchronisation:
 * capturable in a CUDA graph).
 *   mode_state device, 3 int32, in/out: [m_prev, tau_cool, stopped]; on
 *              return [m*, tau_cool', 1 on a safe stop else 0]
 *   u_out      device, 3: the chosen mode's first command, its n_u entries
 *              followed by zeros (all zero on a safe stop)
 *   Jbar       device, n_modes, or NULL: the augmented costs (+inf = invalid)
 * Calls on one object must not overlap on the GPU. */
int mppi_step_hybrid(exact_hybrid *hybrid, int *mode_state, float *u_out, float *Jbar, void *stream);
/* The batch that runs the modes (for its tile autotuner). */
exact_batch *exact_hybrid_batch(exact_hybrid *hybrid);

#ifdef __cplusplus
}
#endif
#endif /* EXACT_MPPI_H */
