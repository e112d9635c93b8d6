/*
 * exact_oracle.c -- plain FP64 CPU oracle for EXACT-MPPI
 * ("EXACT-MPPI: Exact Signed-Distance Navigation for Arbitrary-Footprint
 * Robots from Point Clouds via Path Integral Control", arXiv 2605.29663).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * library.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may build, load or call it; the product path never does.  It
 * shares no code, header, table or constant generator with the CUDA sources.
 *
 * Everything is double precision and written for readability, not speed: no
 * blocking, no fusion, no reordering beyond what the paper's definitions state.
 * Each function names the section / equation / algorithm it restates.
 *
 * Readings of points where the paper is silent (mirrored in the design notes):
 *  - zero-length polygon edge: clipped projection parameter alpha = 0, i.e.
 *    the distance to the vertex;
 *  - a query point exactly on the boundary returns +0.0;
 *  - masked-out (padding) obstacle points get +inf in a full distance matrix
 *    and never take part in a minimum; a minimum over no valid point is +inf;
 *  - the scored state of horizon step h is q_{h+1} (state_offset = 1) or the
 *    literal q_h of the printed cost sum (state_offset = 0);
 *  - phi_task = w_goal * distance to the goal (nearest point of the waypoint
 *    polyline), phi_ctrl = w_ctrl * |u|^2, plus w_term * terminal goal
 *    distance; clamped perturbations eps' = clamp(u + eps) - u enter the
 *    update; the shifted sequence repeats its last entry.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { OX_FP_POLYGON = 0, OX_FP_RECTS = 1 };
enum { OX_DIFF = 0, OX_ACKERMANN = 1, OX_OMNI = 2, OX_SPIN = 3, OX_PARALLEL = 4 };

int ox_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ox_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * Sec. IV-C.1, rollout-frame transformation: p = R(theta)^T (o - t).
 * R(theta) = [[c, -s], [s, c]], so R^T (dx, dy) = (c dx + s dy, -s dx + c dy).
 * ------------------------------------------------------------------------- */
void ox_body_frame(double ox, double oy, double tx, double ty, double th,
                   double *px, double *py) {
    double c = cos(th), s = sin(th);
    double dx = ox - tx, dy = oy - ty;
    *px = c * dx + s * dy;
    *py = -s * dx + c * dy;
}

/* ---------------------------------------------------------------------------
 * Sec. IV-C.2, point-to-box signed distance for a box with centre c and
 * half-extent s:  a = |p - c| - s (elementwise),
 *   d_box = || max(a, 0) ||_2 + min(max(a_x, a_y), 0).
 * ------------------------------------------------------------------------- */
double ox_sdf_box(double px, double py, double cx, double cy, double sx, double sy) {
    double ax = fabs(px - cx) - sx;
    double ay = fabs(py - cy) - sy;
    double mx = ax > 0.0 ? ax : 0.0;
    double my = ay > 0.0 ? ay : 0.0;
    double inner = ax > ay ? ax : ay;
    if (inner > 0.0) inner = 0.0;
    return sqrt(mx * mx + my * my) + inner;
}

/* Rectangle cover: d_rect = min_j d_box,j (Sec. IV-C.2).  rects = R x (cx, cy, sx, sy). */
double ox_sdf_rect(double px, double py, const double *rects, int R) {
    double best = INFINITY;
    for (int j = 0; j < R; ++j) {
        const double *b = rects + 4 * j;
        double d = ox_sdf_box(px, py, b[0], b[1], b[2], b[3]);
        if (d < best) best = d;
    }
    return best;
}

/* ---------------------------------------------------------------------------
 * Sec. IV-C.3, distance to the edge e_b = v_{b+1} - v_b:
 *   alpha_b = max(0, min(1, (p - v_b).e_b / |e_b|^2)),
 *   d_seg,b = || p - (v_b + alpha_b e_b) ||.
 * (The printed formula places the parenthesis around v_b + alpha_b; the
 *  product alpha_b e_b is the reading that makes it a point on the segment.)
 * ------------------------------------------------------------------------- */
double ox_seg_dist(double px, double py, double vx, double vy, double wx, double wy) {
    double ex = wx - vx, ey = wy - vy;
    double len2 = ex * ex + ey * ey;
    double alpha = 0.0;
    if (len2 > 0.0) {
        alpha = ((px - vx) * ex + (py - vy) * ey) / len2;
        if (alpha < 0.0) alpha = 0.0;
        if (alpha > 1.0) alpha = 1.0;
    }
    double qx = vx + alpha * ex, qy = vy + alpha * ey;
    double rx = px - qx, ry = py - qy;
    return sqrt(rx * rx + ry * ry);
}

/* Sec. IV-C.3 sign: point-in-polygon by ray casting.  A horizontal ray from
 * p towards +x toggles the parity at every edge that straddles the line
 * y = p_y (one end strictly above, the other not) and whose crossing lies
 * strictly to the right of p.  Returns 1 inside, 0 outside. */
int ox_inside_poly(double px, double py, const double *v, int B) {
    int inside = 0;
    for (int b = 0; b < B; ++b) {
        double vx = v[2 * b], vy = v[2 * b + 1];
        int nb = (b + 1) % B;
        double wx = v[2 * nb], wy = v[2 * nb + 1];
        int above_v = vy > py, above_w = wy > py;
        if (above_v != above_w) {
            double x_cross = vx + (py - vy) * (wx - vx) / (wy - vy);
            if (px < x_cross) inside = !inside;
        }
    }
    return inside;
}

/* d_poly = sigma * min_b d_seg,b (Sec. IV-C.3).  v = B cyclic vertices. */
double ox_sdf_poly(double px, double py, const double *v, int B) {
    double m = INFINITY;
    for (int b = 0; b < B; ++b) {
        int nb = (b + 1) % B;
        double d = ox_seg_dist(px, py, v[2 * b], v[2 * b + 1], v[2 * nb], v[2 * nb + 1]);
        if (d < m) m = d;
    }
    if (m == 0.0) return 0.0;
    return ox_inside_poly(px, py, v, B) ? -m : m;
}

double ox_sdf(double px, double py, int kind, const double *fp, int n) {
    return kind == OX_FP_RECTS ? ox_sdf_rect(px, py, fp, n) : ox_sdf_poly(px, py, fp, n);
}

/* d_min at one pose (Sec. III-C / IV-D): minimum signed distance over the
 * valid obstacle points after moving them into the body frame of the pose.
 * Returns +inf when no point is valid; *arg receives the first index that
 * attains the minimum (or -1). */
double ox_dmin_pose(const double *pts, const uint8_t *mask, int N,
                    double x, double y, double th, int kind, const double *fp, int n,
                    int64_t *arg) {
    double best = INFINITY;
    int64_t a = -1;
    for (int i = 0; i < N; ++i) {
        if (mask && !mask[i]) continue;
        double px, py;
        ox_body_frame(pts[2 * i], pts[2 * i + 1], x, y, th, &px, &py);
        double d = ox_sdf(px, py, kind, fp, n);
        if (d < best) { best = d; a = i; }
    }
    if (arg) *arg = a;
    return best;
}

/* Batched signed distance (Sec. IV-D, Experiment 1): for every pose and
 * every point, the body-frame signed distance; per pose the masked minimum
 * and its first argmin.  dist (P x N), dmin (P) and argmin (P) may be NULL. */
void ox_sdf_batch(const double *pts, const uint8_t *mask, int N,
                  const double *poses, int P, int kind, const double *fp, int n,
                  double *dist, double *dmin, int64_t *argmin) {
    #pragma omp parallel for schedule(dynamic, 8)
    for (int p = 0; p < P; ++p) {
        double x = poses[3 * p], y = poses[3 * p + 1], th = poses[3 * p + 2];
        double best = INFINITY;
        int64_t a = -1;
        for (int i = 0; i < N; ++i) {
            int valid = !mask || mask[i];
            double px, py;
            ox_body_frame(pts[2 * i], pts[2 * i + 1], x, y, th, &px, &py);
            double d = ox_sdf(px, py, kind, fp, n);
            if (dist) dist[(int64_t)p * N + i] = valid ? d : INFINITY;
            if (valid && d < best) { best = d; a = i; }
        }
        if (dmin) dmin[p] = best;
        if (argmin) argmin[p] = a;
    }
}

/* ---------------------------------------------------------------------------
 * Sec. III-D kinematics and forward-Euler propagation
 *   q_{h+1} = q_h + F_m(q_h, u_h) dt   (x, y use the old heading theta_h).
 * n_u: diff 2 (v, w), ackermann 2 (v, delta), omni 3 (vx, vy, w),
 *      spin 1 (w), parallel 1 (v_para).
 * ------------------------------------------------------------------------- */
void ox_kinematics(int model, double L, double th, const double *u, double F[3]) {
    double c = cos(th), s = sin(th);
    switch (model) {
    case OX_DIFF:      F[0] = u[0] * c; F[1] = u[0] * s; F[2] = u[1]; break;
    case OX_ACKERMANN: F[0] = u[0] * c; F[1] = u[0] * s; F[2] = u[0] / L * tan(u[1]); break;
    case OX_OMNI:      F[0] = u[0] * c - u[1] * s; F[1] = u[0] * s + u[1] * c; F[2] = u[2]; break;
    case OX_SPIN:      F[0] = 0.0; F[1] = 0.0; F[2] = u[0]; break;
    case OX_PARALLEL:  F[0] = -u[0] * s; F[1] = u[0] * c; F[2] = 0.0; break;
    default:           F[0] = F[1] = F[2] = NAN; break;
    }
}

int ox_model_nu(int model) {
    switch (model) {
    case OX_DIFF: case OX_ACKERMANN: return 2;
    case OX_OMNI: return 3;
    case OX_SPIN: case OX_PARALLEL: return 1;
    default: return 0;
    }
}

/* states: (T+1) x 3, states[0] = q0. u: T x nu. */
void ox_rollout(int model, double L, const double q0[3], const double *u, int T, int nu,
                double dt, double *states) {
    states[0] = q0[0]; states[1] = q0[1]; states[2] = q0[2];
    for (int h = 0; h < T; ++h) {
        double F[3];
        const double *q = states + 3 * h;
        ox_kinematics(model, L, q[2], u + (int64_t)h * nu, F);
        states[3 * (h + 1) + 0] = q[0] + F[0] * dt;
        states[3 * (h + 1) + 1] = q[1] + F[1] * dt;
        states[3 * (h + 1) + 2] = q[2] + F[2] * dt;
    }
}

/* Distance from (x, y) to the guidance: a single goal point, or the nearest
 * point of the waypoint polyline (Sec. IV-A weak guidance; phi_task reading). */
double ox_goal_dist(double x, double y, const double *wp, int W) {
    if (W <= 0) return 0.0;
    if (W == 1) {
        double dx = x - wp[0], dy = y - wp[1];
        return sqrt(dx * dx + dy * dy);
    }
    double best = INFINITY;
    for (int k = 0; k + 1 < W; ++k) {
        double d = ox_seg_dist(x, y, wp[2 * k], wp[2 * k + 1], wp[2 * k + 2], wp[2 * k + 3]);
        if (d < best) best = d;
    }
    return best;
}

/* Alg. 1 parameters (names follow the paper; task/control weights and the
 * clamp / state_offset switches are the readings listed above). */
typedef struct {
    int K, T, nu, model;
    double dt, lambda, d_safe, w_coll, w_rep, w_inf, w_goal, w_term, w_ctrl, wheelbase;
    double u_min[3], u_max[3];
    int clamp, state_offset;
} ox_params;

/* phi_obs (Sec. IV-E): w_coll * I(d < 0) + w_rep * max(d_safe - d, 0)^2. */
double ox_phi_obs(double d, double d_safe, double w_coll, double w_rep) {
    double gap = d_safe - d;
    if (gap < 0.0) gap = 0.0;
    return w_coll * (d < 0.0 ? 1.0 : 0.0) + w_rep * gap * gap;
}

static int near_threshold(double d, double d_safe, double tol) {
    return fabs(d) < tol || fabs(d - d_safe) < tol;
}

/* Cost of one control sequence u (T x nu, already clamped), Sec. III-E cost
 * J plus the unsafe flag chi (Sec. IV-E).  dmin_out (T) may be NULL; *near
 * counts horizon steps whose d_min lies within tol of 0 or d_safe.
 * vel (N x 2) or NULL: time-indexed obstacle prediction (the extension of
 * Sec. V-F) -- at step h the points are at o + t v, t = (h + state_offset) dt
 * the time of the scored state; moved (N x 2) is scratch for them. */
static double sequence_cost(const ox_params *P, const double q0[3], const double *u,
                            const double *cloud, const double *vel, double *moved,
                            const uint8_t *mask, int N,
                            const double *wp, int W, int kind, const double *fp, int n,
                            double *states, double *dmin_out, int *chi_out,
                            int *near, double tol) {
    int T = P->T, nu = P->nu;
    ox_rollout(P->model, P->wheelbase, q0, u, T, nu, P->dt, states);
    double J = 0.0;
    int chi = 0, nn = 0;
    for (int h = 0; h < T; ++h) {
        const double *s = states + 3 * (h + P->state_offset);
        const double *pts = cloud;
        if (vel) {
            double t = (double)(h + P->state_offset) * P->dt;
            for (int i = 0; i < 2 * N; ++i) moved[i] = cloud[i] + t * vel[i];
            pts = moved;
        }
        double d = ox_dmin_pose(pts, mask, N, s[0], s[1], s[2], kind, fp, n, NULL);
        if (dmin_out) dmin_out[h] = d;
        double u2 = 0.0;
        for (int j = 0; j < nu; ++j) u2 += u[h * nu + j] * u[h * nu + j];
        J += P->w_goal * ox_goal_dist(s[0], s[1], wp, W)
           + P->w_ctrl * u2
           + ox_phi_obs(d, P->d_safe, P->w_coll, P->w_rep);
        if (d < P->d_safe) chi = 1;
        if (near_threshold(d, P->d_safe, tol)) ++nn;
    }
    const double *qT = states + 3 * T;
    J += P->w_term * ox_goal_dist(qT[0], qT[1], wp, W);
    *chi_out = chi;
    if (near) *near += nn;
    return J;
}

static double clamp_dim(const ox_params *P, int j, double u) {
    if (!P->clamp) return u;
    if (u < P->u_min[j]) u = P->u_min[j];
    if (u > P->u_max[j]) u = P->u_max[j];
    return u;
}

/* Algorithm 1, one batched control cycle, followed step by step.
 *   in : q0 (3), cloud (N x 2) + mask (N or NULL), vel (N x 2 point
 *        velocities for time-indexed predictions, or NULL), waypoints
 *        (W x 2), U (T x nu), eps (K x T x nu), footprint.
 *   out: U (T x nu, shifted or reset), u_star (nu), costs J~ (K), weights
 *        omega (K), *valid, U_upd (updated nominal before shift/reset),
 *        dmin (K x T) and dmin_nom (T) when non-NULL, *J_nom = the cost J of
 *        the updated nominal (scored like a sample, zero noise) when non-NULL,
 *        *n_near = number of (sample, step) and nominal steps whose d_min lies
 *        within near_tol of 0 or d_safe (where FP32 and FP64 may legitimately
 *        disagree).
 * Returns 0, or -1 on bad arguments / allocation failure. */
int ox_mppi_step(const ox_params *P, const double q0[3],
                 const double *cloud, const double *vel, const uint8_t *mask, int N,
                 const double *wp, int W, double *U, const double *eps,
                 int kind, const double *fp, int n,
                 double *u_star, double *costs, double *weights, int *valid,
                 double *U_upd, double *dmin, double *dmin_nom, double *J_nom,
                 int *n_near, double near_tol) {
    int K = P->K, T = P->T, nu = P->nu;
    if (K <= 0 || T <= 0 || nu != ox_model_nu(P->model) || !(P->lambda > 0.0)) return -1;
    double *epsc = (double *)malloc(sizeof(double) * (size_t)K * T * nu);
    double *Jt = (double *)malloc(sizeof(double) * (size_t)K);
    if (!epsc || !Jt) { free(epsc); free(Jt); return -1; }
    int near_total = 0;

    /* Steps 1-2: sample, propagate, evaluate d_min, accumulate J and chi. */
    #pragma omp parallel for schedule(dynamic, 4) reduction(+:near_total)
    for (int r = 0; r < K; ++r) {
        double *u = (double *)malloc(sizeof(double) * (size_t)T * nu);
        double *st = (double *)malloc(sizeof(double) * (size_t)(T + 1) * 3);
        double *mv = vel ? (double *)malloc(sizeof(double) * (size_t)2 * (N > 0 ? N : 1)) : NULL;
        for (int h = 0; h < T; ++h)
            for (int j = 0; j < nu; ++j) {
                int64_t k = ((int64_t)r * T + h) * nu + j;
                double uh = U[h * nu + j];
                double v = clamp_dim(P, j, uh + eps[k]);
                u[h * nu + j] = v;
                /* the perturbation that was actually applied */
                epsc[k] = P->clamp ? v - uh : eps[k];
            }
        int chi = 0, nn = 0;
        double J = sequence_cost(P, q0, u, cloud, vel, mv, mask, N, wp, W, kind, fp, n, st,
                                 dmin ? dmin + (int64_t)r * T : NULL, &chi, &nn, near_tol);
        /* Step 3: J~ = J + w_inf I(chi). */
        Jt[r] = J + P->w_inf * (chi ? 1.0 : 0.0);
        near_total += nn;
        free(u); free(st); free(mv);
    }

    /* Step 3: beta = min J~, omega = exp(-(J~ - beta)/lambda) / sum. */
    double beta = INFINITY;
    for (int r = 0; r < K; ++r) if (Jt[r] < beta) beta = Jt[r];
    double Z = 0.0;
    for (int r = 0; r < K; ++r) Z += exp(-(Jt[r] - beta) / P->lambda);
    for (int r = 0; r < K; ++r) {
        double w = exp(-(Jt[r] - beta) / P->lambda) / Z;
        if (weights) weights[r] = w;
        if (costs) costs[r] = Jt[r];
    }
    /* u_h <- u_h + sum_r omega_r eps_h^(r). */
    for (int h = 0; h < T; ++h)
        for (int j = 0; j < nu; ++j) {
            double acc = 0.0;
            for (int r = 0; r < K; ++r)
                acc += exp(-(Jt[r] - beta) / P->lambda) / Z * epsc[((int64_t)r * T + h) * nu + j];
            U[h * nu + j] += acc;
        }

    /* Step 4: roll out the updated nominal and validate d_min >= d_safe. */
    double *u = (double *)malloc(sizeof(double) * (size_t)T * nu);
    double *st = (double *)malloc(sizeof(double) * (size_t)(T + 1) * 3);
    double *dn = (double *)malloc(sizeof(double) * (size_t)T);
    double *mv = vel ? (double *)malloc(sizeof(double) * (size_t)2 * (N > 0 ? N : 1)) : NULL;
    for (int h = 0; h < T; ++h)
        for (int j = 0; j < nu; ++j) u[h * nu + j] = clamp_dim(P, j, U[h * nu + j]);
    int chi_nom = 0, nn = 0;
    double Jn = sequence_cost(P, q0, u, cloud, vel, mv, mask, N, wp, W, kind, fp, n, st, dn, &chi_nom, &nn,
                              near_tol);
    if (J_nom) *J_nom = Jn;
    int ok = 1;
    for (int h = 0; h < T; ++h) if (!(dn[h] >= P->d_safe)) ok = 0;
    near_total += nn;
    if (dmin_nom) memcpy(dmin_nom, dn, sizeof(double) * (size_t)T);
    if (U_upd) memcpy(U_upd, U, sizeof(double) * (size_t)T * nu);

    if (ok) {
        for (int j = 0; j < nu; ++j) u_star[j] = U[j];
        for (int h = 0; h + 1 < T; ++h)
            for (int j = 0; j < nu; ++j) U[h * nu + j] = U[(h + 1) * nu + j];
        /* the last entry is repeated (shift-fill reading) */
    } else {
        for (int j = 0; j < nu; ++j) u_star[j] = 0.0;
        for (int k = 0; k < T * nu; ++k) U[k] = 0.0;
    }
    if (valid) *valid = ok;
    if (n_near) *n_near = near_total;
    free(u); free(st); free(dn); free(mv); free(epsc); free(Jt);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Hybrid-mode selection (Sec. IV-F, Algorithm 2, steps 1 and 2).  Every mode
 * m of the set has already run its own Algorithm 1 cycle, giving the cost
 * J[m] of its updated nominal and its validation flag valid[m].
 *   Jbar_m = J_m + lambda_switch * I(m != m_prev) if valid, else +inf;
 *   all +inf          -> safe stop: returns -1, *m_prev and *tau unchanged;
 *   m* = argmin Jbar  (the lowest mode index among equal values);
 *   tau > 0 and m* != m_prev -> m* = m_prev (cooldown; only when m_prev is a
 *                        mode of the set: m_prev = -1 means "none yet");
 *   tau = tau_max if m* != m_prev else max(tau - 1, 0);  m_prev = m*.
 * Jbar (M) receives the augmented costs when non-NULL.  Returns m*.
 * ------------------------------------------------------------------------- */
int ox_hybrid_select(int M, const double *J, const int *valid, double lambda_switch, int tau_max,
                     int *m_prev, int *tau, double *Jbar) {
    int best = -1;
    double best_J = INFINITY;
    for (int m = 0; m < M; ++m) {
        double jb = valid[m] ? J[m] + (m != *m_prev ? lambda_switch : 0.0) : INFINITY;
        if (Jbar) Jbar[m] = jb;
        if (jb < best_J) { best_J = jb; best = m; }
    }
    if (best < 0) return -1;
    int ms = best;
    if (*tau > 0 && ms != *m_prev && *m_prev >= 0 && *m_prev < M) ms = *m_prev;
    if (ms != *m_prev) *tau = tau_max;
    else *tau = *tau > 0 ? *tau - 1 : 0;
    *m_prev = ms;
    return ms;
}

/* ---------------------------------------------------------------------------
 * Polar nearest-range histogram (learned-proposal feature): obstacle points
 * moved into the robot frame at (x, y, th); bin = floor((atan2(py, px) + pi)
 * / (2 pi) * nbins), clamped to nbins - 1; value = min(r_max, min range).
 * ------------------------------------------------------------------------- */
void ox_polar_hist(const double *pts, const uint8_t *mask, int N, double x, double y,
                   double th, int nbins, double r_max, double *out) {
    for (int b = 0; b < nbins; ++b) out[b] = r_max;
    for (int i = 0; i < N; ++i) {
        if (mask && !mask[i]) continue;
        double px, py;
        ox_body_frame(pts[2 * i], pts[2 * i + 1], x, y, th, &px, &py);
        double r = sqrt(px * px + py * py);
        int b = (int)floor((atan2(py, px) + M_PI) / (2.0 * M_PI) * nbins);
        if (b < 0) b = 0;
        if (b > nbins - 1) b = nbins - 1;
        if (r < out[b]) out[b] = r;
    }
}

/* ---------------------------------------------------------------------------
 * Learned-proposal network input of one robot (project feature layout; the
 * paper has no learned component):
 *   [hist / r_max (nbins), goal in the robot frame / r_max (2),
 *    previous command (v, omega), |goal| / r_max, cos and sin of the goal
 *    bearing, previous nominal U (T x 2)].
 * The goal is moved into the robot frame as any obstacle point (Sec. IV-C.1);
 * the bearing is atan2 of its robot-frame coordinates (0 for a goal at the
 * robot's position).  out has nbins + 7 + 2 T entries.
 * ------------------------------------------------------------------------- */
void ox_proposal_features(const double *hist, int nbins, double r_max, double x, double y, double th,
                          double goal_x, double goal_y, const double *prev_cmd, const double *U_prev, int T,
                          double *out) {
    for (int k = 0; k < nbins; ++k) out[k] = hist[k] / r_max;
    double gx, gy;
    ox_body_frame(goal_x, goal_y, x, y, th, &gx, &gy);
    double range = sqrt(gx * gx + gy * gy);
    double bearing = atan2(gy, gx);
    out[nbins + 0] = gx / r_max;
    out[nbins + 1] = gy / r_max;
    out[nbins + 2] = prev_cmd[0];
    out[nbins + 3] = prev_cmd[1];
    out[nbins + 4] = range / r_max;
    out[nbins + 5] = cos(bearing);
    out[nbins + 6] = sin(bearing);
    for (int k = 0; k < 2 * T; ++k) out[nbins + 7 + k] = U_prev[k];
}

/* The two candidate nominals of a proposal-guided cycle: the proposal's
 * U_prev + shift and the plain U_prev (n entries each). */
void ox_proposal_prepare(const double *U_prev, const double *shift, int64_t n, double *U_prop, double *U_plain) {
    for (int64_t e = 0; e < n; ++e) {
        U_prop[e] = U_prev[e] + shift[e];
        U_plain[e] = U_prev[e];
    }
}

/* Fallback rule of the proposal-guided cycle for one robot: keep the
 * proposal candidate only when its best sample cost is strictly lower than
 * plain MPPI's (on a tie plain MPPI is kept); copy the kept candidate's
 * nominal (TN entries) and command (nu entries).  Returns 1 when the
 * proposal is kept. */
int ox_proposal_select(const double *costs_prop, const double *costs_plain, int K, const double *U_prop,
                       const double *U_plain, const double *u_prop, const double *u_plain, int TN, int nu,
                       double *U_out, double *u_out) {
    double best_prop = INFINITY, best_plain = INFINITY;
    for (int r = 0; r < K; ++r) {
        if (costs_prop[r] < best_prop) best_prop = costs_prop[r];
        if (costs_plain[r] < best_plain) best_plain = costs_plain[r];
    }
    int pick = best_prop < best_plain;
    for (int e = 0; e < TN; ++e) U_out[e] = pick ? U_prop[e] : U_plain[e];
    for (int j = 0; j < nu; ++j) u_out[j] = pick ? u_prop[j] : u_plain[j];
    return pick;
}

/* ---------------------------------------------------------------------------
 * Proposal MLP: y = W3 g(W2 g(W1 x + b1) + b2) + b3 with the exact GELU
 * g(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)).  Row-major weights:
 * W1 (H x D), W2 (H x H), W3 (O x H).  Batch rows are independent.
 * Loss = mean over batch and outputs of (y - target)^2.
 * ------------------------------------------------------------------------- */
static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_grad(double z) {
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
}

static void dense(const double *W, const double *b, const double *x, int in, int out, double *y) {
    for (int o = 0; o < out; ++o) {
        double acc = b[o];
        for (int i = 0; i < in; ++i) acc += W[(int64_t)o * in + i] * x[i];
        y[o] = acc;
    }
}

void ox_mlp_forward(const double *W1, const double *b1, const double *W2, const double *b2,
                    const double *W3, const double *b3, int D, int H, int O,
                    const double *x, int B, double *y) {
    #pragma omp parallel for schedule(static)
    for (int r = 0; r < B; ++r) {
        double *z1 = (double *)malloc(sizeof(double) * H * 2);
        double *z2 = z1 + H;
        dense(W1, b1, x + (int64_t)r * D, D, H, z1);
        for (int k = 0; k < H; ++k) z1[k] = gelu(z1[k]);
        dense(W2, b2, z1, H, H, z2);
        for (int k = 0; k < H; ++k) z2[k] = gelu(z2[k]);
        dense(W3, b3, z2, H, O, y + (int64_t)r * O);
        free(z1);
    }
}

/* Loss and analytic gradients by the chain rule (no reordering tricks). */
double ox_mlp_loss_grad(const double *W1, const double *b1, const double *W2, const double *b2,
                        const double *W3, const double *b3, int D, int H, int O,
                        const double *x, const double *tgt, int B,
                        double *gW1, double *gb1, double *gW2, double *gb2,
                        double *gW3, double *gb3) {
    memset(gW1, 0, sizeof(double) * (size_t)H * D); memset(gb1, 0, sizeof(double) * H);
    memset(gW2, 0, sizeof(double) * (size_t)H * H); memset(gb2, 0, sizeof(double) * H);
    memset(gW3, 0, sizeof(double) * (size_t)O * H); memset(gb3, 0, sizeof(double) * O);
    double *a1 = (double *)malloc(sizeof(double) * H), *h1 = (double *)malloc(sizeof(double) * H);
    double *a2 = (double *)malloc(sizeof(double) * H), *h2 = (double *)malloc(sizeof(double) * H);
    double *y = (double *)malloc(sizeof(double) * O), *dy = (double *)malloc(sizeof(double) * O);
    double *dh2 = (double *)malloc(sizeof(double) * H), *dh1 = (double *)malloc(sizeof(double) * H);
    double loss = 0.0, scale = 1.0 / ((double)B * O);
    for (int r = 0; r < B; ++r) {
        const double *xr = x + (int64_t)r * D;
        dense(W1, b1, xr, D, H, a1);
        for (int k = 0; k < H; ++k) h1[k] = gelu(a1[k]);
        dense(W2, b2, h1, H, H, a2);
        for (int k = 0; k < H; ++k) h2[k] = gelu(a2[k]);
        dense(W3, b3, h2, H, O, y);
        for (int o = 0; o < O; ++o) {
            double e = y[o] - tgt[(int64_t)r * O + o];
            loss += e * e * scale;
            dy[o] = 2.0 * e * scale;
        }
        for (int o = 0; o < O; ++o) {
            gb3[o] += dy[o];
            for (int k = 0; k < H; ++k) gW3[(int64_t)o * H + k] += dy[o] * h2[k];
        }
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int o = 0; o < O; ++o) s += W3[(int64_t)o * H + k] * dy[o];
            dh2[k] = s * gelu_grad(a2[k]);
        }
        for (int k = 0; k < H; ++k) {
            gb2[k] += dh2[k];
            for (int i = 0; i < H; ++i) gW2[(int64_t)k * H + i] += dh2[k] * h1[i];
        }
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int k = 0; k < H; ++k) s += W2[(int64_t)k * H + i] * dh2[k];
            dh1[i] = s * gelu_grad(a1[i]);
        }
        for (int i = 0; i < H; ++i) {
            gb1[i] += dh1[i];
            for (int d = 0; d < D; ++d) gW1[(int64_t)i * D + d] += dh1[i] * xr[d];
        }
    }
    free(a1); free(h1); free(a2); free(h2); free(y); free(dy); free(dh2); free(dh1);
    return loss;
}

/* Adam (Kingma & Ba 2015), step t >= 1, bias-corrected moments. */
void ox_adam_step(double *w, const double *g, double *m, double *v, int64_t n, int t,
                  double lr, double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int64_t k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        double mh = m[k] / c1, vh = v[k] / c2;
        w[k] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Signed distance of M body-frame points to one footprint (no transform). */
void ox_sdf_points(const double *pts, int64_t M, int kind, const double *fp, int n, double *out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) out[i] = ox_sdf(pts[2 * i], pts[2 * i + 1], kind, fp, n);
}

/* Ray-casting inside flag of M body-frame points (polygon only). */
void ox_inside_points(const double *pts, int64_t M, const double *v, int B, int32_t *out) {
    for (int64_t i = 0; i < M; ++i) out[i] = ox_inside_poly(pts[2 * i], pts[2 * i + 1], v, B);
}
