// mppi_common.cuh -- device pieces of the MPPI control cycle shared by the
// single-scene and batched kernels: kinematics, warp-parallel Euler rollout,
// guidance distance and the obstacle penalty.
#pragma once

#include "common.cuh"

namespace exact {

constexpr int kMaxPerLane = (EXACT_MAX_HORIZON + 31) / 32;   // rollout steps held by one lane

// Device copy of the cycle parameters (float, as on the boundary).
struct MppiP {
    int K, T, nu, model;
    float dt, lambda, d_safe, w_coll, w_rep, w_inf, w_goal, w_term, w_ctrl, wheelbase;
    float u_min[3], u_max[3];
    int clamp, state_offset;
};

// Sec. III-D kinematics: heading rate (independent of the state for every
// model) and the planar velocity at heading (c, s).
__device__ __forceinline__ float heading_rate(int model, float L, float u0, float u1, float u2) {
    switch (model) {
    case EXACT_MM_DIFF: return u1;
    case EXACT_MM_ACKERMANN: return u0 / L * tanf(u1);
    case EXACT_MM_OMNI: return u2;
    case EXACT_MM_SPIN: return u0;
    default: return 0.f;
    }
}
__device__ __forceinline__ void planar_velocity(int model, float c, float s, float u0, float u1,
                                                float &fx, float &fy) {
    switch (model) {
    case EXACT_MM_DIFF:
    case EXACT_MM_ACKERMANN: fx = u0 * c; fy = u0 * s; break;
    case EXACT_MM_OMNI: fx = fmaf(u0, c, -(u1 * s)); fy = fmaf(u0, s, u1 * c); break;
    case EXACT_MM_PARALLEL: fx = -(u0 * s); fy = u0 * c; break;
    default: fx = 0.f; fy = 0.f; break;
    }
}

__device__ __forceinline__ float clamp_u(const MppiP &P, int j, float v) {
    return P.clamp ? fminf(fmaxf(v, P.u_min[j]), P.u_max[j]) : v;
}

__device__ __forceinline__ float warp_incl_scan(float v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Distance from (x, y) to the guidance: one goal point or the nearest point
// of the waypoint polyline (task-cost reading).
__device__ __forceinline__ float guidance_dist(float x, float y, const float *__restrict__ wp, int W) {
    if (W == 1) {
        const float dx = x - wp[0], dy = y - wp[1];
        return sqrtf(fmaf(dx, dx, dy * dy));
    }
    float best = finf();
    for (int k = 0; k + 1 < W; ++k) {
        const float vx = wp[2 * k], vy = wp[2 * k + 1];
        const float ex = wp[2 * k + 2] - vx, ey = wp[2 * k + 3] - vy;
        const float dx = x - vx, dy = y - vy;
        const float len2 = fmaf(ex, ex, ey * ey);
        const float t = len2 > 0.f ? __saturatef(fmaf(dx, ex, dy * ey) / len2) : 0.f;
        const float qx = fmaf(-t, ex, dx), qy = fmaf(-t, ey, dy);
        best = fminf(best, fmaf(qx, qx, qy * qy));
    }
    return sqrtf(best);
}

// Warp-parallel forward-Euler rollout (Sec. III-D).  Lane l holds steps
// h = l*per .. l*per+per-1 (blocked).  Because the heading rate depends only
// on the control, theta_h is a prefix sum of rate*dt, and x, y are prefix
// sums of the planar velocity at the old heading theta_h times dt.
// ufetch(h, j) returns the (clamped) control.  Outputs per held step: the
// scored state s_h (q_{h+1} or q_h), the control, and on every lane the
// terminal state q_T.
struct LaneRollout {
    float x[kMaxPerLane], y[kMaxPerLane], th[kMaxPerLane];
    float u[kMaxPerLane][3];
    float qTx, qTy, qTth;
    int per;
};

template <class UF>
__device__ __forceinline__ void warp_rollout(const MppiP &P, float x0, float y0, float th0, UF ufetch,
                                             LaneRollout &R) {
    const int lane = threadIdx.x & 31;
    const int T = P.T;
    const int per = (T + 31) >> 5;
    R.per = per;
    const int base = lane * per;
    float rate[kMaxPerLane];
    float tot = 0.f;
    // elements e >= per (warp-uniform) hold no step: their work is skipped
#pragma unroll
    for (int e = 0; e < kMaxPerLane; ++e) {
        const int h = base + e;
        const bool ok = e < per && h < T;
        rate[e] = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) R.u[e][j] = 0.f;
        if (e < per) {
#pragma unroll
            for (int j = 0; j < 3; ++j) R.u[e][j] = (ok && j < P.nu) ? ufetch(h, j) : 0.f;
            rate[e] = ok ? heading_rate(P.model, P.wheelbase, R.u[e][0], R.u[e][1], R.u[e][2]) * P.dt : 0.f;
        }
        tot += rate[e];
    }
    // theta_h (before step h): exclusive prefix over all steps
    const float incl = warp_incl_scan(tot);
    float run = incl - tot;
    float thb[kMaxPerLane], fx[kMaxPerLane], fy[kMaxPerLane];
    float tx = 0.f, ty = 0.f;
#pragma unroll
    for (int e = 0; e < kMaxPerLane; ++e) {
        thb[e] = th0 + run;
        run += rate[e];
        fx[e] = fy[e] = 0.f;
        if (e < per) {
            float sn, cs;
            sincosf(thb[e], &sn, &cs);
            planar_velocity(P.model, cs, sn, R.u[e][0], R.u[e][1], fx[e], fy[e]);
            const bool ok = base + e < T;
            fx[e] = ok ? fx[e] * P.dt : 0.f;
            fy[e] = ok ? fy[e] * P.dt : 0.f;
        }
        tx += fx[e];
        ty += fy[e];
    }
    const float ix = warp_incl_scan(tx), iy = warp_incl_scan(ty);
    float rx = ix - tx, ry = iy - ty;
    float rth = incl - tot;
#pragma unroll
    for (int e = 0; e < kMaxPerLane; ++e) {
        if (P.state_offset) {
            rx += fx[e]; ry += fy[e]; rth += rate[e];
            R.x[e] = x0 + rx; R.y[e] = y0 + ry; R.th[e] = th0 + rth;
        } else {
            R.x[e] = x0 + rx; R.y[e] = y0 + ry; R.th[e] = thb[e];
            rx += fx[e]; ry += fy[e];
        }
    }
    R.qTx = x0 + __shfl_sync(0xffffffffu, ix, 31);
    R.qTy = y0 + __shfl_sync(0xffffffffu, iy, 31);
    R.qTth = th0 + __shfl_sync(0xffffffffu, incl, 31);
}

}  // namespace exact
