// common.cuh -- device building blocks shared by the EXACT-MPPI kernels.
//
// Footprint constants travel as kernel parameters (constant bank), so every
// edge / box term of the fully unrolled evaluators is an immediate constant
// operand: no shared-memory or global loads inside the hot loops.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "exact_mppi.h"

namespace exact {

constexpr int kBlock = 256;                 // threads per block of the SDF / MPPI kernels
constexpr unsigned long long kNoKey = ~0ull;

__device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

// Polygon footprint (Sec. IV-B.2) padded to E edges.  Padding vertices repeat
// vertex 0, which adds zero-length edges: their clipped projection is 0 (the
// distance to a vertex already covered) and both ends lie at the same height,
// so they never toggle the crossing parity.
template <int E>
struct PolyC {
    float vx[E], vy[E];     // vertices v_b
    float exn[E], eyn[E];   // e_b / |e_b|^2   (0 for a zero-length edge)
    float ex[E], ey[E];     // e_b = v_{b+1} - v_b
    float kx[E];            // e_bx / e_by      (0 when e_by == 0)
    float bcx, bcy, brad;   // bounding circle: centre, radius (rounded up)
};

// Rectangle cover (Sec. IV-B.1) padded to R boxes by repeating box 0.
template <int R>
struct RectC {
    float cx[R], cy[R], sx[R], sy[R];
    float bcx, bcy, brad;   // bounding circle: centre, radius (rounded up)
};

// ---------------------------------------------------------------- transform
// Sec. IV-C.1: p = R(theta)^T (o - t) = (c dx + s dy, -s dx + c dy).
__device__ __forceinline__ void body_frame(float ox, float oy, float tx, float ty, float c, float s,
                                           float &px, float &py) {
    const float dx = ox - tx, dy = oy - ty;
    px = fmaf(c, dx, s * dy);
    py = fmaf(c, dy, -(s * dx));
}

// ---------------------------------------------------------------- polygon
// Sec. IV-C.3 for two independent body-frame points.  Returns the squared
// unsigned distance min_b d_seg,b^2 in m* and the crossing parity in the
// sign bit of s*.
//
// Distance: alpha = sat(d . e / |e|^2), q = d - alpha e, d_seg^2 = |q|^2 with
// d = p - v_b.  Sign: the ray from p towards +x crosses edge b when the two
// end heights straddle p_y and the crossing lies right of p.  With
// dy_b = p_y - v_by, "v_b above p" is the sign bit of dy_b, so the straddle
// is the sign bit of dy_b * dy_{b+1}; the crossing abscissa test
// p_x < v_bx + dy_b e_bx / e_by is the sign of g = dy_b k_b - dx_b being
// clear.  Both ends of a vertex use the same dy, so the parity is consistent.
// Three-input minimum (one instruction on sm_100-class GPUs).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

struct PolyAcc {
    float dxa0, dya0, dxa1, dya1;   // p - v_b for the two points
    float mm0, mm1;                 // running min of d_seg^2
    unsigned ss0, ss1;              // crossing parity (sign bit)
};

// Edge B (a compile-time index, so every footprint term is an immediate
// constant-bank operand) for both points; returns the two squared segment
// distances and advances the vertex differences to v_{B+1}.
template <int E, int B>
__device__ __forceinline__ void poly_edge(const PolyC<E> &P, float px0, float py0, float px1, float py1,
                                          const PolyAcc &z, PolyAcc &a, float &q0, float &q1) {
    float dxb0, dyb0, dxb1, dyb1;
    if constexpr (B + 1 < E) {
        dxb0 = px0 - P.vx[B + 1]; dyb0 = py0 - P.vy[B + 1];
        dxb1 = px1 - P.vx[B + 1]; dyb1 = py1 - P.vy[B + 1];
    } else {
        dxb0 = z.dxa0; dyb0 = z.dya0; dxb1 = z.dxa1; dyb1 = z.dya1;
    }
    const float t0 = __saturatef(fmaf(a.dya0, P.eyn[B], a.dxa0 * P.exn[B]));
    const float t1 = __saturatef(fmaf(a.dya1, P.eyn[B], a.dxa1 * P.exn[B]));
    const float qx0 = fmaf(-t0, P.ex[B], a.dxa0), qy0 = fmaf(-t0, P.ey[B], a.dya0);
    const float qx1 = fmaf(-t1, P.ex[B], a.dxa1), qy1 = fmaf(-t1, P.ey[B], a.dya1);
    q0 = fmaf(qy0, qy0, qx0 * qx0);
    q1 = fmaf(qy1, qy1, qx1 * qx1);
    const float g0 = fmaf(a.dya0, P.kx[B], -a.dxa0), g1 = fmaf(a.dya1, P.kx[B], -a.dxa1);
    const float X0 = a.dya0 * dyb0, X1 = a.dya1 * dyb1;
    a.ss0 ^= __float_as_uint(X0) & ~__float_as_uint(g0);
    a.ss1 ^= __float_as_uint(X1) & ~__float_as_uint(g1);
    a.dxa0 = dxb0; a.dya0 = dyb0; a.dxa1 = dxb1; a.dya1 = dyb1;
}

// Edges B and B+1 (E is even), folded into the running minimum with one
// three-input min per point; recursion unrolls all E edges.
template <int E, int B>
__device__ __forceinline__ void poly_edges(const PolyC<E> &P, float px0, float py0, float px1, float py1,
                                           const PolyAcc &z, PolyAcc &a) {
    if constexpr (B < E) {
        float qa0, qa1, qb0, qb1;
        poly_edge<E, B>(P, px0, py0, px1, py1, z, a, qa0, qa1);
        poly_edge<E, B + 1>(P, px0, py0, px1, py1, z, a, qb0, qb1);
        a.mm0 = fmin3(a.mm0, qa0, qb0);
        a.mm1 = fmin3(a.mm1, qa1, qb1);
        poly_edges<E, B + 2>(P, px0, py0, px1, py1, z, a);
    }
}

template <int E>
__device__ __forceinline__ void poly_eval2(const PolyC<E> &P, float px0, float py0, float px1, float py1,
                                           float &m0, float &m1, unsigned &s0, unsigned &s1) {
    static_assert(E % 2 == 0, "edge count is padded to an even number");
    PolyAcc z;
    z.dxa0 = px0 - P.vx[0]; z.dya0 = py0 - P.vy[0];
    z.dxa1 = px1 - P.vx[0]; z.dya1 = py1 - P.vy[0];
    z.mm0 = z.mm1 = finf();
    z.ss0 = z.ss1 = 0u;
    PolyAcc a = z;
    poly_edges<E, 0>(P, px0, py0, px1, py1, z, a);
    m0 = a.mm0; m1 = a.mm1; s0 = a.ss0; s1 = a.ss1;
}

// ---------------------------------------------------------------- rect cover
// Sec. IV-C.2: d_box = |max(a,0)| + min(max(a_x,a_y),0), a = |p - c| - s, and
// d_rect = min_j d_box.  For every box one of the two terms is zero, so
// min_j d_box = sqrt(min_j |max(a_j,0)|^2) + min(min_j max(a_jx,a_jy), 0)
// exactly (sqrt is correctly rounded, hence monotone).  The clamp is taken
// as a + |a| = 2 max(a, 0) (an add with an absolute-value operand, exact),
// so the evaluator tracks 4 |max(a,0)|^2 and halves the root at the end:
// both scalings by powers of two are exact.
template <int R, int J>
__device__ __forceinline__ void rect_box(const RectC<R> &Q, float px, float py, float &n4, float &mx2) {
    const float ax = fabsf(px - Q.cx[J]) - Q.sx[J];
    const float ay = fabsf(py - Q.cy[J]) - Q.sy[J];
    const float ux = ax + fabsf(ax), uy = ay + fabsf(ay);
    n4 = fmaf(uy, uy, ux * ux);
    mx2 = fmaxf(ax, ay);
}

template <int R, int J>
__device__ __forceinline__ void rect_boxes(const RectC<R> &Q, float px, float py, float &nn, float &in) {
    if constexpr (J + 1 < R) {
        float na, ia, nb, ib;
        rect_box<R, J>(Q, px, py, na, ia);
        rect_box<R, J + 1>(Q, px, py, nb, ib);
        nn = fmin3(nn, na, nb);
        in = fmin3(in, ia, ib);
        rect_boxes<R, J + 2>(Q, px, py, nn, in);
    } else if constexpr (J < R) {
        float na, ia;
        rect_box<R, J>(Q, px, py, na, ia);
        nn = fminf(nn, na);
        in = fminf(in, ia);
    }
}

// n4 = min_j 4 |max(a_j, 0)|^2, inner = min_j max(a_jx, a_jy).
template <int R>
__device__ __forceinline__ void rect_eval(const RectC<R> &Q, float px, float py, float &n4, float &inner) {
    float nn = finf(), in = finf();
    rect_boxes<R, 0>(Q, px, py, nn, in);
    n4 = nn;
    inner = in;
}
// Mixed key: the (negative) depth inside, 4 x the squared distance outside.
__device__ __forceinline__ float rect_key(float n4, float inner) { return inner < 0.f ? inner : n4; }
__device__ __forceinline__ float rect_key_to_dist(float key) { return key < 0.f ? key : 0.5f * sqrtf(key); }

// ---------------------------------------------------------------- keys
// Order-preserving float <-> uint32 map (total order, -0 < +0).
__device__ __forceinline__ unsigned f2ord(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ unsigned long long pack_key(float key, unsigned idx) {
    return ((unsigned long long)f2ord(key) << 32) | idx;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace exact

namespace exact {

// Uniform evaluation interface over the two footprint kinds.  For two
// body-frame points it yields the order key (monotone in the signed
// distance: the signed squared distance for polygons, the signed depth or
// squared distance for rectangle covers) and, when asked, the signed
// distance itself.  key_to_dist maps a key back to the same distance.
template <int E>
__device__ __forceinline__ void eval2(const PolyC<E> &P, float px0, float py0, float px1, float py1,
                                      float &k0, float &k1) {
    float m0, m1;
    unsigned s0, s1;
    poly_eval2(P, px0, py0, px1, py1, m0, m1, s0, s1);
    k0 = __uint_as_float(__float_as_uint(m0) | (s0 & 0x80000000u));
    k1 = __uint_as_float(__float_as_uint(m1) | (s1 & 0x80000000u));
}
template <int R>
__device__ __forceinline__ void eval2(const RectC<R> &Q, float px0, float py0, float px1, float py1,
                                      float &k0, float &k1) {
    float n0, i0, n1, i1;
    rect_eval(Q, px0, py0, n0, i0);
    rect_eval(Q, px1, py1, n1, i1);
    k0 = rect_key(n0, i0);
    k1 = rect_key(n1, i1);
}
// Signed squared distance key -> signed distance (sign bit carried over).
template <int E>
__device__ __forceinline__ float key_to_dist(const PolyC<E> &, float key) {
    const unsigned b = __float_as_uint(key);
    return __uint_as_float(__float_as_uint(sqrtf(__uint_as_float(b & 0x7fffffffu))) | (b & 0x80000000u));
}
template <int R>
__device__ __forceinline__ float key_to_dist(const RectC<R> &, float key) { return rect_key_to_dist(key); }

template <class FPC> struct fp_traits;
template <int E> struct fp_traits<PolyC<E>> {
    static constexpr int kind = EXACT_FP_POLYGON;
    static constexpr int size = E;
};
template <int R> struct fp_traits<RectC<R>> {
    static constexpr int kind = EXACT_FP_RECTS;
    static constexpr int size = R;
};

}  // namespace exact
