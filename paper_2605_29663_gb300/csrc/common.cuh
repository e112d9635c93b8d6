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

// ---------------------------------------------------------------- device errors
// A context (or batch) error word: the first nonzero exact_status a kernel
// records stays until the host reads and clears it.  err may be NULL (no word).
__device__ __forceinline__ void report_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}
// Index checks of the debug build (-DEXACT_DEBUG_CHECKS): a failed check
// records EXACT_ECAPACITY and the caller skips the access.  In the release
// build the condition is not evaluated.
#ifdef EXACT_DEBUG_CHECKS
#define EXACT_DCHECK(cond, err) ((cond) ? true : (::exact::report_error((err), EXACT_ECAPACITY), false))
#else
#define EXACT_DCHECK(cond, err) true
#endif

// ---------------------------------------------------------------- async copies
// Bulk copies global -> shared memory on the TMA engine, completed on an
// mbarrier (transaction bytes), and 8-byte cp.async copies (no register round
// trip).  An mbarrier is initialised once per kernel and its phases are
// counted; a wait on a phase is bounded by kWaitNs of wall time, after which
// it reports EXACT_ETIMEOUT and gives up.
constexpr unsigned long long kWaitNs = 20ull * 1000 * 1000;   // 20 ms

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive on the barrier announcing `bytes` of transactions for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of phase `parity`; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}
// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned
// shared dst, completing as transaction bytes on bar.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Two FP32 lanes in one 64-bit register pair, for the packed f32x2
// arithmetic of sm_100-class GPUs: one instruction does the same IEEE
// round-to-nearest operation on both lanes, so a packed chain gives the
// bits of the scalar chain it replaces while taking half the issue slots.
typedef unsigned long long f2x;

// Polygon footprint (Sec. IV-B.2) padded to E edges.  Padding vertices repeat
// vertex 0, which adds zero-length edges: their clipped projection is 0 (the
// distance to a vertex already covered) and both ends lie at the same height,
// so they never toggle the crossing parity.  The edge terms are stored as
// lane pairs (the same value in both lanes) for the packed evaluator, with
// the signs folded in so that every step is an add, multiply or fma.
template <int E>
struct PolyC {
    f2x nvx[E], nvy[E];     // -v_b
    f2x exn[E];             // e_bx / |e_b|^2   (0 for a zero-length edge)
    f2x nex[E], ney[E];     // -e_b,  e_b = v_{b+1} - v_b
    f2x nkx[E];             // -e_bx / e_by     (0 when e_by == 0)
    float eyn[E];           // e_by / |e_b|^2   (scalar: its fma saturates)
    float bcx, bcy, brad;   // bounding circle: centre, radius (rounded up)
    float bhx, bhy;         // bounding box about (bcx, bcy): half extents (rounded up)
};

// Rectangle cover (Sec. IV-B.1) padded to R boxes by repeating box 0.
template <int R>
struct RectC {
    f2x ncx[R], ncy[R];     // -c pairs
    float cx[R], cy[R], sx[R], sy[R];
    float bcx, bcy, brad;   // bounding circle: centre, radius (rounded up)
    float bhx, bhy;         // bounding box about (bcx, bcy): half extents (rounded up)
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
// Sec. IV-C.3 for two body-frame points, one per lane.  Returns the squared
// unsigned distance min_b d_seg,b^2 in m* and the crossing parity in the
// sign bit of s*.
//
// Distance: alpha = sat(d . e / |e|^2), q = d - alpha e, d_seg^2 = |q|^2 with
// d = p - v_b.  Sign: the ray from p towards +x crosses edge b when the two
// end heights straddle p_y and the crossing lies right of p.  With
// dy_b = p_y - v_by, "v_b above p" is the sign bit of dy_b, so the straddle
// is the sign bit of dy_b * dy_{b+1}; the crossing abscissa test
// p_x < v_bx + dy_b e_bx / e_by holds when h = dx_b - dy_b k_b is negative
// (k_b = e_bx / e_by), i.e. when the sign bit of h is set.  Both ends of a
// vertex use the same dy, so every crossing is counted once.  A point exactly
// on the crossing abscissa (h = 0) lies on the boundary, where either sign
// is the exact distance 0.
// Three-input minimum (one instruction on sm_100-class GPUs).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ f2x pack2(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f2x v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

struct PolyAcc {
    f2x dxa, dya;           // p - v_b for the two points
    float mm0, mm1;         // running min of d_seg^2
    unsigned ss0, ss1;      // crossing parity (sign bit)
};

// What an edge pass computes: the squared segment distances (kDist), the
// crossing parity (kSign), or both.
constexpr int kDist = 1, kSign = 2;

// Edge B (a compile-time index, so every footprint term is a constant-bank
// operand) for both points; returns the two squared segment distances and
// advances the vertex differences to v_{B+1}.  Only the clipped projection
// runs per lane: f32x2 has no saturating form.
template <int E, int B, int PART>
__device__ __forceinline__ void poly_edge(const PolyC<E> &P, f2x PX, f2x PY, const PolyAcc &z, PolyAcc &a,
                                          float &q0, float &q1) {
    f2x dxb, dyb;
    if constexpr (B + 1 < E) {
        if constexpr (PART & kDist) dxb = add2(PX, P.nvx[B + 1]);
        dyb = add2(PY, P.nvy[B + 1]);
    } else {
        dxb = z.dxa;
        dyb = z.dya;
    }
    if constexpr (PART & kDist) {
        float u0, u1, dy0, dy1;
        unpack2(mul2(a.dxa, P.exn[B]), u0, u1);
        unpack2(a.dya, dy0, dy1);
        const f2x t = pack2(__saturatef(fmaf(dy0, P.eyn[B], u0)), __saturatef(fmaf(dy1, P.eyn[B], u1)));
        const f2x qx = fma2(t, P.nex[B], a.dxa), qy = fma2(t, P.ney[B], a.dya);
        unpack2(fma2(qy, qy, mul2(qx, qx)), q0, q1);
    }
    if constexpr (PART & kSign) {
        if constexpr (!(PART & kDist) && B + 1 < E) dxb = add2(PX, P.nvx[B + 1]);
        float h0, h1, x0, x1;
        unpack2(fma2(a.dya, P.nkx[B], a.dxa), h0, h1);
        unpack2(mul2(a.dya, dyb), x0, x1);
        a.ss0 ^= __float_as_uint(x0) & __float_as_uint(h0);
        a.ss1 ^= __float_as_uint(x1) & __float_as_uint(h1);
    }
    a.dxa = dxb;
    a.dya = dyb;
}

// Edges B and B+1 (E is even), folded into the running minimum with one
// three-input min per point; recursion unrolls all E edges.
template <int E, int B, int PART>
__device__ __forceinline__ void poly_edges(const PolyC<E> &P, f2x PX, f2x PY, const PolyAcc &z, PolyAcc &a) {
    if constexpr (B < E) {
        float qa0, qa1, qb0, qb1;
        poly_edge<E, B, PART>(P, PX, PY, z, a, qa0, qa1);
        poly_edge<E, B + 1, PART>(P, PX, PY, z, a, qb0, qb1);
        if constexpr (PART & kDist) {
            a.mm0 = fmin3(a.mm0, qa0, qb0);
            a.mm1 = fmin3(a.mm1, qa1, qb1);
        }
        poly_edges<E, B + 2, PART>(P, PX, PY, z, a);
    }
}

// The parts PART of the evaluation for two points: each part takes the same
// operations as in the full evaluation, so its results are the same bits.
template <int E, int PART = kDist | kSign>
__device__ __forceinline__ void poly_eval2(const PolyC<E> &P, float px0, float py0, float px1, float py1,
                                           float &m0, float &m1, unsigned &s0, unsigned &s1) {
    static_assert(E % 2 == 0, "edge count is padded to an even number");
    const f2x PX = pack2(px0, px1), PY = pack2(py0, py1);
    PolyAcc z;
    z.dxa = add2(PX, P.nvx[0]);
    z.dya = add2(PY, P.nvy[0]);
    z.mm0 = z.mm1 = finf();
    z.ss0 = z.ss1 = 0u;
    PolyAcc a = z;
    poly_edges<E, 0, PART>(P, PX, PY, z, a);
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
// Box J for two points, one per f32x2 lane (the differences and the squared
// norm packed, the absolute values per lane: f32x2 has no absolute-value
// form).  PART kDist: 4 |max(a,0)|^2 in n*; kSign: max(a_x, a_y) in m*.
template <int R, int J, int PART>
__device__ __forceinline__ void rect_box2(const RectC<R> &Q, f2x PX, f2x PY, float &n0, float &n1, float &m0,
                                          float &m1) {
    float dx0, dx1, dy0, dy1;
    unpack2(add2(PX, Q.ncx[J]), dx0, dx1);
    unpack2(add2(PY, Q.ncy[J]), dy0, dy1);
    const float ax0 = fabsf(dx0) - Q.sx[J], ay0 = fabsf(dy0) - Q.sy[J];
    const float ax1 = fabsf(dx1) - Q.sx[J], ay1 = fabsf(dy1) - Q.sy[J];
    if constexpr (PART & kDist) {
        const f2x UX = pack2(ax0 + fabsf(ax0), ax1 + fabsf(ax1)), UY = pack2(ay0 + fabsf(ay0), ay1 + fabsf(ay1));
        unpack2(fma2(UY, UY, mul2(UX, UX)), n0, n1);
    }
    if constexpr (PART & kSign) {
        m0 = fmaxf(ax0, ay0);
        m1 = fmaxf(ax1, ay1);
    }
}

// All boxes, folded with three-input minima into n = min_j 4 |max(a_j,0)|^2
// (kDist) and inner = min_j max(a_jx, a_jy) (kSign).
template <int R, int J, int PART>
__device__ __forceinline__ void rect_boxes2(const RectC<R> &Q, f2x PX, f2x PY, float &nn0, float &nn1, float &in0,
                                            float &in1) {
    if constexpr (J + 1 < R) {
        float na0, na1, ia0, ia1, nb0, nb1, ib0, ib1;
        rect_box2<R, J, PART>(Q, PX, PY, na0, na1, ia0, ia1);
        rect_box2<R, J + 1, PART>(Q, PX, PY, nb0, nb1, ib0, ib1);
        if constexpr (PART & kDist) { nn0 = fmin3(nn0, na0, nb0); nn1 = fmin3(nn1, na1, nb1); }
        if constexpr (PART & kSign) { in0 = fmin3(in0, ia0, ib0); in1 = fmin3(in1, ia1, ib1); }
        rect_boxes2<R, J + 2, PART>(Q, PX, PY, nn0, nn1, in0, in1);
    } else if constexpr (J < R) {
        float na0, na1, ia0, ia1;
        rect_box2<R, J, PART>(Q, PX, PY, na0, na1, ia0, ia1);
        if constexpr (PART & kDist) { nn0 = fminf(nn0, na0); nn1 = fminf(nn1, na1); }
        if constexpr (PART & kSign) { in0 = fminf(in0, ia0); in1 = fminf(in1, ia1); }
    }
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
    float n0 = finf(), n1 = finf(), i0 = finf(), i1 = finf();
    rect_boxes2<R, 0, kDist | kSign>(Q, pack2(px0, px1), pack2(py0, py1), n0, n1, i0, i1);
    k0 = rect_key(n0, i0);
    k1 = rect_key(n1, i1);
}
// The same keys with the depth pass taken only where it can decide: for a
// point in (or on) some box the outside norm n is 0 (NaN for a non-finite
// point); elsewhere every box has max(a_x, a_y) > 0 and the key is n.  Pays
// where the ALU pipe is the bound (the MPPI sample phase), not in the full
// matrix, where the extra branch costs more than the depth terms.
template <int R>
__device__ __forceinline__ void eval2_lazy_depth(const RectC<R> &Q, float px0, float py0, float px1, float py1,
                                                 float &k0, float &k1) {
    const f2x PX = pack2(px0, px1), PY = pack2(py0, py1);
    float n0 = finf(), n1 = finf(), i0 = finf(), i1 = finf();
    rect_boxes2<R, 0, kDist>(Q, PX, PY, n0, n1, i0, i1);
    k0 = n0;
    k1 = n1;
    if (!(n0 > 0.f) || !(n1 > 0.f)) {
        rect_boxes2<R, 0, kSign>(Q, PX, PY, n0, n1, i0, i1);
        k0 = rect_key(n0, i0);
        k1 = rect_key(n1, i1);
    }
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
