// internal.h -- host-side objects and dispatch shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"
#include "exact_mppi.h"

struct exact_footprint {
    int kind;    // exact_fp_kind
    int n;       // vertices or boxes given by the caller
    int n_pad;   // evaluator size the constants are padded to
    // polygon: per-edge constants (see exact::PolyC); rects: boxes
    float vx[EXACT_MAX_POLY_VERTICES], vy[EXACT_MAX_POLY_VERTICES];
    float exn[EXACT_MAX_POLY_VERTICES], eyn[EXACT_MAX_POLY_VERTICES];
    float ex[EXACT_MAX_POLY_VERTICES], ey[EXACT_MAX_POLY_VERTICES];
    float kx[EXACT_MAX_POLY_VERTICES];
    float cx[EXACT_MAX_RECTS], cy[EXACT_MAX_RECTS], sx[EXACT_MAX_RECTS], sy[EXACT_MAX_RECTS];
    float bcx, bcy, brad;   // bounding circle (body frame), radius rounded up
    float bhx, bhy;         // half extents of the bounding box about (bcx, bcy), rounded up
};

struct exact_ctx {
    int device = 0;
    int sm_count = 0;
    void *scratch = nullptr;     // growable device arena
    size_t scratch_bytes = 0;
    int *d_err = nullptr;        // device error word (exact_status)
    long long mppi_layout = -1;  // (K, T, parts) of the last mppi_step; -1 = arena reused otherwise
    bool stats = false;          // mppi_step also records cycle statistics
    exact_cycle_stats *d_stats = nullptr;   // device record of those statistics
};

namespace exact {

// Grow the context arena to at least `bytes` (synchronous when it grows).
int ensure_scratch(exact_ctx *ctx, size_t bytes);
int current_sm_count();
// Arena bytes needed by exact_sdf_batch (n_poses) and mppi_step (K, T).
size_t sdf_scratch_bytes(int n_poses);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The first kArenaHeader bytes of a context arena hold the MPPI cycle's
// control words at fixed offsets (they must survive calls of other shapes
// and other entry points); per-call arrays start after them.
constexpr size_t kArenaHeader = 256;
struct ArenaHeader {
    unsigned long long beta_enc;   // ~order(J~) of the best sample, via atomicMax; 0 = empty
    unsigned ticket[2];            // finished update / validation blocks
    int bad;                       // validation failed (written by the last validation block)
    unsigned long long vticket;    // validation blocks finished (low word) and failed (high word)
};
static_assert(sizeof(ArenaHeader) <= 64, "the batched step clears 64 bytes of control words per scene");

template <int E>
inline PolyC<E> make_poly(const exact_footprint *fp) {
    PolyC<E> P;
    // the same float in both lanes of a pair
    auto both = [](float f) {
        uint32_t u;
        memcpy(&u, &f, sizeof u);
        return ((unsigned long long)u << 32) | u;
    };
    for (int b = 0; b < E; ++b) {
        P.nvx[b] = both(-fp->vx[b]); P.nvy[b] = both(-fp->vy[b]);
        P.exn[b] = both(fp->exn[b]); P.eyn[b] = fp->eyn[b];
        P.nex[b] = both(-fp->ex[b]); P.ney[b] = both(-fp->ey[b]);
        P.nkx[b] = both(-fp->kx[b]);
    }
    P.bcx = fp->bcx; P.bcy = fp->bcy; P.brad = fp->brad;
    P.bhx = fp->bhx; P.bhy = fp->bhy;
    return P;
}

template <int R>
inline RectC<R> make_rect(const exact_footprint *fp) {
    RectC<R> Q;
    for (int j = 0; j < R; ++j) {
        Q.cx[j] = fp->cx[j]; Q.cy[j] = fp->cy[j]; Q.sx[j] = fp->sx[j]; Q.sy[j] = fp->sy[j];
        uint32_t ux, uy;
        const float mx = -fp->cx[j], my = -fp->cy[j];
        memcpy(&ux, &mx, 4); memcpy(&uy, &my, 4);
        Q.ncx[j] = ((unsigned long long)ux << 32) | ux; Q.ncy[j] = ((unsigned long long)uy << 32) | uy;
    }
    Q.bcx = fp->bcx; Q.bcy = fp->bcy; Q.brad = fp->brad;
    Q.bhx = fp->bhx; Q.bhy = fp->bhy;
    return Q;
}

// Calls f(constants) with the footprint's constant block of its padded size.
template <class F>
int with_footprint(const exact_footprint *fp, F &&f) {
    if (fp->kind == EXACT_FP_POLYGON) {
        switch (fp->n_pad) {
        case 4: return f(make_poly<4>(fp));
        case 6: return f(make_poly<6>(fp));
        case 8: return f(make_poly<8>(fp));
        case 10: return f(make_poly<10>(fp));
        case 12: return f(make_poly<12>(fp));
        case 14: return f(make_poly<14>(fp));
        case 16: return f(make_poly<16>(fp));
        case 24: return f(make_poly<24>(fp));
        case 32: return f(make_poly<32>(fp));
        case 40: return f(make_poly<40>(fp));
        case 48: return f(make_poly<48>(fp));
        case 56: return f(make_poly<56>(fp));
        case 64: return f(make_poly<64>(fp));
        default: return EXACT_EINVAL;
        }
    }
    switch (fp->n_pad) {
    case 1: return f(make_rect<1>(fp));
    case 2: return f(make_rect<2>(fp));
    case 3: return f(make_rect<3>(fp));
    case 4: return f(make_rect<4>(fp));
    case 5: return f(make_rect<5>(fp));
    case 6: return f(make_rect<6>(fp));
    case 7: return f(make_rect<7>(fp));
    case 8: return f(make_rect<8>(fp));
    default: return EXACT_EINVAL;
    }
}

// with_footprint for the footprints whose MPPI evaluator prunes point by
// point (rectangle covers, polygons of up to 16 edges); EXACT_EINVAL for any
// other.
template <class F>
int with_small_footprint(const exact_footprint *fp, F &&f) {
    if (fp->kind == EXACT_FP_POLYGON) {
        switch (fp->n_pad) {
        case 4: return f(make_poly<4>(fp));
        case 6: return f(make_poly<6>(fp));
        case 8: return f(make_poly<8>(fp));
        case 10: return f(make_poly<10>(fp));
        case 12: return f(make_poly<12>(fp));
        case 14: return f(make_poly<14>(fp));
        case 16: return f(make_poly<16>(fp));
        default: return EXACT_EINVAL;
        }
    }
    switch (fp->n_pad) {
    case 1: return f(make_rect<1>(fp));
    case 2: return f(make_rect<2>(fp));
    case 3: return f(make_rect<3>(fp));
    case 4: return f(make_rect<4>(fp));
    case 5: return f(make_rect<5>(fp));
    case 6: return f(make_rect<6>(fp));
    case 7: return f(make_rect<7>(fp));
    case 8: return f(make_rect<8>(fp));
    default: return EXACT_EINVAL;
    }
}

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? EXACT_OK : EXACT_ECUDA; }

}  // namespace exact
