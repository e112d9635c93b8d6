// mppi_cycle.cuh -- the three phases of one control cycle (Algorithm 1) as
// block-level device bodies, shared by the single-scene kernels (mppi.cu)
// and the batched persistent kernels (batched.cu):
//   sample_body    one sample r: rollout, every (step, point) body-frame
//                  signed distance, per-step minima, J~ (Sec. III-E, IV-C..E);
//                  when no d_min output is wanted, points that cannot come
//                  within d_safe of the footprint are skipped (sub-chunk
//                  circles, then the footprint's bounding box per point or
//                  per 16-point fine sub-chunk; per-point circles for small
//                  clouds)
//   update_body    one chunk of samples: weights and weighted clipped noise
//                  into a partial slot (Alg. 1 step 3)
//   validate_body  one (step, point chunk) of the nominal: adds the partial
//                  slots (U_upd), rolls the nominal out, d_min >= d_safe;
//                  the scene's last block writes u*, the shifted or reset U
//                  and the valid flag (Alg. 1 step 4), and the nominal's
//                  cost when asked (the J_m of Alg. 2)
// Blocks never wait for each other: the last block of a phase is found with
// an atomic ticket.  A footprint is reached through an evaluator object that
// provides eval2 (two points -> two order keys) and dist (key -> signed
// distance), either with compile-time constants or from shared memory.
#pragma once

#include "internal.h"
#include "mppi_common.cuh"

namespace exact {

constexpr int kUpdBlock = 256;
constexpr int kUpdTile = 8192;    // floats of noise one update block stages (32 KB)
constexpr int kStage = 4096;      // obstacle points staged in shared memory per pass
// Points per pass for static (float2 position) or predicted (float4
// position + velocity) clouds: both fill the same 32 KB of shared memory.
template <bool MOVING>
__host__ __device__ constexpr int stage_points_of() { return MOVING ? kStage / 2 : kStage; }
constexpr int kValChunkPairs = 1024;

// Everything the phases need about one scene.
struct SceneView {
    MppiP P;
    const float *state;
    const float2 *pts;
    const float2 *vel;  // N point velocities (time-indexed prediction), or NULL: static points
    const uint8_t *mask;
    int N;
    const float *wp;
    int W;
    float *U;
    const float *noise;
    float *u_star, *costs, *weights, *U_upd_out, *dmin;
    float *nom_cost;    // 1 or NULL: cost J of the updated nominal
    int *valid;
    int *err;           // device error word (exact_status; first error kept), or NULL
    ArenaHeader *hdr;   // beta, tickets, validation flag
    double *Jt;         // K   J~ = J + w_inf I(chi)
    float *wt;          // K   unnormalised weights
    float *part;        // G x (T*nu + 1) partial sums
    unsigned *dkey;     // K x T  per-step keys exchanged between horizon parts
    unsigned *tk;       // K      finished horizon parts of each sample
    unsigned *vkey;     // T      nominal's per-step minimum key (complemented order key; 0 = empty)
    int upd_chunk, upd_blocks, val_chunks;
    int parts;          // blocks per sample (horizon split); 1 = one block per sample
};

// samples per update block: the block's noise tile fits kUpdTile floats,
// and K is spread over about 64 blocks (at least 8 samples each) so that
// the tiles load in parallel
inline int upd_chunk_for(int K, int T, int nu) {
    int c = kUpdTile / (T * nu);
    if (c > 256) c = 256;
    int spread = (K + 63) / 64;
    if (spread < 8) spread = 8;
    if (c > spread) c = spread;
    return c < 1 ? 1 : c;
}
inline int upd_blocks_for(int K, int T, int nu) {
    const int c = upd_chunk_for(K, T, nu);
    return (K + c - 1) / c;
}

// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialization attribute may start while its predecessor on
// the stream drains; grid_dep_wait blocks until the predecessor has
// completed and its writes are visible (a no-op without the attribute).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with the programmatic-serialization attribute (see grid_dep_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

inline int val_chunks_for(int N) {
    const int np = (N + 1) / 2;
    return np > kValChunkPairs ? (np + kValChunkPairs - 1) / kValChunkPairs : 1;
}

// Blocks per sample: split the horizon when there are too few samples to
// fill the GPU (about `target` blocks), at most 8 parts and one step each.
// Two samples per sample block (see sample_body) when the scene has enough
// samples to fill the GPU at half the blocks (K >= 4 per SM) and both
// horizons fit the block's step slots; never with a split horizon.
inline int pair_samples(int K, int T, int parts, int sms) {
    return parts == 1 && 2 * T <= EXACT_MAX_HORIZON && K >= 4 * (sms > 0 ? sms : 148) ? 1 : 0;
}

inline int parts_for(int K, int T, int target) {
    if (K >= target) return 1;
    int p = (target + K - 1) / K;
    if (p > 8) p = 8;
    if (p > T) p = T;
    return p < 1 ? 1 : p;
}

// Per-scene arena bytes after the header (n_u = 3 gives the most update blocks).
inline size_t scene_scratch_bytes(int K, int T, int parts) {
    size_t b = 0;
    b += align_up((size_t)K * sizeof(double), 256);
    b += align_up((size_t)K * sizeof(float), 256);
    b += align_up((size_t)upd_blocks_for(K, T, 3) * (T * 3 + 1) * sizeof(float), 256);
    b += align_up((size_t)T * sizeof(unsigned), 256);
    if (parts > 1) {
        b += align_up((size_t)K * T * sizeof(unsigned), 256);
        b += align_up((size_t)K * sizeof(unsigned), 256);
    }
    return b;
}
inline void carve_scene(SceneView &V, char *p, int K, int T, int parts) {
    V.Jt = reinterpret_cast<double *>(p); p += align_up((size_t)K * sizeof(double), 256);
    V.wt = reinterpret_cast<float *>(p); p += align_up((size_t)K * sizeof(float), 256);
    V.part = reinterpret_cast<float *>(p); p += align_up((size_t)upd_blocks_for(K, T, 3) * (T * 3 + 1) * sizeof(float), 256);
    V.vkey = reinterpret_cast<unsigned *>(p); p += align_up((size_t)T * sizeof(unsigned), 256);
    V.parts = parts;
    V.dkey = nullptr;
    V.tk = nullptr;
    if (parts > 1) {
        V.dkey = reinterpret_cast<unsigned *>(p); p += align_up((size_t)K * T * sizeof(unsigned), 256);
        V.tk = reinterpret_cast<unsigned *>(p);
    }
}

// Order-preserving map of a double onto uint64 (total order).
__device__ __forceinline__ unsigned long long d2ord(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord2d(unsigned long long u) {
    return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

// ---------------------------------------------------------------- evaluators
template <class FPC>
struct ConstEval {            // footprint constants in the kernel parameters
    // sub-chunk pruning tests each point against the footprint's bounding
    // box before evaluating it: for polygons (a rectangle cover's evaluation
    // costs about what the test does)
    static constexpr bool kBoxTest = fp_traits<FPC>::kind == EXACT_FP_POLYGON;
    // small footprints: the unpruned loop gives each lane two pairs per
    // iteration (two independent chains; larger footprints would not fit
    // the registers)
    static constexpr bool kPairLoop = fp_traits<FPC>::kind == EXACT_FP_RECTS || fp_traits<FPC>::size <= 6;
    // point-level pruning of small clouds for rectangle covers and polygons
    // of up to 16 edges (another inlined copy of the unrolled evaluator of a
    // larger polygon costs more compile time than the pruning saves)
    static constexpr bool kQueueOk = fp_traits<FPC>::kind == EXACT_FP_RECTS || fp_traits<FPC>::size <= 16;
    FPC f;
    __device__ __forceinline__ void eval2(float px0, float py0, float px1, float py1, float &k0, float &k1) const {
        if constexpr (fp_traits<FPC>::kind == EXACT_FP_RECTS)
            eval2_lazy_depth(f, px0, py0, px1, py1, k0, k1);
        else
            exact::eval2(f, px0, py0, px1, py1, k0, k1);
    }
    __device__ __forceinline__ void eval4(const float (&px)[4], const float (&py)[4], float (&k)[4]) const {
        eval2(px[0], py[0], px[1], py[1], k[0], k[1]);
        eval2(px[2], py[2], px[3], py[3], k[2], k[3]);
    }
    __device__ __forceinline__ float dist(float key) const { return key_to_dist(f, key); }
    __device__ __forceinline__ float3 bound() const { return make_float3(f.bcx, f.bcy, f.brad); }
    __device__ __forceinline__ float4 box() const { return make_float4(f.bcx, f.bcy, f.bhx, f.bhy); }
};

// Footprint constants in shared memory with a run-time edge / box count.
// Polygon (E edges), as lane pairs (the same value twice):
//   C[3b]   = (-v_bx, -v_bx, -v_by, -v_by)                 b <= E, v_E = v_0
//   C[3b+1] = (e_bx/|e_b|^2 twice, -e_bx/e_by twice)       b < E
//   C[3b+2] = (-e_bx, -e_bx, -e_by, -e_by)                 b < E
// then the E scalars e_by/|e_b|^2 from C[3E+1] on.  Rects: C[j] = (cx, cy,
// sx, sy).  The arithmetic is the same sequence of operations as the
// compile-time evaluators, so both give identical keys.
__host__ __device__ constexpr int poly_slot_count(int E) { return 3 * E + 1 + (E + 3) / 4; }

struct SmemEval {
    static constexpr bool kBoxTest = true;   // footprint terms from shared memory: the test pays
    static constexpr bool kPairLoop = true;
    static constexpr bool kQueueOk = true;
    const float4 *C;
    int kind, n;
    float3 bc;    // bounding circle of the footprint (centre, radius)
    float2 bh;    // half extents of its bounding box about the circle's centre
    __device__ __forceinline__ float3 bound() const { return bc; }
    __device__ __forceinline__ float4 box() const { return make_float4(bc.x, bc.y, bh.x, bh.y); }

    // NP lane pairs of points (px[2i], px[2i+1]) against every edge / box;
    // each slot is read once for all of them.
    template <int NP>
    __device__ __forceinline__ void evaln(const float *px, const float *py, float *k) const {
        if (kind == EXACT_FP_POLYGON) {
            // the packed evaluator of poly_eval2 with a run-time edge loop
            // over the slot table of poly_slot_count
            const ulonglong2 *S = reinterpret_cast<const ulonglong2 *>(C);
            const float *eyn = reinterpret_cast<const float *>(C + 3 * n + 1);
            const ulonglong2 v0 = S[0];
            f2x PX[NP], PY[NP], dxa[NP], dya[NP];
            float m[2 * NP];
            unsigned sg[2 * NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                PX[i] = pack2(px[2 * i], px[2 * i + 1]);
                PY[i] = pack2(py[2 * i], py[2 * i + 1]);
                dxa[i] = add2(PX[i], v0.x);
                dya[i] = add2(PY[i], v0.y);
                m[2 * i] = m[2 * i + 1] = finf();
                sg[2 * i] = sg[2 * i + 1] = 0u;
            }
            // one edge for every pair: squared segment distances, parity
            // toggles, and the differences advanced to the next vertex
            auto edge = [&](int b, float ey, float *q) {
                const ulonglong2 kn = S[3 * b + 1], ne = S[3 * b + 2], vn = S[3 * b + 3];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    const f2x dxb = add2(PX[i], vn.x), dyb = add2(PY[i], vn.y);
                    float u0, u1, dy0, dy1;
                    unpack2(mul2(dxa[i], kn.x), u0, u1);
                    unpack2(dya[i], dy0, dy1);
                    const f2x t = pack2(__saturatef(fmaf(dy0, ey, u0)), __saturatef(fmaf(dy1, ey, u1)));
                    const f2x qx = fma2(t, ne.x, dxa[i]), qy = fma2(t, ne.y, dya[i]);
                    unpack2(fma2(qy, qy, mul2(qx, qx)), q[2 * i], q[2 * i + 1]);
                    float h0, h1, x0, x1;
                    unpack2(fma2(dya[i], kn.y, dxa[i]), h0, h1);
                    unpack2(mul2(dya[i], dyb), x0, x1);
                    sg[2 * i] ^= __float_as_uint(x0) & __float_as_uint(h0);
                    sg[2 * i + 1] ^= __float_as_uint(x1) & __float_as_uint(h1);
                    dxa[i] = dxb;
                    dya[i] = dyb;
                }
            };
            // the edge count is padded to an even number: two edges per
            // step, folded with one three-input minimum per point
            for (int b = 0; b < n; b += 2) {
                const float2 ey = *reinterpret_cast<const float2 *>(eyn + b);
                float qa[2 * NP], qb[2 * NP];
                edge(b, ey.x, qa);
                edge(b + 1, ey.y, qb);
#pragma unroll
                for (int i = 0; i < 2 * NP; ++i) m[i] = fmin3(m[i], qa[i], qb[i]);
            }
#pragma unroll
            for (int i = 0; i < 2 * NP; ++i) k[i] = __uint_as_float(__float_as_uint(m[i]) | (sg[i] & 0x80000000u));
        } else {
            float nn[2 * NP], in[2 * NP];
#pragma unroll
            for (int i = 0; i < 2 * NP; ++i) nn[i] = in[i] = finf();
            for (int j = 0; j < n; ++j) {
                const float4 q = C[j];
#pragma unroll
                for (int i = 0; i < 2 * NP; ++i) {
                    const float ax = fabsf(px[i] - q.x) - q.z, ay = fabsf(py[i] - q.y) - q.w;
                    const float ux = ax + fabsf(ax), uy = ay + fabsf(ay);
                    nn[i] = fminf(nn[i], fmaf(uy, uy, ux * ux));
                    in[i] = fminf(in[i], fmaxf(ax, ay));
                }
            }
#pragma unroll
            for (int i = 0; i < 2 * NP; ++i) k[i] = rect_key(nn[i], in[i]);
        }
    }
    __device__ __forceinline__ void eval2(float px0, float py0, float px1, float py1, float &k0, float &k1) const {
        const float px[2] = {px0, px1}, py[2] = {py0, py1};
        float k[2];
        evaln<1>(px, py, k);
        k0 = k[0];
        k1 = k[1];
    }
    __device__ __forceinline__ void eval4(const float (&px)[4], const float (&py)[4], float (&k)[4]) const {
        evaln<2>(px, py, k);
    }
    __device__ __forceinline__ float dist(float key) const {
        if (kind == EXACT_FP_POLYGON) {
            const unsigned b = __float_as_uint(key);
            return __uint_as_float(__float_as_uint(sqrtf(__uint_as_float(b & 0x7fffffffu))) | (b & 0x80000000u));
        }
        return rect_key_to_dist(key);
    }
};

// ---------------------------------------------------------------- chunk bounds
// The staged points are cut into sub-chunks of 64 * ppl consecutive points
// (ppl pairs per lane of a warp).  For each, circ = (centre, radius, max
// speed) of its valid points (radius -1 when it has none).
constexpr int kSub = 64;
constexpr float kPruneSlack = 1e-3f;   // m: far above the float rounding of the distances
constexpr int kPruneMin = 1024;        // points: smaller clouds are pruned point by point (see steps_min_keys)
constexpr int kQueueAll = 1024;        // entries of the block's queues of kept (step, point) pairs
constexpr int kFine = 16;              // points of a fine sub-chunk (a quarter of a sub-chunk)
// Sample-phase code paths compiled into a kernel: every path (chosen per
// call), or only the point-level pruning of small clouds (the caller passes
// no d_min output and fewer than kPruneMin points) -- a smaller kernel whose
// code each block fetches once per cycle.
constexpr int kPathAny = 0, kPathPoints = 1;
constexpr int kQueueFine = 640;        // entries of the block's queues of kept fine sub-chunks

// An ordered cloud of N points carries the circles of its ceil(N / kSub)
// sub-chunks and, after them (256-byte aligned), those of its ceil(N / kFine)
// fine sub-chunks.
__host__ __device__ constexpr int fine_circle_offset(int N) { return (((N + kSub - 1) / kSub) + 15) & ~15; }
__host__ __device__ constexpr size_t circle_bytes(int N) {
    return ((size_t)fine_circle_offset(N) + ((((size_t)N + kFine - 1) / kFine + 15) & ~(size_t)15)) * 16u;
}

template <bool MOVING>
__device__ __forceinline__ void chunk_circles(const float2 *pts, int n, float4 *circ, int ppl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int sz = kSub * ppl;
    const int nsub = (n + sz - 1) / sz;
    for (int s = warp; s < nsub; s += nwarps) {
        float lx = finf(), ly = finf(), hx = -finf(), hy = -finf(), v2 = 0.f;
        for (int i = s * sz + lane; i < min(n, (s + 1) * sz); i += 32) {
            float x, y;
            if constexpr (MOVING) {
                const float4 a = reinterpret_cast<const float4 *>(pts)[i];
                x = a.x; y = a.y;
                if (a.x == a.x) v2 = fmaxf(v2, fmaf(a.z, a.z, a.w * a.w));
            } else {
                x = pts[i].x; y = pts[i].y;
            }
            lx = fminf(lx, x); hx = fmaxf(hx, x); ly = fminf(ly, y); hy = fmaxf(hy, y);   // NaN (masked) ignored
        }
        lx = warp_min_f(lx); ly = warp_min_f(ly); hx = -warp_min_f(-hx); hy = -warp_min_f(-hy);
        const bool any = lx <= hx;
        const float cx = 0.5f * (lx + hx), cy = 0.5f * (ly + hy);
        float r2 = 0.f;
        for (int i = s * sz + lane; i < min(n, (s + 1) * sz); i += 32) {
            float x, y;
            if constexpr (MOVING) {
                const float4 a = reinterpret_cast<const float4 *>(pts)[i];
                x = a.x; y = a.y;
            } else {
                x = pts[i].x; y = pts[i].y;
            }
            if (x == x) r2 = fmaxf(r2, fmaf(x - cx, x - cx, (y - cy) * (y - cy)));
        }
        r2 = -warp_min_f(-r2);
        if (MOVING) v2 = -warp_min_f(-v2);
        if (lane == 0)
            circ[s] = any ? make_float4(cx, cy, sqrtf(r2) * 1.000001f, MOVING ? sqrtf(v2) * 1.000001f : 0.f)
                          : make_float4(0.f, 0.f, -1.f, 0.f);
    }
}

// ---------------------------------------------------------------- cloud order
// Pruning pays only when 64 consecutive points lie close together.  Scans
// deliver clouds in that order; for any other order one block rewrites the
// cloud in Morton order of a 64 x 64 grid over its bounding box (a counting
// sort: histogram, prefix sum, scatter).  Masked and non-finite points go
// last, as NaN, so the copy needs no mask.  The order inside a grid cell
// follows the scatter's atomics; nothing computed from the cloud depends on
// it (minima over points are exact whatever the order).
constexpr int kSortCells = 64 * 64;
constexpr int kSortThreads = 1024;
constexpr int kSortRegs = 4;   // points per thread kept in registers (clouds of up to 4,096)
struct SortSmem {
    int cnt[kSortCells + 1];
    float red[4][kSortThreads / 32];
    float box[4];
    int part[kSortThreads / 32];
};

__device__ __forceinline__ unsigned morton6(unsigned x, unsigned y) {
    unsigned r = 0u;
#pragma unroll
    for (int b = 0; b < 6; ++b) r |= (((x >> b) & 1u) << (2 * b)) | (((y >> b) & 1u) << (2 * b + 1));
    return r;
}

template <bool MOVING>
__device__ __forceinline__ void sort_cloud_block(const float2 *__restrict__ pts, const float2 *__restrict__ vel,
                                                 const uint8_t *__restrict__ mask, int N, float2 *__restrict__ opts,
                                                 float2 *__restrict__ ovel, SortSmem &sm) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    grid_dep_release();   // the sample kernel may start its rollouts meanwhile
    auto valid = [&](int i, float2 &p) {
        p = pts[i];
        return (!mask || mask[i]) && isfinite(p.x) && isfinite(p.y);
    };
    // clouds of up to kSortRegs points per thread are read once and kept in
    // registers (point tid + k nt in slot k); larger ones are re-read per pass
    const bool inreg = N <= kSortRegs * nt;
    float2 rp[kSortRegs];
    bool rv[kSortRegs];
    if (inreg) {
#pragma unroll
        for (int k = 0; k < kSortRegs; ++k) {
            const int i = tid + k * nt;
            rv[k] = i < N && valid(i, rp[k]);
        }
    }
    float lx = finf(), ly = finf(), hx = -finf(), hy = -finf();
    auto grow = [&](float2 p) { lx = fminf(lx, p.x); hx = fmaxf(hx, p.x); ly = fminf(ly, p.y); hy = fmaxf(hy, p.y); };
    if (inreg) {
#pragma unroll
        for (int k = 0; k < kSortRegs; ++k)
            if (rv[k]) grow(rp[k]);
    } else {
        for (int i = tid; i < N; i += nt) {
            float2 p;
            if (valid(i, p)) grow(p);
        }
    }
    lx = warp_min_f(lx); ly = warp_min_f(ly); hx = -warp_min_f(-hx); hy = -warp_min_f(-hy);
    if (lane == 0) { sm.red[0][warp] = lx; sm.red[1][warp] = ly; sm.red[2][warp] = hx; sm.red[3][warp] = hy; }
    for (int c = tid; c <= kSortCells; c += nt) sm.cnt[c] = 0;
    __syncthreads();
    if (warp == 0) {   // the warps' boxes, reduced by one warp
        const bool w = lane < nw;
        lx = warp_min_f(w ? sm.red[0][lane] : finf());
        ly = warp_min_f(w ? sm.red[1][lane] : finf());
        hx = -warp_min_f(w ? -sm.red[2][lane] : finf());
        hy = -warp_min_f(w ? -sm.red[3][lane] : finf());
        if (lane == 0) { sm.box[0] = lx; sm.box[1] = ly; sm.box[2] = hx; sm.box[3] = hy; }
    }
    __syncthreads();
    lx = sm.box[0]; ly = sm.box[1]; hx = sm.box[2]; hy = sm.box[3];
    const float sx = 64.f / fmaxf(hx - lx, 1e-6f), sy = 64.f / fmaxf(hy - ly, 1e-6f);
    auto cell_of = [&](bool ok, float2 p) -> int {
        if (!ok) return kSortCells;
        const int qx = min(63, max(0, (int)((p.x - lx) * sx))), qy = min(63, max(0, (int)((p.y - ly) * sy)));
        return (int)morton6((unsigned)qx, (unsigned)qy);
    };
    int rc[kSortRegs];
    if (inreg) {
#pragma unroll
        for (int k = 0; k < kSortRegs; ++k) {
            rc[k] = cell_of(rv[k], rp[k]);
            if (tid + k * nt < N) atomicAdd(&sm.cnt[rc[k]], 1);
        }
    } else {
        for (int i = tid; i < N; i += nt) {
            float2 p;
            const bool ok = valid(i, p);
            atomicAdd(&sm.cnt[cell_of(ok, p)], 1);
        }
    }
    __syncthreads();
    // exclusive prefix over the kSortCells + 1 counts: contiguous segments per thread
    const int per = (kSortCells + 1 + nt - 1) / nt, c0 = tid * per, c1 = min(kSortCells + 1, c0 + per);
    int s = 0;
    for (int c = c0; c < c1; ++c) s += sm.cnt[c];
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm.part[warp] = inc;
    __syncthreads();
    if (warp == 0) {   // exclusive prefix of the warps' totals, by one warp
        const int v = lane < nw ? sm.part[lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        __syncwarp();
        if (lane < nw) sm.part[lane] = x - v;
    }
    __syncthreads();
    const int base = sm.part[warp];
    int run = base + inc - s;
    for (int c = c0; c < c1; ++c) {
        const int v = sm.cnt[c];
        sm.cnt[c] = run;
        run += v;
    }
    __syncthreads();
    const float qnan = __int_as_float(0x7fffffff);
    auto place = [&](int i, int c, float2 p) {
        const int pos = atomicAdd(&sm.cnt[c], 1);
        opts[pos] = c < kSortCells ? p : make_float2(qnan, qnan);
        if (MOVING) ovel[pos] = c < kSortCells ? vel[i] : make_float2(0.f, 0.f);
    };
    if (inreg) {
#pragma unroll
        for (int k = 0; k < kSortRegs; ++k) {
            const int i = tid + k * nt;
            if (i < N) place(i, rc[k], rp[k]);
        }
    } else {
        for (int i = tid; i < N; i += nt) {
            float2 p;
            const bool ok = valid(i, p);
            place(i, cell_of(ok, p), p);
        }
    }
}

// Bounding circles (centre, radius, max speed) of the 64-point sub-chunks of
// an ordered cloud in global memory, one warp per sub-chunk; the same values
// chunk_circles computes for one staged pass, computed once per cycle.  The
// circles of the 16-point fine sub-chunks (same construction over a half
// warp's points) follow at circ + fine_circle_offset(N).
template <bool MOVING>
__device__ __forceinline__ void cloud_circles(const float2 *__restrict__ pts, const float2 *__restrict__ vel, int N,
                                              float4 *__restrict__ circ) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nsub = (N + kSub - 1) / kSub;
    for (int s = warp; s < nsub; s += nwarps) {
        float x[2], y[2], v2 = 0.f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = s * kSub + k * 32 + lane;
            x[k] = y[k] = __int_as_float(0x7fffffff);
            if (i < N) {
                x[k] = pts[i].x; y[k] = pts[i].y;
                if (MOVING && x[k] == x[k]) v2 = fmaxf(v2, fmaf(vel[i].x, vel[i].x, vel[i].y * vel[i].y));
            }
        }
        float lx = warp_min_f(fminf(x[0], x[1])), ly = warp_min_f(fminf(y[0], y[1]));
        float hx = -warp_min_f(-fmaxf(x[0], x[1])), hy = -warp_min_f(-fmaxf(y[0], y[1]));
        const bool any = lx <= hx;
        const float cx = 0.5f * (lx + hx), cy = 0.5f * (ly + hy);
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (x[k] == x[k]) r2 = fmaxf(r2, fmaf(x[k] - cx, x[k] - cx, (y[k] - cy) * (y[k] - cy)));
        r2 = -warp_min_f(-r2);
        if (MOVING) v2 = -warp_min_f(-v2);
        if (lane == 0)
            circ[s] = any ? make_float4(cx, cy, sqrtf(r2) * 1.000001f, MOVING ? sqrtf(v2) * 1.000001f : 0.f)
                          : make_float4(0.f, 0.f, -1.f, 0.f);
        // fine sub-chunk 2k + (lane >> 4): points k * 32 + lane of this sub-chunk
        float4 *fine = circ + fine_circle_offset(N);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float flx = x[k], fly = y[k], fhx = x[k], fhy = y[k], fv2 = 0.f;
            if (MOVING && x[k] == x[k]) {
                const int i = s * kSub + k * 32 + lane;
                fv2 = fmaf(vel[i].x, vel[i].x, vel[i].y * vel[i].y);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {   // within each half warp; NaN (masked, absent) ignored
                flx = fminf(flx, __shfl_xor_sync(0xffffffffu, flx, o));
                fly = fminf(fly, __shfl_xor_sync(0xffffffffu, fly, o));
                fhx = fmaxf(fhx, __shfl_xor_sync(0xffffffffu, fhx, o));
                fhy = fmaxf(fhy, __shfl_xor_sync(0xffffffffu, fhy, o));
                if (MOVING) fv2 = fmaxf(fv2, __shfl_xor_sync(0xffffffffu, fv2, o));
            }
            const bool fany = flx <= fhx;
            const float fcx = 0.5f * (flx + fhx), fcy = 0.5f * (fly + fhy);
            float fr2 = x[k] == x[k] ? fmaf(x[k] - fcx, x[k] - fcx, (y[k] - fcy) * (y[k] - fcy)) : 0.f;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) fr2 = fmaxf(fr2, __shfl_xor_sync(0xffffffffu, fr2, o));
            const int f = s * (kSub / kFine) + 2 * k + (lane >> 4);
            if ((lane & 15) == 0 && f * kFine < N)
                fine[f] = fany ? make_float4(fcx, fcy, sqrtf(fr2) * 1.000001f, MOVING ? sqrtf(fv2) * 1.000001f : 0.f)
                               : make_float4(0.f, 0.f, -1.f, 0.f);
        }
    }
}

// ---------------------------------------------------------------- sample phase
// Position of the k-th (from 0) set bit of m; k < popc(m).
__device__ __forceinline__ int nth_set_bit64(unsigned long long m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 32; w > 0; w >>= 1) {
        const unsigned long long low = m & ((1ull << w) - 1ull);
        const int c = __popcll(low);
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return pos;
}

// Per-step minimum of the body-frame key over n staged points for the steps
// [h0, h0 + nh) whose poses are in shared memory.  Masked points were staged
// as NaN, which every evaluator turns into a +inf key (NaN terms are dropped
// by min, and the canonical NaN has a clear sign bit, so it never toggles the
// crossing parity).  A ragged last pair repeats its first point.
//
// MOVING: each staged entry is (o_x, o_y, v_x, v_y) and the point of step h
// is the constant-velocity prediction o + t_h v at the time t_h of the scored
// state (the time-indexed obstacle prediction of Sec. V-F).
//
// Schedule when pruning (cap >= 0), in three block-wide phases:
//  1. one lane per (step, sub-chunk): keep the pair unless the sub-chunk's
//     circle lies farther than `cap` (plus a slack far above rounding) from
//     the footprint's bounding circle at that step (cw);
//  2. a prefix sum of the kept pairs per step (bit masks in msk);
//  3. every warp walks an equal contiguous share of the kept (step,
//     sub-chunk) list; polygons and shared-memory footprints keep the points
//     that lie within cap of the footprint's bounding box in that step's
//     body frame and evaluate them through the warp's queue (queue:
//     kQueueAll ints of shared memory); rectangle covers keep the 16-point
//     fine sub-chunks whose circles (circf, from the ordered cloud) come
//     within cap of that box and evaluate them through the queue qfine
//     (kQueueFine ints), or, without fine circles, evaluate every point and
//     fold each step's minimum into keyh[h] (one warp shuffle-min and one
//     shared atomicMin per step run).
// With queue_points (clouds below kPruneMin) the phases are replaced by a
// point-level test against the footprint's bounding circle, feeding the
// same kind of queue.  Pruning never changes a result: cap = d_safe is passed only
// when no d_min output is wanted, and every cost term and the validation
// test are the same for any d >= d_safe; a skipped point is provably farther
// than that.  Without pruning (cap < 0) items (step h, chunk of 128 pairs)
// are dealt to the warps round-robin, each ending in one warp shuffle-min and
// one shared atomicMin on the key of step h.
template <bool MOVING = false, int PATH = kPathAny, class EV>
__device__ __forceinline__ void steps_min_keys(const EV &ev, const float2 *pts, int n, const float4 *pose,
                                               const float4 *cw, int h0, int nh, unsigned *keyh, int ppl,
                                               const float4 *circ, float cap, unsigned *msk, int *pre,
                                               int *queue, bool queue_points, const float4 *circf, int *qfine,
                                               int *err = nullptr) {
    const int npairs = (n + 1) >> 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nsub = (n + kSub * ppl - 1) / (kSub * ppl);
    // pair j (points 2j, 2j+1; an odd tail repeats the last point) in the
    // body frame of step h
    auto pair_at = [&](int j, int h, float &px0, float &py0, float &px1, float &py1) {
        const float4 q = pose[h];
        float2 o0, o1;
        if constexpr (MOVING) {
            const float th = cw[h].z;
            const float4 *p4 = reinterpret_cast<const float4 *>(pts);
            const float4 a0 = p4[2 * j], a1 = p4[min(2 * j + 1, n - 1)];
            o0 = make_float2(fmaf(th, a0.z, a0.x), fmaf(th, a0.w, a0.y));
            o1 = make_float2(fmaf(th, a1.z, a1.x), fmaf(th, a1.w, a1.y));
        } else {
            o0 = pts[2 * j];
            o1 = pts[min(2 * j + 1, n - 1)];
        }
        body_frame(o0.x, o0.y, q.x, q.y, q.z, q.w, px0, py0);
        body_frame(o1.x, o1.y, q.x, q.y, q.z, q.w, px1, py1);
    };
    if (PATH == kPathAny && (cap < 0.f || (queue_points && !EV::kQueueOk))) {   // no pruning
        const int span = 32 * 4;   // pairs per item
        const int nchunk = npairs > 0 ? (npairs + span - 1) / span : 0;
        const int items = nh * nchunk;
        for (int it = warp; it < items; it += nwarps) {
            const int hh = it / nchunk, c = it - hh * nchunk;
            const int h = h0 + hh;
            const float4 q = pose[h];
            const float th = cw[h].z;
            float best = finf();
            const int jend = min(npairs, (c + 1) * span);
            if constexpr (EV::kPairLoop) {
                for (int j = c * span + lane; j < jend; j += 64) {
                    const bool two = j + 32 < jend;
                    float px[4], py[4], k[4];
                    pair_at(j, h, px[0], py[0], px[1], py[1]);
                    pair_at(two ? j + 32 : j, h, px[2], py[2], px[3], py[3]);
                    ev.eval4(px, py, k);
                    best = fmin3(best, k[0], k[1]);
                    if (two) best = fmin3(best, k[2], k[3]);
                }
            } else {
                for (int j = c * span + lane; j < jend; j += 32) {
                    float2 o0, o1;
                    if constexpr (MOVING) {
                        const float4 *p4 = reinterpret_cast<const float4 *>(pts);
                        const float4 a0 = p4[2 * j], a1 = p4[min(2 * j + 1, n - 1)];
                        o0 = make_float2(fmaf(th, a0.z, a0.x), fmaf(th, a0.w, a0.y));
                        o1 = make_float2(fmaf(th, a1.z, a1.x), fmaf(th, a1.w, a1.y));
                    } else {
                        o0 = pts[2 * j];
                        o1 = pts[min(2 * j + 1, n - 1)];
                    }
                    float px0, py0, px1, py1;
                    body_frame(o0.x, o0.y, q.x, q.y, q.z, q.w, px0, py0);
                    body_frame(o1.x, o1.y, q.x, q.y, q.z, q.w, px1, py1);
                    float k0, k1;
                    ev.eval2(px0, py0, px1, py1, k0, k1);
                    best = fmin3(best, k0, k1);
                }
            }
            best = warp_min_f(best);
            if (lane == 0) atomicMin(keyh + h, f2ord(best));
        }
        return;
    }
    if constexpr (EV::kQueueOk) if (PATH == kPathPoints || queue_points) {
        // Point-level pruning (clouds below kPruneMin, no sort, no circles).
        // Every warp first bounds the sample's trajectory by one circle
        // (cb, rb) that holds the footprint's bounding circle at every step
        // plus cap and the slack of the chunk test (taken for a circle of
        // radius 0), then walks its contiguous share of the point pairs: a
        // point outside that circle (grown by t_max |v|_1 for predicted
        // points) is farther than cap from the footprint at every step; each
        // point inside is tested against every step's circle, one lane per
        // step.  Kept (step, point) entries are appended to the warp's queue
        // and evaluated 64 at a time, two per lane (the two lanes of the
        // packed evaluator may hold points of different steps: the footprint
        // is the same in every body frame), each key folded into its step's
        // minimum with a shared atomicMin.  A warp's queue holds kQueueAll /
        // warps entries: with 128 or more a flush waits for 64 entries, with
        // fewer every iteration that adds some flushes them.
        const float3 bc = ev.bound();
        const float lim = cap + kPruneSlack;
        const int cap_q = kQueueAll / nwarps;
        const int flush_at = cap_q >= 128 ? 64 : 1;
        int *q = queue + warp * cap_q;
        int qn = 0;   // warp-uniform
        auto point_at = [&](int i, int h) -> float2 {
            if constexpr (MOVING) {
                const float th = cw[h].z;
                const float4 a = reinterpret_cast<const float4 *>(pts)[i];
                return make_float2(fmaf(th, a.z, a.x), fmaf(th, a.w, a.y));
            } else {
                return pts[i];
            }
        };
        auto flush = [&](int cnt) {   // entries [0, cnt), cnt <= 64
            __syncwarp();
            const int a = 2 * lane;
            if (a < cnt) {
                const bool two = a + 1 < cnt;
                int ea = q[a], eb = two ? q[a + 1] : ea;
                if (!EXACT_DCHECK((ea & 4095) < n && (ea >> 12) < nh, err)) ea = 0;   // debug build: skip
                if (!EXACT_DCHECK((eb & 4095) < n && (eb >> 12) < nh, err)) eb = 0;
                const int ha = h0 + (ea >> 12), hb = h0 + (eb >> 12);
                const float2 oa = point_at(ea & 4095, ha), ob = point_at(eb & 4095, hb);
                const float4 pa = pose[ha], pb = pose[hb];
                float pxa, pya, pxb, pyb;
                body_frame(oa.x, oa.y, pa.x, pa.y, pa.z, pa.w, pxa, pya);
                body_frame(ob.x, ob.y, pb.x, pb.y, pb.z, pb.w, pxb, pyb);
                float ka, kb;
                ev.eval2(pxa, pya, pxb, pyb, ka, kb);
                atomicMin(keyh + ha, f2ord(ka));
                if (two) atomicMin(keyh + hb, f2ord(kb));
            }
            __syncwarp();
        };
        // the trajectory's circle: centre of the step circles' bounding box,
        // radius max_h |cw_h - cb| + reach_h with a relative margin far above
        // the rounding of the step tests
        float lx = finf(), ly = finf(), hx = -finf(), hy = -finf(), tmax = 0.f;
        for (int k = lane; k < nh; k += 32) {
            const float4 c = cw[h0 + k];
            lx = fminf(lx, c.x); hx = fmaxf(hx, c.x); ly = fminf(ly, c.y); hy = fmaxf(hy, c.y);
            tmax = fmaxf(tmax, c.z);
        }
        lx = warp_min_f(lx); ly = warp_min_f(ly); hx = -warp_min_f(-hx); hy = -warp_min_f(-hy);
        if (MOVING) tmax = -warp_min_f(-tmax);
        const float cbx = 0.5f * (lx + hx), cby = 0.5f * (ly + hy);
        float rb = 0.f;
        for (int k = lane; k < nh; k += 32) {
            const float4 c = cw[h0 + k];
            const float dx = c.x - cbx, dy = c.y - cby;
            rb = fmaxf(rb, sqrtf(fmaf(dx, dx, dy * dy)) + bc.z + lim + 1e-5f * (fabsf(c.x) + fabsf(c.y)));
        }
        rb = -warp_min_f(-rb);
        rb = fmaf(rb, 1e-5f, rb) + 1e-5f;
        auto near_path = [&](int i) {   // NaN (masked) never kept
            float x, y, g = rb;
            if constexpr (MOVING) {
                const float4 a = reinterpret_cast<const float4 *>(pts)[i];
                x = a.x; y = a.y;
                g = fmaf(tmax * 1.0001f, fabsf(a.z) + fabsf(a.w), g);
            } else {
                x = pts[i].x; y = pts[i].y;
            }
            g = fmaf(1e-5f, fabsf(x) + fabsf(y), g);
            const float dx = x - cbx, dy = y - cby;
            return fmaf(dx, dx, dy * dy) <= g * g;
        };
        const int p0 = (int)(((long long)npairs * warp) / nwarps), p1 = (int)(((long long)npairs * (warp + 1)) / nwarps);
        for (int pb = p0; pb < p1; pb += 32) {
            const int j = pb + lane;
            const bool c0 = j < p1 && near_path(2 * j);
            const bool c1 = j < p1 && 2 * j + 1 < n && near_path(2 * j + 1);
            unsigned b0 = __ballot_sync(0xffffffffu, c0), b1 = __ballot_sync(0xffffffffu, c1);
            while (b0 | b1) {   // the candidates in lane order, each against every step
                int i;
                if (b0) {
                    i = 2 * (pb + __ffs(b0) - 1);
                    b0 &= b0 - 1u;
                } else {
                    i = 2 * (pb + __ffs(b1) - 1) + 1;
                    b1 &= b1 - 1u;
                }
                for (int k0 = 0; k0 < nh; k0 += 32) {
                    const int k = k0 + lane;
                    bool keep = false;
                    if (k < nh) {
                        const float4 c = cw[h0 + k];
                        const float reach = bc.z + lim + 1e-5f * (fabsf(c.x) + fabsf(c.y));
                        const float2 o = point_at(i, h0 + k);
                        const float dx = o.x - c.x, dy = o.y - c.y;
                        const float f = fmaf(1e-5f, fabsf(o.x) + fabsf(o.y), reach);
                        keep = fmaf(dx, dx, dy * dy) <= f * f;
                    }
                    const unsigned bk = __ballot_sync(0xffffffffu, keep);
                    if (bk) {
                        if (keep) q[qn + __popc(bk & ((1u << lane) - 1u))] = (k << 12) | i;
                        qn += __popc(bk);
                        if (qn >= flush_at) {
                            const int f = min(qn, 64);
                            flush(f);
                            for (int e = lane; e < qn - f; e += 32) q[e] = q[f + e];
                            __syncwarp();
                            qn -= f;
                        }
                    }
                }
            }
        }
        if (qn > 0) flush(qn);
        return;
    }
    if constexpr (PATH == kPathAny) {
        const float brad = ev.bound().z;
        const float lim = cap >= 0.f ? cap + kPruneSlack : finf();
        // 1. per (step, sub-chunk) tests, 32 sub-chunks per ballot
        for (int idx = warp; idx < 2 * nh; idx += nwarps) {
            const int hh = idx >> 1, s = ((idx & 1) << 5) + lane;
            bool keep = false;
            if (s < nsub) {
                const float4 cc = circ[s];
                if (cc.z >= 0.f) {
                    const float4 cq = cw[h0 + hh];
                    const float dx = cc.x - cq.x, dy = cc.y - cq.y;
                    float reach = cc.z + brad + 1e-5f * (fabsf(cc.x) + fabsf(cc.y) + fabsf(cq.x) + fabsf(cq.y));
                    if (MOVING) reach = fmaf(cq.z, cc.w, reach);
                    const float far = reach + lim;   // drop iff |centre - footprint centre| > far
                    keep = !(fmaf(dx, dx, dy * dy) > far * far);
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) msk[idx] = b;
        }
        __syncthreads();
        // 2. exclusive prefix of the per-step counts
        if (warp == 0) {
            int run = 0;
            for (int base = 0; base < nh; base += 32) {
                const int hh = base + lane;
                const int cnt = hh < nh ? __popc(msk[2 * hh]) + __popc(msk[2 * hh + 1]) : 0;
                int inc = cnt;
    #pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                if (hh < nh) pre[hh] = run + inc - cnt;
                run += __shfl_sync(0xffffffffu, inc, 31);
            }
            if (lane == 0) pre[nh] = run;
        }
        __syncthreads();
        // 3. this warp's share [e0, e1) of the kept list, in (step, sub-chunk) order
        const int L = pre[nh];
        const int e0 = (int)(((long long)L * warp) / nwarps), e1 = (int)(((long long)L * (warp + 1)) / nwarps);
        if (e0 >= e1) return;
        int lo = 0, hi = nh - 1;   // the step holding entry e0: the last with pre <= e0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= e0) lo = mid; else hi = mid - 1;
        }
        int hh = lo;
        unsigned long long m = ((unsigned long long)msk[2 * hh + 1] << 32) | msk[2 * hh];
        for (int k = pre[hh]; k < e0; ++k) m &= m - 1ull;
        if constexpr (EV::kBoxTest) {
            // Polygons and shared-memory footprints: the points of a kept
            // sub-chunk are moved into the body frame of its step and kept only
            // if they lie within cap (plus the slack) of the footprint's bounding
            // box there; the kept ones go through the warp's queue, as in the
            // point-level path.  The evaluator gives the same key for that
            // body-frame point, and sd_F >= sd_box everywhere for a footprint F
            // inside the box, so a dropped point is provably farther than cap.
            // (For a rectangle cover the test costs about what the evaluation
            // does, and the kept points are evaluated directly below.)
            const float4 fb = ev.box();
            const int cap_q = kQueueAll / nwarps;
            const int flush_at = cap_q >= 128 ? 64 : 1;
            int *q = queue + warp * cap_q;
            int qn = 0;   // warp-uniform
            auto point_at = [&](int i, int h) -> float2 {
                if constexpr (MOVING) {
                    const float th = cw[h].z;
                    const float4 a = reinterpret_cast<const float4 *>(pts)[i];
                    return make_float2(fmaf(th, a.z, a.x), fmaf(th, a.w, a.y));
                } else {
                    return pts[i];
                }
            };
            int e = e0, jb = 0, jend = 0;
            for (;;) {
                if (jb >= jend && e < e1) {   // next kept (step, sub-chunk) entry
                    while (m == 0ull && EXACT_DCHECK(hh + 1 < nh, err)) {
                        ++hh;
                        m = ((unsigned long long)msk[2 * hh + 1] << 32) | msk[2 * hh];
                    }
                    if (m == 0ull) {   // debug build: the list ended early
                        e = e1;
                    } else {
                        const int s = __ffsll((long long)m) - 1;
                        m &= m - 1ull;
                        ++e;
                        jb = s * 32 * ppl;
                        jend = min(npairs, (s + 1) * 32 * ppl);
                    }
                }
                const bool more = jb < jend;
                const int j = jb + lane;   // points 2j and 2j + 1 of step slot hh
                bool k0 = false, k1 = false;
                if (more && j < jend) {
                    const float4 qp = pose[h0 + hh];
                    auto near_box = [&](float2 o) {
                        float px, py;
                        body_frame(o.x, o.y, qp.x, qp.y, qp.z, qp.w, px, py);
                        const float ax = fabsf(px - fb.x) - fb.z, ay = fabsf(py - fb.y) - fb.w;
                        const float l = fmaf(1e-5f, fabsf(px) + fabsf(py), lim);
                        const float mx = fmaxf(ax, 0.f), my = fmaxf(ay, 0.f);
                        return ax <= l && ay <= l && fmaf(mx, mx, my * my) <= l * l;   // NaN (masked): false
                    };
                    k0 = near_box(point_at(2 * j, h0 + hh));
                    if (2 * j + 1 < n) k1 = near_box(point_at(2 * j + 1, h0 + hh));
                }
                jb += 32;
                const unsigned b0 = __ballot_sync(0xffffffffu, k0), b1 = __ballot_sync(0xffffffffu, k1);
                if (b0 | b1) {
                    const unsigned below = (1u << lane) - 1u;
                    const int pos = qn + __popc(b0 & below) + __popc(b1 & below);
                    if (k0) q[pos] = (hh << 12) | (2 * j);
                    if (k1) q[pos + (k0 ? 1 : 0)] = (hh << 12) | (2 * j + 1);
                    qn += __popc(b0) + __popc(b1);
                }
                if (qn >= flush_at || (!more && qn > 0)) {
                    // evaluate entries [0, f), f <= 64, and move the rest to the front
                    const int f = min(qn, 64);
                    __syncwarp();
                    const int a = 2 * lane;
                    if (a < f) {
                        const bool two = a + 1 < f;
                        int ea = q[a], eb = two ? q[a + 1] : ea;
                        if (!EXACT_DCHECK((ea & 4095) < n && (ea >> 12) < nh, err)) ea = 0;   // debug build: skip
                        if (!EXACT_DCHECK((eb & 4095) < n && (eb >> 12) < nh, err)) eb = 0;
                        const int ha = h0 + (ea >> 12), hb = h0 + (eb >> 12);
                        const float2 oa = point_at(ea & 4095, ha), ob = point_at(eb & 4095, hb);
                        const float4 pa = pose[ha], pb = pose[hb];
                        float pxa, pya, pxb, pyb;
                        body_frame(oa.x, oa.y, pa.x, pa.y, pa.z, pa.w, pxa, pya);
                        body_frame(ob.x, ob.y, pb.x, pb.y, pb.z, pb.w, pxb, pyb);
                        float ka, kb;
                        ev.eval2(pxa, pya, pxb, pyb, ka, kb);
                        atomicMin(keyh + ha, f2ord(ka));
                        if (two) atomicMin(keyh + hb, f2ord(kb));
                    }
                    __syncwarp();
                    for (int i = lane; i < qn - f; i += 32) q[i] = q[f + i];
                    __syncwarp();
                    qn -= f;
                }
                if (!more && qn == 0) return;
            }
        }
        if (circf) {
            // Rectangle covers with the fine circles of an ordered cloud: the
            // four 16-point fine sub-chunks of every kept (step, sub-chunk) entry
            // are tested against the footprint's bounding box in the step's body
            // frame (one lane per fine sub-chunk, eight entries per warp
            // iteration, each lane decoding its own entry from pre and msk); the
            // kept ones go through the warp's queue and are evaluated four at a
            // time, eight lanes (one pair each) per fine sub-chunk, whose step
            // minimum is folded over the eight lanes and into keyh[h] with one
            // shared atomicMin.  Every point of a fine sub-chunk lies within its
            // circle (radius grown by t_h times its largest speed when MOVING),
            // sd_F >= sd_box for a footprint F inside the box, and sd_box is
            // 1-Lipschitz, so a dropped fine sub-chunk holds no point within cap.
            const float4 fb = ev.box();
            const int capf = kQueueFine / nwarps;   // >= 40 for up to 16 warps: 3 left + 32 added fit
            int *q = qfine + warp * capf;
            int qn = 0;   // warp-uniform
            const int nfine = (n + kFine - 1) / kFine;
            for (int e = e0;; e += 8) {
                const bool more = e < e1;
                const int my = e + (lane >> 2);
                bool keep = false;
                int code = 0;
                if (more && my < e1) {
                    int lo = 0, hi = nh - 1;   // the step holding entry my: the last with pre <= my
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (pre[mid] <= my) lo = mid; else hi = mid - 1;
                    }
                    const unsigned long long mm = ((unsigned long long)msk[2 * lo + 1] << 32) | msk[2 * lo];
                    const int fi = nth_set_bit64(mm, my - pre[lo]) * (kSub / kFine) + (lane & 3);
                    if (fi < nfine) {
                        const float4 c = circf[fi];
                        if (c.z >= 0.f) {
                            const float4 qp = pose[h0 + lo];
                            float px, py;
                            body_frame(c.x, c.y, qp.x, qp.y, qp.z, qp.w, px, py);
                            float reach = c.z + 1e-5f * (fabsf(c.x) + fabsf(c.y) + fabsf(qp.x) + fabsf(qp.y));
                            if (MOVING) reach = fmaf(cw[h0 + lo].z, c.w, reach);
                            const float l = reach + lim;
                            const float ax = fabsf(px - fb.x) - fb.z, ay = fabsf(py - fb.y) - fb.w;
                            const float mx = fmaxf(ax, 0.f), my2 = fmaxf(ay, 0.f);
                            keep = ax <= l && ay <= l && fmaf(mx, mx, my2 * my2) <= l * l;
                        }
                    }
                    code = (lo << 12) | fi;
                }
                const unsigned b = __ballot_sync(0xffffffffu, keep);
                if (keep) q[qn + __popc(b & ((1u << lane) - 1u))] = code;
                qn += __popc(b);
                while (qn >= 4 || (!more && qn > 0)) {
                    // evaluate entries [0, f), f <= 4, and move the rest to the front
                    const int f = min(qn, 4);
                    __syncwarp();
                    const int slot = lane >> 3, pr = lane & 7;
                    float best = finf();
                    int sh = 0;
                    if (slot < f) {
                        int ce = q[slot];
                        if (!EXACT_DCHECK((ce >> 12) < nh && (ce & 4095) < nfine, err)) ce = 0;   // debug build: skip
                        sh = ce >> 12;
                        const int j = (ce & 4095) * (kFine / 2) + pr;   // pair j of the staged points
                        if (j < npairs) {
                            const int h = h0 + sh;
                            const float4 qp = pose[h];
                            float2 o0, o1;
                            if constexpr (MOVING) {
                                const float th = cw[h].z;
                                const float4 *p4 = reinterpret_cast<const float4 *>(pts);
                                const float4 a0 = p4[2 * j], a1 = p4[min(2 * j + 1, n - 1)];
                                o0 = make_float2(fmaf(th, a0.z, a0.x), fmaf(th, a0.w, a0.y));
                                o1 = make_float2(fmaf(th, a1.z, a1.x), fmaf(th, a1.w, a1.y));
                            } else {
                                o0 = pts[2 * j];
                                o1 = pts[min(2 * j + 1, n - 1)];
                            }
                            float px0, py0, px1, py1;
                            body_frame(o0.x, o0.y, qp.x, qp.y, qp.z, qp.w, px0, py0);
                            body_frame(o1.x, o1.y, qp.x, qp.y, qp.z, qp.w, px1, py1);
                            float k0, k1;
                            ev.eval2(px0, py0, px1, py1, k0, k1);
                            best = fminf(k0, k1);
                        }
                    }
    #pragma unroll
                    for (int o = 4; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
                    if (slot < f && pr == 0 && best < finf()) atomicMin(keyh + h0 + sh, f2ord(best));
                    __syncwarp();
                    for (int i = lane; i < qn - f; i += 32) q[i] = q[f + i];
                    __syncwarp();
                    qn -= f;
                }
                if (!more) return;
            }
        }
        float best = finf();
        for (int e = e0; e < e1; ++e) {
            if (!EXACT_DCHECK(hh < nh, err)) break;
            while (m == 0ull) {   // step done: fold its minimum, move to the next step with entries
                best = warp_min_f(best);
                if (lane == 0 && best < finf()) atomicMin(keyh + h0 + hh, f2ord(best));
                best = finf();
                ++hh;
                m = ((unsigned long long)msk[2 * hh + 1] << 32) | msk[2 * hh];
            }
            const int s = __ffsll((long long)m) - 1;
            m &= m - 1ull;
            const int h = h0 + hh;
            const float4 q = pose[h];
            const float th = cw[h].z;
            for (int j = s * 32 * ppl + lane; j < min(npairs, (s + 1) * 32 * ppl); j += 32) {
                float2 o0, o1;
                if constexpr (MOVING) {
                    const float4 *p4 = reinterpret_cast<const float4 *>(pts);
                    const float4 a0 = p4[2 * j], a1 = p4[min(2 * j + 1, n - 1)];
                    o0 = make_float2(fmaf(th, a0.z, a0.x), fmaf(th, a0.w, a0.y));
                    o1 = make_float2(fmaf(th, a1.z, a1.x), fmaf(th, a1.w, a1.y));
                } else {
                    o0 = pts[2 * j];
                    o1 = pts[min(2 * j + 1, n - 1)];
                }
                float px0, py0, px1, py1;
                body_frame(o0.x, o0.y, q.x, q.y, q.z, q.w, px0, py0);
                body_frame(o1.x, o1.y, q.x, q.y, q.z, q.w, px1, py1);
                float k0, k1;
                ev.eval2(px0, py0, px1, py1, k0, k1);
                best = fmin3(best, k0, k1);
            }
        }
        best = warp_min_f(best);
        if (lane == 0 && best < finf()) atomicMin(keyh + h0 + hh, f2ord(best));
    }
}

// Copy points [base, base + n) into shared memory, masked ones as NaN, with
// the nt threads t0 = 0 .. nt - 1 of the calling group (a multiple of 32;
// they meet on named barrier 1).  Static clouds whose source is 16-byte
// aligned go through one TMA bulk copy (cp.async.bulk, completed on the
// mbarrier bar, initialised once per kernel, whose completed phases *uses
// counts; bounded wait; an odd last point by a plain load); predicted
// clouds through 8-byte cp.async copies into the (position, velocity) float4
// of each point.  Neither passes the points through registers.  After the
// copies have landed, masked points are overwritten with NaN.  A source that
// is only 8-byte aligned is staged through registers, eight loads per thread
// in flight.  Ends without a block barrier: the caller synchronises.
template <bool MOVING = false>
__device__ __forceinline__ void stage_points(float2 *dst, const float2 *__restrict__ pts,
                                             const float2 *__restrict__ vel, const uint8_t *__restrict__ mask,
                                             int base, int n, int t0, int nt, unsigned long long *bar,
                                             unsigned *uses, int *err) {
    const float qnan = __int_as_float(0x7fffffff);
    const bool aligned = ((uintptr_t)(pts + base) & 15u) == 0;
    if (!MOVING && aligned) {
        const int nb = n & ~1;   // points moved by the bulk copy (a multiple of 16 bytes)
        const unsigned parity = *uses & 1u;   // the phase this copy completes
        if (t0 == 0 && nb > 0) {
            fence_proxy_async_smem();   // earlier reads of the stage come before the copy's writes
            mbar_arrive_expect_tx(bar, (unsigned)nb * sizeof(float2));
            bulk_copy_g2s(dst, pts + base, (unsigned)nb * sizeof(float2), bar);
        }
        if (t0 == 0 && nb < n) dst[nb] = __ldg(pts + base + nb);
        asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");   // every thread has read *uses
        if (nb > 0) {
            if (!mbar_wait(bar, parity)) {
                report_error(err, EXACT_ETIMEOUT);
                mbar_wait(bar, parity);   // once more for the copy still in flight, then go on
            }
            if (t0 == 0) *uses += 1u;   // read again only after the caller's block barrier
        }
    } else if (MOVING) {   // positions and velocities are 8-byte aligned (checked by the host)
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (int i = t0; i < n; i += nt) {
            cp_async8(&d4[i].x, pts + base + i);
            cp_async8(&d4[i].z, vel + base + i);
        }
        cp_async_wait_all();
    } else {
        for (int i0 = t0; i0 < n; i0 += 8 * nt) {   // static cloud, source only 8-byte aligned
            float2 p[8], v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * nt;
                p[k] = i < n ? __ldg(pts + base + i) : make_float2(0.f, 0.f);
                if constexpr (MOVING) v[k] = i < n ? __ldg(vel + base + i) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * nt;
                if (i < n) {
                    if constexpr (MOVING)
                        reinterpret_cast<float4 *>(dst)[i] = make_float4(p[k].x, p[k].y, v[k].x, v[k].y);
                    else
                        dst[i] = p[k];
                }
            }
        }
    }
    if (mask) {
        // after the copies: masked points become NaN (every evaluator turns
        // them into a +inf key); a point's copy and its overwrite are made by
        // the same thread, or ordered by the completed wait (bulk copy) and
        // the named barrier (odd last point)
        for (int i = t0; i < n; i += nt)
            if (!__ldg(mask + base + i)) {
                if constexpr (MOVING) {
                    reinterpret_cast<float4 *>(dst)[i].x = qnan;
                    reinterpret_cast<float4 *>(dst)[i].y = qnan;
                } else {
                    dst[i] = make_float2(qnan, qnan);
                }
            }
    }
}

// Float-float numbers hi + lo (|lo| <= ulp(hi) / 2, about 48 significant
// bits) for the cost sums: the terms are large (w_coll, w_inf scale) and are
// summed over the horizon, which needs more than float precision; FP64 would
// give it, but a dependent FP64 operation takes about 65 cycles on this GPU
// against under 5 for FP32.  two_sum is Knuth's error-free sum; ff_add adds
// the low parts and renormalises with Dekker's fast two-sum.  Both are
// commutative bit for bit, so a butterfly reduction leaves the same value on
// every lane.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return ff{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo), h = s.hi + e;
    return ff{h, e - (h - s.hi)};
}
__device__ __forceinline__ ff ff_add(ff a, float b) { return ff_add(a, ff{b, 0.f}); }
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff warp_sum_ff(ff a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        a = ff_add(a, ff{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
    return a;
}

// acc + phi_obs(d) (Sec. IV-E): w_coll I(d < 0) + w_rep max(d_safe - d, 0)^2,
// the gap exact as a float-float and its square and product kept to about
// 48 bits.  A non-finite d adds nothing.
__device__ __forceinline__ ff add_phi_obs(const MppiP &P, float d, ff acc) {
    if (d < 0.f) acc = ff_add(acc, P.w_coll);
    const ff g = two_sum(P.d_safe, -d);
    if (g.hi > 0.f) {
        const float p = g.hi * g.hi, pe = fmaf(g.hi, g.hi, -p) + 2.f * g.hi * g.lo;
        const float q = P.w_rep * p, qe = fmaf(P.w_rep, p, -q) + P.w_rep * pe;
        acc = ff_add(acc, ff{q, qe});
    }
    return acc;
}

struct SampleSmem {
    float4 circ[kStage / kSub];            // sub-chunk bounding circles
    unsigned msk[2 * EXACT_MAX_HORIZON];   // kept (step, sub-chunk) pairs, 64 bits per step
    int pre[EXACT_MAX_HORIZON + 1];        // exclusive prefix of their counts
    union {
        int queue[kQueueAll];              // per-warp queues of kept (step, point) entries
        float4 circf[kStage / kFine];      // fine sub-chunk circles (rectangle covers)
    };
    int qfine[kQueueFine];                 // per-warp queues of kept (step, fine sub-chunk) entries
    float4 cw[EXACT_MAX_HORIZON];      // footprint circle centre (world) and t_h per step
    float4 pose[EXACT_MAX_HORIZON];
    float stage[EXACT_MAX_HORIZON];
    unsigned key[EXACT_MAX_HORIZON];
    unsigned long long bar;            // mbarrier of the bulk copies that stage the points
    unsigned bar_uses;                 // its completed phases
    float term[2];
    bool last;
};

// Every kernel that runs sample_body starts with this (thread 0 initialises
// the staging mbarrier; all threads then pass a block barrier).
__device__ __forceinline__ void sample_smem_init(SampleSmem &sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        sm.bar_uses = 0u;
    }
    __syncthreads();
}

// Horizon part p of sample r of a scene (steps [p T / parts, (p+1) T / parts)).
// s_pts holds min(N, kStage) points; when `staged` is true the first chunk
// is already there (same scene as the block's previous sample) and is not
// reloaded.  With several parts, each publishes its per-step keys and the
// last part of the sample (atomic ticket) gathers the others' and forms J~
// exactly as a single block would (same per-step data, same summation
// order), so the split never changes a bit of the result.  Ends with a
// __syncthreads.  MOVING: V.vel holds the points' velocities and every step
// sees the predicted cloud (see steps_min_keys).
// circ: bounding circles of the 64-point sub-chunks of an ordered cloud
// (cloud_circles), or NULL.  (Kept out of SceneView: a larger SceneView
// parameter block made the compiler spill in the large-footprint kernels.)
// r2 >= 0: the block takes a second sample r2 of the same scene (parts == 1,
// 2T <= EXACT_MAX_HORIZON, blockDim >= 96): warps 0 and 1 roll the two out
// side by side, the per-step slots hold sample r's steps then r2's (slot
// s T + h), one pass over the staged points serves both, and warps 0 and 1
// form the two J~.  Each sample's J~ takes exactly the operations of the
// one-sample path.
template <bool MOVING = false, int PATH = kPathAny, class EV>
__device__ __forceinline__ void sample_body(const SceneView &V, const EV &ev, int r, int p, SampleSmem &sm,
                                            float2 *s_pts, bool staged, int pairs_per_lane,
                                            const float4 *circ = nullptr, int r2 = -1) {
    const MppiP &P = V.P;
    const int T = P.T, nu = P.nu, N = V.N;
    constexpr int kS = stage_points_of<MOVING>();
    const int ns = r2 >= 0 ? 2 : 1;   // samples in this block
    const int h0 = (p * T) / V.parts, h1 = ((p + 1) * T) / V.parts;
    const int k0 = ns == 2 ? 0 : h0, nk = ns == 2 ? 2 * T : h1 - h0;   // step slots [k0, k0 + nk)
    for (int h = k0 + (int)threadIdx.x; h < k0 + nk; h += blockDim.x) sm.key[h] = f2ord(finf());
    if (r == 0 && p == 0 && threadIdx.x == 0 &&
        !(isfinite(V.state[0]) && isfinite(V.state[1]) && isfinite(V.state[2])))
        report_error(V.err, EXACT_EINVAL);   // a start state the host could not see is not finite
    const int n0 = min(N, kS);
    const float3 bc = ev.bound();
    const int warp = threadIdx.x >> 5;
    if (warp < ns) {
        const int rs = warp == 0 ? r : r2, off = warp * T;
        const float *U = V.U;
        const float *eps = V.noise + (size_t)rs * T * nu;
        LaneRollout R;
        warp_rollout(P, V.state[0], V.state[1], V.state[2],
                     [&](int h, int j) { return clamp_u(P, j, U[h * nu + j] + eps[h * nu + j]); }, R);
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int e = 0; e < kMaxPerLane; ++e) {
            const int h = lane * R.per + e;
            if (e < R.per && h < T) {
                float sn, cs;
                sincosf(R.th[e], &sn, &cs);
                sm.pose[off + h] = make_float4(R.x[e], R.y[e], cs, sn);
                sm.cw[off + h] = make_float4(fmaf(cs, bc.x, fmaf(-sn, bc.y, R.x[e])),
                                             fmaf(sn, bc.x, fmaf(cs, bc.y, R.y[e])),
                                             (float)(h + P.state_offset) * P.dt, 0.f);
                const float u2 = fmaf(R.u[e][0], R.u[e][0], fmaf(R.u[e][1], R.u[e][1], R.u[e][2] * R.u[e][2]));
                sm.stage[off + h] = fmaf(P.w_goal, guidance_dist(R.x[e], R.y[e], V.wp, V.W), P.w_ctrl * u2);
            }
        }
        if (lane == 0) sm.term[warp] = P.w_term * guidance_dist(R.qTx, R.qTy, V.wp, V.W);
        grid_dep_wait();   // launched early behind a cloud-ordering kernel: the cloud is ready now
    } else {
        grid_dep_wait();
        if (!staged)
            stage_points<MOVING>(s_pts, V.pts, V.vel, V.mask, 0, n0, threadIdx.x - 32 * ns, blockDim.x - 32 * ns, &sm.bar,
                                 &sm.bar_uses, V.err);
    }
    __syncthreads();
    const bool prune = PATH == kPathAny && !V.dmin && N >= kPruneMin;
    // sub-chunk circles: copied from the ordered cloud's (64-point sub-chunks),
    // or computed from the staged points
    const bool pre_circ = circ != nullptr && pairs_per_lane == 1;
    // rectangle covers test the fine sub-chunks of the kept sub-chunks too
    // (polygons test single points instead; see steps_min_keys)
    const bool fine = pre_circ && !EV::kBoxTest;
    const float4 *circ_f = fine ? circ + fine_circle_offset(N) : nullptr;
    if (!staged && prune) {
        if (pre_circ)
            for (int s = threadIdx.x; s < (n0 + kSub - 1) / kSub; s += blockDim.x) sm.circ[s] = circ[s];
        else
            chunk_circles<MOVING>(s_pts, n0, sm.circ, pairs_per_lane);
        if (fine)
            for (int s = threadIdx.x; s < (n0 + kFine - 1) / kFine; s += blockDim.x) sm.circf[s] = circ_f[s];
        __syncthreads();
    }
    // without a d_min output the costs only need min(d_min, d_safe): far
    // sub-chunks (clouds of kPruneMin points or more) or far points (smaller
    // clouds, one pass) are skipped
    const float cap = V.dmin ? -1.f : fmaxf(P.d_safe, 0.f);
    steps_min_keys<MOVING, PATH>(ev, s_pts, n0, sm.pose, sm.cw, k0, nk, sm.key, pairs_per_lane, sm.circ, cap, sm.msk,
                                 sm.pre, sm.queue, !V.dmin && N < kPruneMin, fine ? sm.circf : nullptr, sm.qfine,
                                 V.err);
    if constexpr (PATH == kPathAny) for (int base = kS; base < N; base += kS) {   // clouds larger than the stage
        const int n = min(kS, N - base);
        __syncthreads();
        stage_points<MOVING>(s_pts, V.pts, V.vel, V.mask, base, n, threadIdx.x, blockDim.x, &sm.bar, &sm.bar_uses,
                             V.err);
        __syncthreads();
        if (prune) {
            if (pre_circ)
                for (int s = threadIdx.x; s < (n + kSub - 1) / kSub; s += blockDim.x) sm.circ[s] = circ[base / kSub + s];
            else
                chunk_circles<MOVING>(s_pts, n, sm.circ, pairs_per_lane);
            if (fine)
                for (int s = threadIdx.x; s < (n + kFine - 1) / kFine; s += blockDim.x)
                    sm.circf[s] = circ_f[base / kFine + s];
            __syncthreads();
        }
        steps_min_keys<MOVING>(ev, s_pts, n, sm.pose, sm.cw, k0, nk, sm.key, pairs_per_lane, sm.circ, cap, sm.msk,
                               sm.pre, sm.queue, false, fine ? sm.circf : nullptr, sm.qfine, V.err);
    }
    grid_dep_release();
    __syncthreads();
    if (V.parts > 1) {
        for (int h = h0 + (int)threadIdx.x; h < h1; h += blockDim.x) V.dkey[(size_t)r * T + h] = sm.key[h];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) sm.last = atomicAdd(V.tk + r, 1u) == (unsigned)V.parts - 1;
        __syncthreads();
        if (!sm.last) return;
        __threadfence();
        for (int h = threadIdx.x; h < T; h += blockDim.x)
            if (h < h0 || h >= h1) sm.key[h] = __ldcg(V.dkey + (size_t)r * T + h);
        __syncthreads();
    }
    if (warp < ns) {
        const int rs = warp == 0 ? r : r2, off = warp * T, lane = threadIdx.x & 31;
        ff acc{0.f, 0.f};
        bool unsafe = false;
        for (int h = lane; h < T; h += 32) {
            const float key = ord2f(sm.key[off + h]);
            const float d = key == finf() ? finf() : ev.dist(key);
            if (V.dmin) V.dmin[(size_t)rs * T + h] = d;
            acc = add_phi_obs(P, d, ff_add(acc, sm.stage[off + h]));
            unsafe |= d < P.d_safe;
        }
        acc = warp_sum_ff(acc);
        const bool chi = __any_sync(0xffffffffu, unsafe);
        if (lane == 0) {
            // J~ = J + w_inf I(chi) (Sec. IV-E), summed as a float-float and
            // kept as a double; beta = min J~ is gathered with one 64-bit
            // atomic per sample into the scene's header (complemented key;
            // 0 = empty)
            acc = ff_add(acc, sm.term[warp]);
            if (chi) acc = ff_add(acc, P.w_inf);
            const double jt = ff_to_d(acc);
            V.Jt[rs] = jt;
            atomicMax(&V.hdr->beta_enc, ~d2ord(jt));
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- update phase
struct UpdateSmem {
    float tile[kUpdTile];
    float w[256];
    float f[kUpdBlock / 32];
};

// Chunk b of a scene's samples (blockDim == kUpdBlock): it stages its noise
// rows (contiguous, coalesced, eight loads in flight per thread) before
// waiting for the sample phase, then forms w_r = exp(-(J~_r - beta)/lambda)
// and leaves sum_r w_r eps'_r and sum_r w_r in its partial slot.
__device__ __forceinline__ void update_body(const SceneView &V, int b, UpdateSmem &sm) {
    const MppiP &P = V.P;
    const int K = P.K, T = P.T, nu = P.nu, TN = T * nu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = b * V.upd_chunk, r1 = min(K, r0 + V.upd_chunk), nr = r1 - r0;
    const float *U = V.U;

    // the validation launch may place its blocks now: they read the nominal
    // and then wait for this grid (PDL lets them in only once every block of
    // this grid has started, so they never take a slot this grid needs)
    grid_dep_release();
    const float *src = V.noise + (size_t)r0 * TN;
    const int n = nr * TN;
    bool finite = true;
    for (int i0 = tid; i0 < n; i0 += 8 * kUpdBlock) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k * kUpdBlock;
            v[k] = i < n ? __ldg(src + i) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k * kUpdBlock;
            if (i < n) {
                const int e = i % TN;
                finite &= isfinite(v[k]);
                sm.tile[i] = P.clamp ? clamp_u(P, e % nu, U[e] + v[k]) - U[e] : v[k];
            }
        }
    }
    if (b == 0)
        for (int e = tid; e < TN; e += kUpdBlock) finite &= isfinite(U[e]);
    if (!finite) report_error(V.err, EXACT_EINVAL);   // non-finite noise or nominal (device data)
    grid_dep_wait();   // J~ and beta come from the sample phase
    const double beta = ord2d(~V.hdr->beta_enc);
    if (V.parts > 1)   // the sample phase is over: rearm its per-sample part tickets
        for (int i = tid; i < nr; i += kUpdBlock) V.tk[r0 + i] = 0u;
    float z = 0.f;
    for (int i = tid; i < nr; i += kUpdBlock) {
        const float w = expf(-(float)(V.Jt[r0 + i] - beta) / P.lambda);
        sm.w[i] = w;
        V.wt[r0 + i] = w;
        z += w;
    }
    z = warp_sum_f(z);
    if (lane == 0) sm.f[warp] = z;
    __syncthreads();
    float *part = V.part + (size_t)b * (TN + 1);
    for (int e = tid; e < TN; e += kUpdBlock) {
        float a0 = 0.f, a1 = 0.f;
        int i = 0;
        for (; i + 1 < nr; i += 2) {
            a0 = fmaf(sm.w[i], sm.tile[i * TN + e], a0);
            a1 = fmaf(sm.w[i + 1], sm.tile[(i + 1) * TN + e], a1);
        }
        if (i < nr) a0 = fmaf(sm.w[i], sm.tile[i * TN + e], a0);
        part[e] = a0 + a1;
    }
    if (tid == 0) {
        float zb = 0.f;
        for (int w = 0; w < kUpdBlock / 32; ++w) zb += sm.f[w];
        part[TN] = zb;
    }
}

// ---------------------------------------------------------------- validation
constexpr int kRedSlices = kBlock / 32;   // slot slices of the partial reduction

struct ValidateSmem {
    float red[kRedSlices][EXACT_MAX_HORIZON * 3 + 1];
    float U[EXACT_MAX_HORIZON * 3];
    float4 pose;
    float Z;
    float mn[32];
    bool last, ok;
};

// Block (step h, point chunk c) of a scene's validation (blockDim == kBlock).
// Every block adds the update blocks' partial slots itself (fixed order, so
// all blocks hold the same U_upd = U + sum_r w_r eps'_r / sum_r w_r), rolls
// the updated nominal out to its step, and checks the nominal's clearance
// over its chunk of points.  Block 0 also writes U_upd and the blocks share
// out the normalised weights and the costs.  The scene's last block (atomic
// ticket) writes u*, the shifted (last entry repeated) or reset U, the valid
// flag, and empties beta for the next cycle.  When the nominal's cost is
// requested, every block also publishes the minimum key of its chunk of its
// step (one complemented 32-bit order key per step, atomicMax) and the last
// block scores the nominal exactly like a sample (Sec. III-E, IV-E; the cost
// J_m of Algorithm 2) and empties the step keys.
template <bool MOVING = false, class EV>
__device__ __forceinline__ void validate_body(const SceneView &V, const EV &ev, int h, int c, ValidateSmem &sm,
                                              const float4 *circ = nullptr) {
    const MppiP &P = V.P;
    const int K = P.K, T = P.T, nu = P.nu, TN = T * nu, G = V.upd_blocks;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblocks = T * V.val_chunks, self = h * V.val_chunks + c;
    if (!EXACT_DCHECK(h < T && c < V.val_chunks, V.err)) return;   // debug build: a block outside the table
    // the nominal U and the start state stay unchanged until this kernel's
    // last block: read them while the update phase drains
    for (int e = tid; e < TN; e += kBlock) sm.U[e] = V.U[e];
    grid_dep_wait();   // the partial slots come from the update phase
    grid_dep_release();   // a dependent launch (the hybrid selection) waits for this grid's end anyway

    // partial slots: warp w adds slots w, w + 8, ... for every element (and
    // Z), in that order, with four loads in flight
    for (int e = lane; e <= TN; e += 32) {
        const float *src = V.part + e;
        const size_t st = (size_t)kRedSlices * (TN + 1);
        float a = 0.f;
        int q = warp;
        for (; q + 3 * kRedSlices < G; q += 4 * kRedSlices) {
            const float *b = src + (size_t)q * (TN + 1);
            const float x0 = __ldcg(b), x1 = __ldcg(b + st), x2 = __ldcg(b + 2 * st), x3 = __ldcg(b + 3 * st);
            a += x0;
            a += x1;
            a += x2;
            a += x3;
        }
        for (; q < G; q += kRedSlices) a += __ldcg(src + (size_t)q * (TN + 1));
        sm.red[warp][e] = a;
    }
    __syncthreads();
    if (tid == 0) {
        float z = 0.f;
        for (int w = 0; w < kRedSlices; ++w) z += sm.red[w][TN];
        sm.Z = z;
    }
    __syncthreads();
    const float invZ = 1.f / sm.Z;
    for (int e = tid; e < TN; e += kBlock) {
        float a = 0.f;
        for (int w = 0; w < kRedSlices; ++w) a += sm.red[w][e];
        const float v = sm.U[e] + a * invZ;
        sm.U[e] = v;
        if (self == 0 && V.U_upd_out) V.U_upd_out[e] = v;
    }
    __syncthreads();
    if (warp == 0) {   // the nominal's rollout on warp 0, the other warps share out the outputs
        LaneRollout R;
        warp_rollout(P, V.state[0], V.state[1], V.state[2], [&](int hh, int j) { return clamp_u(P, j, sm.U[hh * nu + j]); },
                     R);
#pragma unroll
        for (int q = 0; q < kMaxPerLane; ++q) {
            if (q < R.per && lane * R.per + q == h) {
                float sn, cs;
                sincosf(R.th[q], &sn, &cs);
                sm.pose = make_float4(R.x[q], R.y[q], cs, sn);
            }
        }
    } else if (V.weights || V.costs) {
        const int r0 = (int)(((long long)K * self) / nblocks), r1 = (int)(((long long)K * (self + 1)) / nblocks);
        for (int r = r0 + tid - 32; r < r1; r += kBlock - 32) {
            if (V.weights) V.weights[r] = __ldcg(V.wt + r) * invZ;
            if (V.costs) V.costs[r] = (float)V.Jt[r];
        }
    }
    __syncthreads();
    const float4 qp = sm.pose;
    const int N = V.N;
    const int npairs = (N + 1) >> 1;
    const int pend = min(npairs, (c + 1) * kValChunkPairs);
    const float th = (float)(h + P.state_offset) * P.dt;   // time of the scored state (MOVING)
    // ordered clouds: skip 64-point sub-chunks farther than d_safe from the
    // footprint (the validation and the nominal's cost only need min(d, d_safe))
    const float3 bc = ev.bound();
    const float cwx = fmaf(qp.z, bc.x, fmaf(-qp.w, bc.y, qp.x)), cwy = fmaf(qp.w, bc.x, fmaf(qp.z, bc.y, qp.y));
    const float vlim = fmaxf(P.d_safe, 0.f) + kPruneSlack + 1e-5f * (fabsf(cwx) + fabsf(cwy));
    float best = finf();
    for (int j = c * kValChunkPairs + tid; j < pend; j += kBlock) {
        if (circ) {   // warp-uniform: the warp's 32 pairs are sub-chunk j / 32
            const float4 cc = __ldg(circ + (j >> 5));
            const float dx = cc.x - cwx, dy = cc.y - cwy;
            float reach = cc.z + bc.z + 1e-5f * (fabsf(cc.x) + fabsf(cc.y));
            if (MOVING) reach = fmaf(th, cc.w, reach);
            const float far = reach + vlim;
            if (cc.z < 0.f || fmaf(dx, dx, dy * dy) > far * far) continue;
        }
        const int i0 = 2 * j, i1 = min(2 * j + 1, N - 1);
        float2 o0 = __ldg(V.pts + i0);
        float2 o1 = __ldg(V.pts + i1);
        if constexpr (MOVING) {
            const float2 v0 = __ldg(V.vel + i0), v1 = __ldg(V.vel + i1);
            o0 = make_float2(fmaf(th, v0.x, o0.x), fmaf(th, v0.y, o0.y));
            o1 = make_float2(fmaf(th, v1.x, o1.x), fmaf(th, v1.y, o1.y));
        }
        float px0, py0, px1, py1;
        body_frame(o0.x, o0.y, qp.x, qp.y, qp.z, qp.w, px0, py0);
        body_frame(o1.x, o1.y, qp.x, qp.y, qp.z, qp.w, px1, py1);
        float k0, k1;
        ev.eval2(px0, py0, px1, py1, k0, k1);
        if (V.mask) {
            k0 = __ldg(V.mask + i0) ? k0 : finf();
            k1 = __ldg(V.mask + i1) ? k1 : finf();
        }
        best = fmin3(best, k0, k1);
    }
    best = warp_min_f(best);
    if (lane == 0) sm.mn[warp] = best;
    __syncthreads();
    if (tid == 0) {
        float b = sm.mn[0];
        for (int w = 1; w < kBlock / 32; ++w) b = fminf(b, sm.mn[w]);
        const float d = b == finf() ? finf() : ev.dist(b);
        const bool bad = !(d >= P.d_safe);
        if (V.nom_cost) atomicMax(V.vkey + h, ~f2ord(b));
        __threadfence();
        // one 64-bit ticket: finished blocks in the low word, failed ones in
        // the high word, so the last block learns the outcome from its own
        // atomic
        const unsigned long long t = atomicAdd(&V.hdr->vticket, bad ? 0x100000001ull : 1ull);
        sm.last = (unsigned)t == (unsigned)nblocks - 1;
        sm.ok = (t >> 32) == 0ull && !bad;
    }
    __syncthreads();
    if (!sm.last) return;
    __threadfence();
    const int ok = sm.ok ? 1 : 0;
    for (int e = tid; e < TN; e += kBlock) {
        const float v = sm.U[e];
        if (e < nu && V.u_star) V.u_star[e] = ok ? v : 0.f;
        V.U[e] = ok ? (e + nu < TN ? sm.U[e + nu] : v) : 0.f;
    }
    if (tid == 0) {
        if (V.valid) *V.valid = ok;
        V.hdr->bad = ok ? 0 : 1;
        V.hdr->beta_enc = 0ull;
    }
    if (V.nom_cost && warp == 0) {
        LaneRollout R;
        warp_rollout(P, V.state[0], V.state[1], V.state[2], [&](int hh, int j) { return clamp_u(P, j, sm.U[hh * nu + j]); },
                     R);
        ff acc{0.f, 0.f};
#pragma unroll
        for (int e = 0; e < kMaxPerLane; ++e) {
            const int hh = lane * R.per + e;
            if (e < R.per && hh < T) {
                const float u2 = fmaf(R.u[e][0], R.u[e][0], fmaf(R.u[e][1], R.u[e][1], R.u[e][2] * R.u[e][2]));
                const float stage = fmaf(P.w_goal, guidance_dist(R.x[e], R.y[e], V.wp, V.W), P.w_ctrl * u2);
                const float key = ord2f(~atomicExch(V.vkey + hh, 0u));
                const float d = key == finf() ? finf() : ev.dist(key);
                acc = add_phi_obs(P, d, ff_add(acc, stage));
            }
        }
        acc = warp_sum_ff(acc);
        if (lane == 0)
            *V.nom_cost = (float)ff_to_d(ff_add(acc, P.w_term * guidance_dist(R.qTx, R.qTy, V.wp, V.W)));
    }
}

}  // namespace exact
