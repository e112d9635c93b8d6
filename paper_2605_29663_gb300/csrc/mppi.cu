// mppi.cu -- mppi_step: one batched EXACT-MPPI control cycle (Algorithm 1).
//
// Three kernels, stream-ordered (and capturable in one CUDA graph):
//   A  mppi_sample_kernel   one block per sample r: warp 0 rolls the sample
//                           out (two warp prefix scans) while the other warps
//                           stage the obstacle points in shared memory; then
//                           every (step, point) body-frame signed distance
//                           with per-step minima in shared memory; then
//                           phi_task + phi_ctrl + phi_obs (double), chi, J.
//   B1 mppi_update_kernel   ceil(K / 128) blocks: beta = min J~ (each block
//                           reduces all K in double), the softmax weights of
//                           its samples and their weighted clipped noise; the
//                           last block (atomic ticket) sums the partials,
//                           writes U_upd and rolls the updated nominal out.
//   B2 mppi_validate_kernel one block per (step, point chunk) of the nominal:
//                           d_min >= d_safe; the last block writes u*, the
//                           shifted or reset U and the valid flag.
// No K x T x N intermediate touches memory; the scratch is per-sample J /
// chi / weights, per-block partial sums and per-step nominal data in the
// context arena.  No block ever waits for another (tickets only).
#include "internal.h"
#include "mppi_common.cuh"

namespace exact {

constexpr int kUpdBlock = 256;
constexpr int kUpdTile = 8192;    // floats of noise one update block stages (32 KB)
constexpr int kStage = 4096;      // obstacle points staged in shared memory per pass

struct MppiScratch {
    ArenaHeader *hdr;   // beta, tickets, validation flag (fixed offset)
    double *Jt;         // K   J~ = J + w_inf I(chi)
    float *wt;          // K   unnormalised weights exp(-(J~ - beta)/lambda)
    float *part;        // G x (T*nu + 1)   per-block weighted noise sums and Z
    float *U_upd;       // T x nu
    float4 *nom_pose;   // T   scored nominal states (x, y, cos, sin)
};

// samples per update block: the block's noise tile fits kUpdTile floats
static int upd_chunk(int T, int nu) {
    const int c = kUpdTile / (T * nu);
    return c < 1 ? 1 : (c > 256 ? 256 : c);
}
static int upd_blocks(int K, int T, int nu) {
    const int c = upd_chunk(T, nu);
    return (K + c - 1) / c;
}

size_t mppi_scratch_bytes(int K, int T) {
    size_t b = kArenaHeader;
    b += align_up((size_t)K * sizeof(double), 256);
    b += align_up((size_t)K * sizeof(float), 256);
    b += align_up((size_t)upd_blocks(K, T, 3) * (T * 3 + 1) * sizeof(float), 256);   // G is largest for n_u = 3
    b += align_up((size_t)T * 3 * sizeof(float), 256);
    b += align_up((size_t)T * sizeof(float4), 256);
    return b;
}

static MppiScratch carve(void *base, int K, int T) {
    char *p = static_cast<char *>(base);
    MppiScratch s;
    s.hdr = reinterpret_cast<ArenaHeader *>(p); p += kArenaHeader;
    s.Jt = reinterpret_cast<double *>(p); p += align_up((size_t)K * sizeof(double), 256);
    s.wt = reinterpret_cast<float *>(p); p += align_up((size_t)K * sizeof(float), 256);
    s.part = reinterpret_cast<float *>(p); p += align_up((size_t)upd_blocks(K, T, 3) * (T * 3 + 1) * sizeof(float), 256);
    s.U_upd = reinterpret_cast<float *>(p); p += align_up((size_t)T * 3 * sizeof(float), 256);
    s.nom_pose = reinterpret_cast<float4 *>(p);
    return s;
}

// Order-preserving map of a double onto uint64 (total order).
__device__ __forceinline__ unsigned long long d2ord(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord2d(unsigned long long u) {
    return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

constexpr int kPairsPerLane = 4;   // point pairs one lane evaluates per work item

// Per-step minimum of the body-frame key over n staged points for the T
// poses in shared memory.  Work items (step h, chunk of 32 * kPairsPerLane
// point pairs) are dealt to the block's warps round-robin; each item ends in
// one warp shuffle-min and one shared-memory atomicMin on the
// order-preserving key of step h.  A ragged last pair repeats its first
// point.  Masked points were staged as NaN, which every evaluator turns into
// a +inf key (NaN terms are dropped by min, and the canonical NaN has a
// clear sign bit, so it never toggles the crossing parity).
template <class FPC>
__device__ __forceinline__ void steps_min_keys(const FPC &fpc, const float2 *pts, int n, const float4 *pose,
                                               int T, unsigned *keyh) {
    const int npairs = (n + 1) >> 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    constexpr int span = 32 * kPairsPerLane;
    const int nchunk = npairs > 0 ? (npairs + span - 1) / span : 0;
    const int items = T * nchunk;
    for (int it = warp; it < items; it += nwarps) {
        const int h = it / nchunk, c = it - h * nchunk;
        const float4 q = pose[h];
        float best = finf();
        const int jend = min(npairs, (c + 1) * span);
        for (int j = c * span + lane; j < jend; j += 32) {
            const float2 o0 = pts[2 * j];
            const float2 o1 = pts[min(2 * j + 1, n - 1)];
            float px0, py0, px1, py1;
            body_frame(o0.x, o0.y, q.x, q.y, q.z, q.w, px0, py0);
            body_frame(o1.x, o1.y, q.x, q.y, q.z, q.w, px1, py1);
            float k0, k1;
            eval2(fpc, px0, py0, px1, py1, k0, k1);
            best = fmin3(best, k0, k1);
        }
        best = warp_min_f(best);
        if (lane == 0) atomicMin(keyh + h, f2ord(best));
    }
}

// Copy points [base, base + n) into shared memory, masked ones as NaN.
// Eight loads per thread are in flight before the first store.
__device__ __forceinline__ void stage_points(float2 *dst, const float2 *__restrict__ pts,
                                             const uint8_t *__restrict__ mask, int base, int n, int t0, int nt) {
    const float qnan = __int_as_float(0x7fffffff);
    for (int i0 = t0; i0 < n; i0 += 8 * nt) {
        float2 p[8];
        bool ok[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k * nt;
            p[k] = i < n ? __ldg(pts + base + i) : make_float2(0.f, 0.f);
            ok[k] = i < n && (!mask || __ldg(mask + base + i));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k * nt;
            if (i < n) dst[i] = ok[k] ? p[k] : make_float2(qnan, qnan);
        }
    }
}

// phi_obs (Sec. IV-E) in double: its terms are large (w_coll, w_inf scale)
// and are summed over the horizon.
__device__ __forceinline__ double phi_obs_d(const MppiP &P, float d) {
    const double gap = fmax((double)P.d_safe - (double)d, 0.0);
    return (d < 0.f ? (double)P.w_coll : 0.0) + (double)P.w_rep * gap * gap;
}

template <class FPC>
__global__ void __launch_bounds__(kBlock)
mppi_sample_kernel(const MppiP P, const FPC fpc, const float *__restrict__ state,
                   const float2 *__restrict__ pts, const uint8_t *__restrict__ mask, int N,
                   const float *__restrict__ wp, int W, const float *__restrict__ U,
                   const float *__restrict__ noise, double *__restrict__ Jt_out, float *__restrict__ dmin_out,
                   ArenaHeader *__restrict__ hdr) {
    extern __shared__ float2 s_pts[];            // min(N, kStage) staged points
    __shared__ float4 s_pose[EXACT_MAX_HORIZON];
    __shared__ float s_stage[EXACT_MAX_HORIZON];
    __shared__ unsigned s_key[EXACT_MAX_HORIZON];
    __shared__ float s_term;
    const int r = blockIdx.x;
    const int T = P.T, nu = P.nu;
    for (int h = threadIdx.x; h < T; h += blockDim.x) s_key[h] = f2ord(finf());
    if (r == 0 && threadIdx.x == 0) {
        // the update and validation kernels that follow on the stream count
        // finished blocks on these tickets; start them from zero every cycle
        hdr->ticket[0] = 0u;
        hdr->ticket[1] = 0u;
        hdr->bad = 0;
    }

    const int n0 = min(N, kStage);
    if (threadIdx.x < 32) {
        const float *eps = noise + (size_t)r * T * nu;
        LaneRollout R;
        warp_rollout(P, state[0], state[1], state[2],
                     [&](int h, int j) { return clamp_u(P, j, U[h * nu + j] + eps[h * nu + j]); }, R);
        const int lane = threadIdx.x;
#pragma unroll
        for (int e = 0; e < kMaxPerLane; ++e) {
            const int h = lane * R.per + e;
            if (e < R.per && h < T) {
                float sn, cs;
                sincosf(R.th[e], &sn, &cs);
                s_pose[h] = make_float4(R.x[e], R.y[e], cs, sn);
                const float u2 = fmaf(R.u[e][0], R.u[e][0], fmaf(R.u[e][1], R.u[e][1], R.u[e][2] * R.u[e][2]));
                s_stage[h] = fmaf(P.w_goal, guidance_dist(R.x[e], R.y[e], wp, W), P.w_ctrl * u2);
            }
        }
        if (lane == 0) s_term = P.w_term * guidance_dist(R.qTx, R.qTy, wp, W);
    } else {
        stage_points(s_pts, pts, mask, 0, n0, threadIdx.x - 32, blockDim.x - 32);
    }
    __syncthreads();
    steps_min_keys(fpc, s_pts, n0, s_pose, T, s_key);
    for (int base = kStage; base < N; base += kStage) {   // clouds larger than the stage
        const int n = min(kStage, N - base);
        __syncthreads();
        stage_points(s_pts, pts, mask, base, n, threadIdx.x, blockDim.x);
        __syncthreads();
        steps_min_keys(fpc, s_pts, n, s_pose, T, s_key);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double acc = 0.0;
        bool unsafe = false;
        for (int h = threadIdx.x; h < T; h += 32) {
            const float key = ord2f(s_key[h]);
            const float d = key == finf() ? finf() : key_to_dist(fpc, key);
            if (dmin_out) dmin_out[(size_t)r * T + h] = d;
            acc += (double)s_stage[h] + phi_obs_d(P, d);
            unsafe |= d < P.d_safe;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const bool chi = __any_sync(0xffffffffu, unsafe);
        if (threadIdx.x == 0) {
            // J~ = J + w_inf I(chi) in double (Sec. IV-E); beta = min J~ is
            // gathered with one 64-bit atomic per sample (the arena header
            // holds its complement, reset to 0 when the cycle ends)
            const double jt = acc + (double)s_term + (chi ? (double)P.w_inf : 0.0);
            Jt_out[r] = jt;
            atomicMax(&hdr->beta_enc, ~d2ord(jt));
        }
    }
}

// B1: block b owns `chunk` consecutive samples, sized so that their noise
// rows (chunk x T x n_u floats, contiguous) fit one shared-memory tile that
// the block loads with coalesced reads.  It forms the unnormalised weights
// w_r = exp(-(J~_r - beta)/lambda) of its samples and the sums
// sum_r w_r eps'_r and sum_r w_r, left in its partial slot.  The last block
// to finish (atomic ticket) adds the partials, writes the normalised
// weights, costs and U_upd, and rolls the updated nominal out.
__global__ void __launch_bounds__(kUpdBlock)
mppi_update_kernel(const MppiP P, int chunk, const float *__restrict__ state, const float *__restrict__ U,
                   const float *__restrict__ noise, MppiScratch S, float *__restrict__ costs,
                   float *__restrict__ weights, float *__restrict__ U_upd_out) {
    __shared__ float s_tile[kUpdTile];
    __shared__ float s_w[256];
    __shared__ float s_f[kUpdBlock / 32];
    __shared__ float s_U[EXACT_MAX_HORIZON * 3];
    __shared__ bool s_last;
    __shared__ float s_Z;
    const int K = P.K, T = P.T, nu = P.nu, TN = T * nu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.x * chunk, r1 = min(K, r0 + chunk), nr = r1 - r0;
    const double beta = ord2d(~S.hdr->beta_enc);

    // stage the noise rows of this block's samples (clipped perturbations),
    // eight loads per thread in flight
    const float *src = noise + (size_t)r0 * TN;
    const int n = nr * TN;
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
                s_tile[i] = P.clamp ? clamp_u(P, e % nu, U[e] + v[k]) - U[e] : v[k];
            }
        }
    }
    float z = 0.f;
    for (int i = tid; i < nr; i += kUpdBlock) {
        const float w = expf(-(float)(S.Jt[r0 + i] - beta) / P.lambda);
        s_w[i] = w;
        S.wt[r0 + i] = w;
        z += w;
    }
    z = warp_sum_f(z);
    if (lane == 0) s_f[warp] = z;
    __syncthreads();
    float *part = S.part + (size_t)blockIdx.x * (TN + 1);
    for (int e = tid; e < TN; e += kUpdBlock) {
        float a0 = 0.f, a1 = 0.f;
        int i = 0;
        for (; i + 1 < nr; i += 2) {
            a0 = fmaf(s_w[i], s_tile[i * TN + e], a0);
            a1 = fmaf(s_w[i + 1], s_tile[(i + 1) * TN + e], a1);
        }
        if (i < nr) a0 = fmaf(s_w[i], s_tile[i * TN + e], a0);
        part[e] = a0 + a1;
    }
    if (tid == 0) {
        float zb = 0.f;
        for (int w = 0; w < kUpdBlock / 32; ++w) zb += s_f[w];
        part[TN] = zb;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&S.hdr->ticket[0], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: totals over the G partial slots (four independent sums per thread)
    const int G = gridDim.x;
    if (warp == 0) {
        float zz = 0.f;
        for (int b = lane; b < G; b += 32) zz += __ldcg(S.part + (size_t)b * (TN + 1) + TN);
        zz = warp_sum_f(zz);
        if (lane == 0) s_Z = zz;
    }
    __syncthreads();
    const float invZ = 1.f / s_Z;
    for (int e = tid; e < TN; e += kUpdBlock) {
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
        int b = 0;
        for (; b + 3 < G; b += 4) {
            t0 += __ldcg(S.part + (size_t)b * (TN + 1) + e);
            t1 += __ldcg(S.part + (size_t)(b + 1) * (TN + 1) + e);
            t2 += __ldcg(S.part + (size_t)(b + 2) * (TN + 1) + e);
            t3 += __ldcg(S.part + (size_t)(b + 3) * (TN + 1) + e);
        }
        for (; b < G; ++b) t0 += __ldcg(S.part + (size_t)b * (TN + 1) + e);
        const float v = U[e] + ((t0 + t1) + (t2 + t3)) * invZ;
        s_U[e] = v;
        S.U_upd[e] = v;
        if (U_upd_out) U_upd_out[e] = v;
    }
    if (weights || costs) {
        for (int r = tid; r < K; r += kUpdBlock) {
            if (weights) weights[r] = __ldcg(S.wt + r) * invZ;
            if (costs) costs[r] = (float)S.Jt[r];
        }
    }
    __syncthreads();
    if (warp == 0) {
        LaneRollout R;
        warp_rollout(P, state[0], state[1], state[2], [&](int h, int j) { return clamp_u(P, j, s_U[h * nu + j]); }, R);
#pragma unroll
        for (int q = 0; q < kMaxPerLane; ++q) {
            const int h = lane * R.per + q;
            if (q < R.per && h < T) {
                float sn, cs;
                sincosf(R.th[q], &sn, &cs);
                S.nom_pose[h] = make_float4(R.x[q], R.y[q], cs, sn);
            }
        }
    }
}

// B2: validation of the updated nominal and the final shift / reset.
template <class FPC>
__global__ void __launch_bounds__(kBlock)
mppi_validate_kernel(const MppiP P, const FPC fpc, const float2 *__restrict__ pts,
                     const uint8_t *__restrict__ mask, int N, int chunks, int chunk_pairs, MppiScratch S,
                     float *__restrict__ U, float *__restrict__ u_star, int *__restrict__ valid_out) {
    __shared__ float s_min[kBlock / 32];
    __shared__ bool s_last;
    const int h = blockIdx.x / chunks, chunk = blockIdx.x - h * chunks;
    const float4 q = S.nom_pose[h];
    const int npairs = (N + 1) >> 1;
    const int pend = min(npairs, (chunk + 1) * chunk_pairs);
    float best = finf();
    for (int j = chunk * chunk_pairs + threadIdx.x; j < pend; j += kBlock) {
        const int i0 = 2 * j, i1 = 2 * j + 1;
        const bool has1 = i1 < N;
        const float2 o0 = __ldg(pts + i0);
        const float2 o1 = has1 ? __ldg(pts + i1) : o0;
        float px0, py0, px1, py1;
        body_frame(o0.x, o0.y, q.x, q.y, q.z, q.w, px0, py0);
        body_frame(o1.x, o1.y, q.x, q.y, q.z, q.w, px1, py1);
        float k0, k1;
        eval2(fpc, px0, py0, px1, py1, k0, k1);
        const bool v0 = mask ? __ldg(mask + i0) != 0 : true;
        const bool v1 = has1 && (mask ? __ldg(mask + i1) != 0 : true);
        // a NaN key fails validation (d >= d_safe is false)
        if (v0) best = (k0 == k0) ? fminf(best, k0) : -finf();
        if (v1) best = (k1 == k1) ? fminf(best, k1) : -finf();
    }
    best = warp_min_f(best);
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = s_min[0];
        for (int w = 1; w < kBlock / 32; ++w) b = fminf(b, s_min[w]);
        const float d = b == finf() ? finf() : key_to_dist(fpc, b);
        if (!(d >= P.d_safe)) atomicExch(&S.hdr->bad, 1);
        __threadfence();
        const unsigned t = atomicAdd(&S.hdr->ticket[1], 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int ok = atomicAdd(&S.hdr->bad, 0) == 0;
    const int T = P.T, nu = P.nu, TN = T * nu;
    for (int e = threadIdx.x; e < TN; e += kBlock) {
        const float v = S.U_upd[e];
        if (e < nu && u_star) u_star[e] = ok ? v : 0.f;
        // shift forward, repeating the last entry; or reset to zero
        U[e] = ok ? (e + nu < TN ? S.U_upd[e + nu] : v) : 0.f;
    }
    if (threadIdx.x == 0) {
        if (valid_out) *valid_out = ok;
        S.hdr->beta_enc = 0ull;   // empty for the next cycle's atomicMax
    }
}

}  // namespace exact

using namespace exact;

static int check_params(const exact_mppi_params *p) {
    if (!p) return EXACT_EINVAL;
    if (p->K < 1 || p->T < 1) return EXACT_EINVAL;
    if (p->K > EXACT_MAX_SAMPLES || p->T > EXACT_MAX_HORIZON) return EXACT_ECAPACITY;
    const int want = p->model == EXACT_MM_DIFF || p->model == EXACT_MM_ACKERMANN ? 2
                   : p->model == EXACT_MM_OMNI ? 3
                   : p->model == EXACT_MM_SPIN || p->model == EXACT_MM_PARALLEL ? 1 : -1;
    if (want < 0 || p->n_u != want) return EXACT_EINVAL;
    if (!(p->lambda > 0.f) || !(p->dt > 0.f) || !isfinite(p->lambda) || !isfinite(p->dt)) return EXACT_EINVAL;
    if (p->model == EXACT_MM_ACKERMANN && !(p->wheelbase > 0.f)) return EXACT_EINVAL;
    return EXACT_OK;
}

static MppiP to_device_params(const exact_mppi_params *p) {
    MppiP d;
    d.K = p->K; d.T = p->T; d.nu = p->n_u; d.model = p->model;
    d.dt = p->dt; d.lambda = p->lambda; d.d_safe = p->d_safe;
    d.w_coll = p->w_coll; d.w_rep = p->w_rep; d.w_inf = p->w_inf;
    d.w_goal = p->w_goal; d.w_term = p->w_term; d.w_ctrl = p->w_ctrl; d.wheelbase = p->wheelbase;
    for (int j = 0; j < 3; ++j) { d.u_min[j] = p->u_min[j]; d.u_max[j] = p->u_max[j]; }
    d.clamp = p->clamp; d.state_offset = p->state_offset ? 1 : 0;
    return d;
}

extern "C" int exact_ctx_reserve(exact_ctx *ctx, int max_poses, int max_K, int max_T) {
    if (!ctx || max_poses < 0 || max_K < 0 || max_T < 0) return EXACT_EINVAL;
    size_t need = sdf_scratch_bytes(max_poses);
    const size_t m = mppi_scratch_bytes(max_K, max_T);
    if (m > need) need = m;
    return ensure_scratch(ctx, need);
}

extern "C" int mppi_step(exact_ctx *ctx, const float *state, const float *cloud, const uint8_t *mask,
                         int n_points, const float *waypoints, int n_wp, float *U, const float *noise,
                         const exact_footprint *fp, const exact_mppi_params *params,
                         float *u_star, float *costs, float *weights, int *valid, float *U_upd,
                         float *dmin, void *stream) {
    if (!ctx || !fp || !state || !U || !noise || !waypoints || n_wp < 1 || n_points < 0) return EXACT_EINVAL;
    if (n_points > 0 && (!cloud || ((uintptr_t)cloud & 7u) != 0)) return EXACT_EINVAL;
    int rc = check_params(params);
    if (rc != EXACT_OK) return rc;
    const MppiP P = to_device_params(params);
    rc = ensure_scratch(ctx, mppi_scratch_bytes(P.K, P.T));
    if (rc != EXACT_OK) return rc;
    const MppiScratch S = carve(ctx->scratch, P.K, P.T);
    cudaStream_t st = (cudaStream_t)stream;
    const float2 *pts = reinterpret_cast<const float2 *>(cloud);
    const int npairs = (n_points + 1) / 2;
    const int chunk_pairs = 1024;
    const int chunks = npairs > chunk_pairs ? (npairs + chunk_pairs - 1) / chunk_pairs : 1;
    const size_t smem = (size_t)min(n_points, kStage) * sizeof(float2);
    return with_footprint(fp, [&](auto fpc) -> int {
        using FPC = decltype(fpc);
        mppi_sample_kernel<FPC><<<P.K, kBlock, smem, st>>>(P, fpc, state, pts, mask, n_points, waypoints, n_wp, U,
                                                            noise, S.Jt, dmin, S.hdr);
        mppi_update_kernel<<<upd_blocks(P.K, P.T, P.nu), kUpdBlock, 0, st>>>(P, upd_chunk(P.T, P.nu), state, U,
                                                                             noise, S, costs, weights, U_upd);
        mppi_validate_kernel<FPC><<<P.T * chunks, kBlock, 0, st>>>(P, fpc, pts, mask, n_points, chunks,
                                                                   chunk_pairs, S, U, u_star, valid);
        return cuda_status(cudaGetLastError());
    });
}
