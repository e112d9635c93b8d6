// mppi.cu -- mppi_step: one EXACT-MPPI control cycle (Algorithm 1) for one
// robot, as three stream-ordered kernels (capturable in one CUDA graph):
//   mppi_sample_kernel    K x parts blocks (sample_body): warp 0 rolls
//                         the sample out while the other warps stage the
//                         obstacle points in shared memory, then every
//                         (step, point) signed distance that can matter
//                         (far point sub-chunks skipped), then J~; when K
//                         is small each sample's horizon is split over
//                         several blocks (parts) to fill the GPU, and when
//                         K is large the register-capped kernels give each
//                         block two samples (K / 2 blocks).
//   mppi_update_kernel    ceil(K / chunk) blocks (update_body): weights and
//                         weighted clipped noise into per-block partial slots.
//   mppi_validate_kernel  T x ceil(N / 2048) blocks (validate_body): each adds
//                         the partial slots (U_upd), rolls the updated nominal
//                         out to its step and checks its clearance; the last
//                         block writes u*, the shifted or reset U and the
//                         valid flag.
// The update and validation kernels use programmatic dependent launch: each
// starts while its predecessor drains and waits (griddepcontrol) only where
// it reads the predecessor's results.
// The footprint constants are kernel parameters (compile-time edge count).
// No K x T x N intermediate exists; scratch is per-sample J~ / weights,
// per-block partial sums and per-step nominal data in the context arena.
// The kernels live in mppi_kernels.cuh; this file instantiates them for
// static clouds and mppi_predicted.cu for clouds with point velocities.
#include "mppi_kernels.cuh"

namespace exact {

// Statistics of the cycle just run (one block, after the validation): the
// normalised weights' effective sample size, J~ minimum and mean, and the
// validation outcome (the flag the validation blocks left in the header).
__global__ void __launch_bounds__(256)
cycle_stats_kernel(const double *__restrict__ Jt, const float *__restrict__ wt, int K, const ArenaHeader *hdr,
                   exact_cycle_stats *stats) {
    __shared__ double s[4][8];
    double z = 0.0, z2 = 0.0, jsum = 0.0, jmin = 1.0e308;
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
        const double w = wt[r], j = Jt[r];
        z += w;
        z2 += w * w;
        jsum += j;
        jmin = fmin(jmin, j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        z += __shfl_xor_sync(0xffffffffu, z, o);
        z2 += __shfl_xor_sync(0xffffffffu, z2, o);
        jsum += __shfl_xor_sync(0xffffffffu, jsum, o);
        jmin = fmin(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = z; s[1][w] = z2; s[2][w] = jsum; s[3][w] = jmin; }
    __syncthreads();
    if (threadIdx.x == 0) {
        z = s[0][0]; z2 = s[1][0]; jsum = s[2][0]; jmin = s[3][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            z += s[0][k]; z2 += s[1][k]; jsum += s[2][k]; jmin = fmin(jmin, s[3][k]);
        }
        const int bad = *(volatile const int *)&hdr->bad;
        stats->cycles += 1;
        stats->validation_failures += bad ? 1 : 0;
        stats->ess = (float)(z * z / z2);
        stats->cost_min = (float)jmin;
        stats->cost_mean = (float)(jsum / K);
        stats->last_valid = bad ? 0 : 1;
    }
}

static int parts_of(const exact_ctx *ctx, int K, int T) {
    return parts_for(K, T, ctx->sm_count > 0 ? ctx->sm_count : 148);
}

int check_params(const exact_mppi_params *p) {
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

MppiP to_device_params(const exact_mppi_params *p) {
    MppiP d;
    d.K = p->K; d.T = p->T; d.nu = p->n_u; d.model = p->model;
    d.dt = p->dt; d.lambda = p->lambda; d.d_safe = p->d_safe;
    d.w_coll = p->w_coll; d.w_rep = p->w_rep; d.w_inf = p->w_inf;
    d.w_goal = p->w_goal; d.w_term = p->w_term; d.w_ctrl = p->w_ctrl; d.wheelbase = p->wheelbase;
    for (int j = 0; j < 3; ++j) { d.u_min[j] = p->u_min[j]; d.u_max[j] = p->u_max[j]; }
    d.clamp = p->clamp; d.state_offset = p->state_offset ? 1 : 0;
    return d;
}

}  // namespace exact

using namespace exact;

extern "C" int exact_ctx_reserve(exact_ctx *ctx, int max_poses, int max_K, int max_T) {
    return exact_ctx_reserve_cloud(ctx, max_poses, max_K, max_T, 0);
}

extern "C" int exact_ctx_reserve_cloud(exact_ctx *ctx, int max_poses, int max_K, int max_T, int max_points) {
    if (!ctx || max_poses < 0 || max_K < 0 || max_T < 0 || max_points < 0) return EXACT_EINVAL;
    size_t need = sdf_scratch_bytes(max_poses);
    const size_t m = kArenaHeader + scene_scratch_bytes(max_K, max_T, parts_of(ctx, max_K, max_T)) +
                     (max_points >= kPruneMin ? cloud_copy_bytes(max_points, true) : 0);
    if (m > need) need = m;
    return ensure_scratch(ctx, need);
}

namespace exact {

int mppi_step_impl(exact_ctx *ctx, const float *state, const float *cloud, const float *velocity,
                   const uint8_t *mask, int n_points, const float *waypoints, int n_wp, float *U,
                   const float *noise, const exact_footprint *fp, const exact_mppi_params *params, float *u_star,
                   float *costs, float *weights, int *valid, float *U_upd, float *dmin, void *stream) {
    if (!ctx || !fp || !state || !U || !noise || !waypoints || n_wp < 1 || n_points < 0) return EXACT_EINVAL;
    if (n_points > 0 && (!cloud || ((uintptr_t)cloud & 7u) != 0)) return EXACT_EINVAL;
    if (n_points > 0 && velocity && ((uintptr_t)velocity & 7u) != 0) return EXACT_EINVAL;
    int rc = check_params(params);
    if (rc != EXACT_OK) return rc;
    const MppiP P = to_device_params(params);
    const int parts = parts_of(ctx, P.K, P.T);
    // without a d_min output the sample phase prunes; it pays when the cloud
    // is in spatial order, so large clouds get a spatially ordered copy
    const bool sort = !dmin && n_points >= kPruneMin;
    const size_t scene_bytes = kArenaHeader + scene_scratch_bytes(P.K, P.T, parts);
    rc = ensure_scratch(ctx, scene_bytes + (sort ? cloud_copy_bytes(n_points, velocity != nullptr) : 0));
    if (rc != EXACT_OK) return rc;
    SceneView V;
    V.P = P;
    V.state = state;
    V.pts = reinterpret_cast<const float2 *>(cloud);
    V.vel = n_points > 0 ? reinterpret_cast<const float2 *>(velocity) : nullptr;
    V.mask = mask;
    V.N = n_points;
    V.wp = waypoints;
    V.W = n_wp;
    V.U = U;
    V.noise = noise;
    V.u_star = u_star; V.costs = costs; V.weights = weights; V.U_upd_out = U_upd; V.dmin = dmin; V.valid = valid;
    V.nom_cost = nullptr;
    V.err = ctx->d_err;
    V.hdr = reinterpret_cast<ArenaHeader *>(ctx->scratch);
    carve_scene(V, static_cast<char *>(ctx->scratch) + kArenaHeader, P.K, P.T, parts);
    V.upd_chunk = upd_chunk_for(P.K, P.T, P.nu);
    V.upd_blocks = upd_blocks_for(P.K, P.T, P.nu);
    V.val_chunks = val_chunks_for(n_points);
    cudaStream_t st = (cudaStream_t)stream;
    // the per-sample part tickets rearm themselves after each cycle; zero
    // them once whenever the arena layout changes
    const long long layout = ((long long)P.K << 24) ^ ((long long)P.T << 8) ^ V.parts;
    if (V.parts > 1 && ctx->mppi_layout != layout) {
        if (cudaMemsetAsync(V.tk, 0, (size_t)P.K * sizeof(unsigned), st) != cudaSuccess) return EXACT_ECUDA;
    }
    ctx->mppi_layout = layout;
    const float4 *cc = nullptr;
    if (sort) {
        char *q = static_cast<char *>(ctx->scratch) + scene_bytes;
        const size_t pbytes = align_up((size_t)n_points * sizeof(float2), 256);
        float2 *copy = reinterpret_cast<float2 *>(q);
        float2 *vcopy = velocity ? reinterpret_cast<float2 *>(q + pbytes) : nullptr;
        float4 *circ = reinterpret_cast<float4 *>(q + pbytes * (velocity ? 2 : 1));
        if (velocity)
            cloud_sort_kernel<true><<<1, kSortThreads, 0, st>>>(V.pts, V.vel, mask, n_points, copy, vcopy, circ);
        else
            cloud_sort_kernel<false><<<1, kSortThreads, 0, st>>>(V.pts, nullptr, mask, n_points, copy, nullptr, circ);
        if (cudaGetLastError() != cudaSuccess) return EXACT_ECUDA;
        V.pts = copy;
        V.vel = vcopy;
        V.mask = nullptr;
        cc = circ;
    }
    rc = launch_cycle(V, fp, st, sort, cc, ctx->sm_count > 0 ? ctx->sm_count : current_sm_count());
    if (rc != EXACT_OK || !ctx->stats) return rc;
    cycle_stats_kernel<<<1, 256, 0, st>>>(V.Jt, V.wt, P.K, V.hdr, ctx->d_stats);
    return cuda_status(cudaGetLastError());
}

// Clouds with point velocities go to mppi_predicted.cu.  Static clouds go to
// the register-capped kernels when the footprint is small (a rectangle cover
// or at most 16 edges: larger polygons need more registers than the cap
// leaves): those of mppi_points.cu when the cloud is pruned point by point,
// those of mppi_dense.cu when the sample grid exceeds four blocks per SM;
// else to the unbounded ones here.
int launch_cycle(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                 int sms) {
    if (sms <= 0) sms = 148;
    if (V.vel) return launch_cycle_moving(V, fp, st, pdl, circ, sms);
    const bool small_fp = fp->kind == EXACT_FP_RECTS || fp->n_pad <= 16;
    // small clouds without a d_min output are pruned point by point: little
    // evaluation work is left, and the capped kernel's occupancy wins
    const bool queued = !V.dmin && V.N < kPruneMin;
    if (small_fp && queued) return launch_cycle_points(V, fp, st, pdl, circ, sms);
    if (small_fp && (long long)V.P.K * V.parts > 4LL * sms) return launch_cycle_dense(V, fp, st, pdl, circ, sms);
    return launch_cycle_t<false, 0>(V, fp, st, pdl, circ, sms);
}

}  // namespace exact

extern "C" int mppi_step(exact_ctx *ctx, const float *state, const float *cloud, const uint8_t *mask,
                         int n_points, const float *waypoints, int n_wp, float *U, const float *noise,
                         const exact_footprint *fp, const exact_mppi_params *params,
                         float *u_star, float *costs, float *weights, int *valid, float *U_upd,
                         float *dmin, void *stream) {
    return exact::mppi_step_impl(ctx, state, cloud, nullptr, mask, n_points, waypoints, n_wp, U, noise, fp, params,
                                 u_star, costs, weights, valid, U_upd, dmin, stream);
}
