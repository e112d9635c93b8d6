// mppi_kernels.cuh -- the three kernels of one single-scene control cycle
// and their stream-ordered launch, templated on static / predicted
// (time-indexed) obstacle points and on the sample kernel's minimum resident
// blocks per SM (MINB).  MINB = 4 caps the sample kernel at 64 registers:
// four blocks per SM, which pays when the grid spans several waves and the
// footprint is small; otherwise MINB = 0 leaves the register count to the
// compiler (about 120 for these bodies; an explicit minimum of one or two
// blocks changed its choices and measured slower, and so did 512-thread
// blocks for small grids).  mppi.cu instantiates the static uncapped cycle,
// mppi_dense.cu the static capped one and mppi_predicted.cu the predicted
// (capped) one, so the three compile in parallel.
#pragma once
#include "mppi_cycle.cuh"

namespace exact {

template <class FPC, bool MOVING, int MINB, int PATH>
__global__ void __launch_bounds__(kBlock, MINB)
mppi_sample_kernel(const SceneView V, const ConstEval<FPC> ev, const float4 *circ, int pair) {
    extern __shared__ float2 s_pts[];   // min(N, stage) staged points (float4 each when MOVING)
    __shared__ SampleSmem sm;
    sample_smem_init(sm);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the validation kernel that follows on the stream counts its
        // finished blocks on this ticket: start it from zero
        V.hdr->ticket[1] = 0u;
        V.hdr->vticket = 0ull;
        V.hdr->bad = 0;
    }
    // pair: block b takes samples 2b and 2b + 1; else sample b / parts,
    // horizon part b % parts.  Only the register-capped static instantiations
    // carry the two-sample path: in the uncapped ones (large polygons) it cost
    // the compiler spills, and predicted clouds measured slower with it.
    const bool two = MINB != 0 && !MOVING && pair;
    const int r = two ? 2 * (int)blockIdx.x : (int)blockIdx.x / V.parts;
    const int p = two ? 0 : (int)blockIdx.x % V.parts;
    sample_body<MOVING, PATH>(V, ev, r, p, sm, s_pts, false, 1, circ, two && r + 1 < V.P.K ? r + 1 : -1);
}

template <bool MOVING>
__global__ void __launch_bounds__(kUpdBlock) mppi_update_kernel(const SceneView V) {
    __shared__ UpdateSmem sm;
    update_body(V, blockIdx.x, sm);
}

template <class FPC, bool MOVING>
__global__ void __launch_bounds__(kBlock) mppi_validate_kernel(const SceneView V, const ConstEval<FPC> ev,
                                                               const float4 *circ) {
    __shared__ ValidateSmem sm;
    validate_body<MOVING>(V, ev, blockIdx.x / V.val_chunks, blockIdx.x % V.val_chunks, sm, circ);
}

// One block rewrites the cloud in spatial order (see sort_cloud_block) and
// takes the bounding circles of its 64-point sub-chunks and of its 16-point
// fine sub-chunks.
template <bool MOVING>
__global__ void __launch_bounds__(kSortThreads)
cloud_sort_kernel(const float2 *pts, const float2 *vel, const uint8_t *mask, int N, float2 *opts, float2 *ovel,
                  float4 *circ) {
    __shared__ SortSmem sm;
    sort_cloud_block<MOVING>(pts, vel, mask, N, opts, ovel, sm);
    __syncthreads();
    cloud_circles<MOVING>(opts, ovel, N, circ);
}

// Bytes of the spatially ordered cloud copy (points, velocities when
// predicted, sub-chunk and fine sub-chunk circles) that follows a scene's
// scratch in the arena.
inline size_t cloud_copy_bytes(int N, bool moving) {
    return align_up((size_t)N * sizeof(float2), 256) * (moving ? 2 : 1) + circle_bytes(N);
}


// The three launches of one cycle for a scene whose scratch is carved.
// pdl: the sample kernel follows a cloud-ordering kernel and may start early
// (its rollouts do not read the cloud; sample_body waits before staging).
// PATH = kPathPoints: only for footprints whose evaluator prunes point by
// point (ConstEval::kQueueOk), cycles without a d_min output and clouds below
// kPruneMin points.
template <bool MOVING, int MINB, int PATH = kPathAny>
int launch_cycle_t(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                   int sms) {
    const size_t smem = (size_t)min(V.N, stage_points_of<MOVING>()) * (MOVING ? sizeof(float4) : sizeof(float2));
    const int pair = MINB != 0 && !MOVING ? pair_samples(V.P.K, V.P.T, V.parts, sms) : 0;
    const int grid = pair ? (V.P.K + 1) / 2 : V.P.K * V.parts;
    auto launch = [&](auto fpc) -> int {
        using FPC = decltype(fpc);
        const ConstEval<FPC> ev{fpc};
        if (pdl) {
            if (launch_dependent(mppi_sample_kernel<FPC, MOVING, MINB, PATH>, grid, kBlock, smem, st, V, ev, circ,
                                 pair) != cudaSuccess)
                return EXACT_ECUDA;
        } else {
            mppi_sample_kernel<FPC, MOVING, MINB, PATH><<<grid, kBlock, smem, st>>>(V, ev, circ, pair);
            if (cudaGetLastError() != cudaSuccess) return EXACT_ECUDA;
        }
        if (launch_dependent(mppi_update_kernel<MOVING>, V.upd_blocks, kUpdBlock, 0, st, V) != cudaSuccess)
            return EXACT_ECUDA;
        if (launch_dependent(mppi_validate_kernel<FPC, MOVING>, V.P.T * V.val_chunks, kBlock, 0, st, V, ev, circ) !=
            cudaSuccess)
            return EXACT_ECUDA;
        return EXACT_OK;
    };
    if constexpr (PATH == kPathPoints)
        return with_small_footprint(fp, launch);
    else
        return with_footprint(fp, launch);
}

// Any cycle (mppi.cu: picks one of the four below), the static capped cycle
// (mppi_dense.cu) and the predicted cycle (mppi_predicted.cu).  sms is the
// SM count of the device the cycle runs on (it sizes the grids).
int launch_cycle(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                 int sms);
int launch_cycle_dense(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                       int sms);
int launch_cycle_moving(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                        int sms);
// The static capped cycle whose sample kernel holds only the point-level
// pruning (mppi_points.cu): small footprints, no d_min output, N < kPruneMin.
int launch_cycle_points(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                        int sms);

// mppi_step with optional point velocities (NULL: static cloud).
int mppi_step_impl(exact_ctx *ctx, const float *state, const float *cloud, const float *velocity,
                   const uint8_t *mask, int n_points, const float *waypoints, int n_wp, float *U,
                   const float *noise, const exact_footprint *fp, const exact_mppi_params *params, float *u_star,
                   float *costs, float *weights, int *valid, float *U_upd, float *dmin, void *stream);

}  // namespace exact
