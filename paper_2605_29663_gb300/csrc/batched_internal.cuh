// batched_internal.cuh -- what batched.cu (plan, generic kernels) and
// batched_uniform.cuh (constant-footprint kernels) share: the device scene
// table entry and the batch plan.
#pragma once

#include "mppi_cycle.cuh"

namespace exact {

constexpr int kFpSlots = poly_slot_count(EXACT_MAX_POLY_VERTICES);   // float4 footprint slots
constexpr size_t kHdrStride = 64;                            // bytes between scene headers

struct SceneDev {
    SceneView V;
    const float2 *src_pts;      // the caller's cloud (V.pts may be its spatially ordered copy)
    const uint8_t *src_mask;
    const float4 *circ;         // sub-chunk circles of the ordered copy, or NULL
    int kind, nfp;
    float3 bc;    // footprint bounding circle
    float2 bh;    // half extents of the footprint's bounding box about the circle's centre
    float4 fpc[kFpSlots];
};

// A sample item is (scene, r); bit 30 of r marks an item that also takes
// sample r + 1 of the same scene (see sample_body).
constexpr int kItemPair = 1 << 30;
__device__ __forceinline__ int item_sample(int2 it) { return it.y & (kItemPair - 1); }
__device__ __forceinline__ int item_second(int2 it) { return (it.y & kItemPair) ? (it.y & (kItemPair - 1)) + 1 : -1; }

__device__ __forceinline__ void load_fp(float4 *dst, const SceneDev &D) {
    const int nf = D.kind == EXACT_FP_POLYGON ? poly_slot_count(D.nfp) : D.nfp;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) dst[i] = D.fpc[i];
}

}  // namespace exact

struct exact_batch {
    int n = 0;
    void *dev = nullptr;
    exact::SceneDev *d_scenes = nullptr;      // for steps
    exact::SceneDev *d_tune = nullptr;        // same, without the dmin outputs (autotuning)
    int2 *d_items = nullptr, *d_upd = nullptr, *d_val = nullptr;
    int n_items = 0, n_upd = 0, n_val = 0;
    char *d_ctrl = nullptr;            // n headers (kHdrStride apart) + queue head
    size_t ctrl_bytes = 0;
    unsigned *d_queue = nullptr;
    int *d_sort = nullptr;             // scenes whose cloud gets a spatially ordered copy
    int n_sort = 0;
    size_t smem = 0;
    int threads = exact::kBlock, pairs = 1, sms = 0, grid = 0;
    bool uniform = false;              // every scene has the same footprint constants
    exact_footprint fp;                // their copy (uniform batches)
    int grid_c = 0;                    // persistent grid of the constant-footprint kernel (0 = not yet known)
    int *d_err = nullptr;              // device error word of the batch (not cleared by steps)
};

namespace exact {
// Sample (validate = false) or validation launch of a batch whose scenes
// share one footprint, footprint constants as kernel parameters
// (batched_uniform.cuh): rectangle covers and polygons of up to 16 edges,
// and larger polygons.
int launch_uniform_small(exact_batch *b, const SceneDev *table, cudaStream_t st, bool validate);
int launch_uniform_large(exact_batch *b, const SceneDev *table, cudaStream_t st, bool validate);
}  // namespace exact
