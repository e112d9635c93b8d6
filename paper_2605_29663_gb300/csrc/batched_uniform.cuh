// batched_uniform.cuh -- the batched cycle's sample and validation kernels
// for a batch whose scenes all share one footprint (the modes of one robot,
// a fleet of identical robots): the footprint constants are kernel
// parameters, as in the single-scene kernels, instead of a per-scene
// shared-memory table.  batched_uniform_small.cu instantiates them for the
// rectangle covers and polygons of up to 16 edges, batched_uniform_large.cu
// for larger polygons, so that the two compile in parallel.
#pragma once

#include "batched_internal.cuh"

namespace exact {

template <class FPC>
__global__ void __launch_bounds__(512, 2)   // <= 64 registers: at least 4 blocks of 256 per SM
batched_sample_kernel_c(const SceneDev *__restrict__ scenes, const int2 *__restrict__ items, int n_items,
                        unsigned *queue, int pairs_per_lane, const ConstEval<FPC> ev) {
    extern __shared__ float4 dyn[];
    float2 *s_pts = reinterpret_cast<float2 *>(dyn + kFpSlots);
    __shared__ SampleSmem sm;
    __shared__ int s_item;
    sample_smem_init(sm);
    int pts_scene = -1;   // block-uniform
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int2 it = items[item];
        const SceneDev &D = scenes[it.x];
        sample_body(D.V, ev, item_sample(it), 0, sm, s_pts, it.x == pts_scene, pairs_per_lane, D.circ,
                    item_second(it));
        pts_scene = D.V.N <= kStage ? it.x : -1;
    }
}

template <class FPC>
__global__ void __launch_bounds__(kBlock)
batched_validate_kernel_c(const SceneDev *__restrict__ scenes, const int2 *__restrict__ table,
                          const ConstEval<FPC> ev) {
    __shared__ ValidateSmem sm;
    const int2 t = table[blockIdx.x];
    const SceneDev &D = scenes[t.x];
    validate_body(D.V, ev, t.y / D.V.val_chunks, t.y % D.V.val_chunks, sm, D.circ);
}

template <class FPC>
int launch_uniform_sample_t(exact_batch *b, const SceneDev *table, cudaStream_t st, const FPC &fpc) {
    auto k = batched_sample_kernel_c<FPC>;
    if (b->grid_c <= 0) {
        int per_sm = 0;
        // staged points (dynamic) and sample state (static) exceed the default 48 KB per block
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, b->threads, b->smem) != cudaSuccess ||
            per_sm < 1)
            return EXACT_ECUDA;
        b->grid_c = b->sms * per_sm;
    }
    if (b->n_sort > 0)   // behind the cloud-ordering kernel: start early (see batched.cu)
        return cuda_status(launch_dependent(k, (unsigned)b->grid_c, (unsigned)b->threads, b->smem, st, table,
                                            (const int2 *)b->d_items, b->n_items, b->d_queue, b->pairs,
                                            ConstEval<FPC>{fpc}));
    k<<<b->grid_c, b->threads, b->smem, st>>>(table, b->d_items, b->n_items, b->d_queue, b->pairs,
                                              ConstEval<FPC>{fpc});
    return cuda_status(cudaGetLastError());
}

template <class FPC>
int launch_uniform_validate_t(exact_batch *b, cudaStream_t st, const FPC &fpc) {
    return cuda_status(launch_dependent(batched_validate_kernel_c<FPC>, (unsigned)b->n_val, (unsigned)kBlock, 0, st,
                                        (const SceneDev *)b->d_scenes, (const int2 *)b->d_val, ConstEval<FPC>{fpc}));
}

// Per size class (returns EXACT_EINVAL for a footprint of the other class).
int launch_uniform_small(exact_batch *b, const SceneDev *table, cudaStream_t st, bool validate);
int launch_uniform_large(exact_batch *b, const SceneDev *table, cudaStream_t st, bool validate);

}  // namespace exact
