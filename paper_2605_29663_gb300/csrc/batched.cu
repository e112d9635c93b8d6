// batched.cu -- many independent scenes advanced by one EXACT-MPPI control
// cycle each (Algorithm 1 per scene) in one persistent launch.
//
// Plan (exact_batch_create, host, once): a device scene table (parameters,
// pointers, footprint constants, scratch addresses), the work-item list of
// the sample phase -- one item per (scene, sample), or per (scene, two
// consecutive samples) when the batch holds at least four samples per SM and
// the scene's horizon fits two in a block's step slots; scenes ordered by
// per-sample cost T * N * edges, heaviest first (longest-processing-time
// order) -- and the block tables of the update and validation phases.
//
// Step (mppi_step_batched, capturable): a memset of the per-scene control
// words and the queue head, then
//   batched_sample_kernel   persistent: SMs x resident blocks; each block
//                           pulls items from an atomic queue and runs
//                           sample_body with the scene's footprint constants
//                           in shared memory (reloaded only when the scene
//                           changes; so are the staged points when the cloud
//                           fits the stage);
//   batched_update_kernel   one block per (scene, sample chunk): weights and
//                           weighted noise into the scene's partial slots;
//   batched_validate_kernel one block per (scene, step, point chunk): U_upd
//                           from the partial slots, the nominal rollout, the
//                           clearance check and the scene's shift / reset.
// The per-scene arithmetic is that of mppi_step (same device bodies, same
// operation order), so a scene of a batch gives the same bits as mppi_step.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <new>
#include <vector>

#include "batched_internal.cuh"

namespace exact {

__global__ void __launch_bounds__(512)
batched_sample_kernel(const SceneDev *__restrict__ scenes, const int2 *__restrict__ items, int n_items,
                      unsigned *queue, int pairs_per_lane) {
    extern __shared__ float4 dyn[];
    float4 *s_fp = dyn;
    float2 *s_pts = reinterpret_cast<float2 *>(dyn + kFpSlots);
    __shared__ SampleSmem sm;
    __shared__ int s_item;
    sample_smem_init(sm);
    int fp_scene = -1, pts_scene = -1;   // block-uniform
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int2 it = items[item];
        const SceneDev &D = scenes[it.x];
        if (it.x != fp_scene) {
            load_fp(s_fp, D);
            __syncthreads();
            fp_scene = it.x;
        }
        const SmemEval ev{s_fp, D.kind, D.nfp, D.bc, D.bh};
        sample_body(D.V, ev, item_sample(it), 0, sm, s_pts, it.x == pts_scene, pairs_per_lane, D.circ,
                    item_second(it));
        pts_scene = D.V.N <= kStage ? it.x : -1;
    }
}

// Spatially ordered cloud copies of the scenes that prune (one block each).
__global__ void __launch_bounds__(kSortThreads)
batched_sort_kernel(const SceneDev *__restrict__ scenes, const int *__restrict__ list) {
    __shared__ SortSmem sm;
    const SceneDev &D = scenes[list[blockIdx.x]];
    sort_cloud_block<false>(D.src_pts, nullptr, D.src_mask, D.V.N, const_cast<float2 *>(D.V.pts), nullptr, sm);
    __syncthreads();
    cloud_circles<false>(D.V.pts, nullptr, D.V.N, const_cast<float4 *>(D.circ));
}

__global__ void __launch_bounds__(kUpdBlock)
batched_update_kernel(const SceneDev *__restrict__ scenes, const int2 *__restrict__ table) {
    __shared__ UpdateSmem sm;
    const int2 t = table[blockIdx.x];
    update_body(scenes[t.x].V, t.y, sm);
}

__global__ void __launch_bounds__(kBlock)
batched_validate_kernel(const SceneDev *__restrict__ scenes, const int2 *__restrict__ table) {
    __shared__ float4 s_fp[kFpSlots];
    __shared__ ValidateSmem sm;
    const int2 t = table[blockIdx.x];
    const SceneDev &D = scenes[t.x];
    load_fp(s_fp, D);
    __syncthreads();
    const SmemEval ev{s_fp, D.kind, D.nfp, D.bc, D.bh};
    validate_body(D.V, ev, t.y / D.V.val_chunks, t.y % D.V.val_chunks, sm, D.circ);
}

int check_params(const exact_mppi_params *p);
MppiP to_device_params(const exact_mppi_params *p);

}  // namespace exact

using namespace exact;


static int batch_grid(exact_batch *b) {
    int per_sm = 0;
    // the staged points and footprint slots (dynamic) plus the sample state
    // (static) exceed the default 48 KB per block
    if (cudaFuncSetAttribute(batched_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) !=
        cudaSuccess)
        return EXACT_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_sample_kernel, b->threads, b->smem) !=
        cudaSuccess)
        return EXACT_ECUDA;
    if (per_sm < 1) return EXACT_EINVAL;
    b->grid = b->sms * per_sm;
    return EXACT_OK;
}

extern "C" int exact_batch_create(int n_scenes, const exact_scene *scenes, exact_batch **out) {
    if (!out || !scenes || n_scenes < 1) return EXACT_EINVAL;
    *out = nullptr;
    if (n_scenes > 4096) return EXACT_ECAPACITY;
    std::vector<SceneDev> host(n_scenes);
    std::vector<size_t> scratch_off(n_scenes);
    size_t scratch_total = 0;
    int max_stage = 0;
    for (int s = 0; s < n_scenes; ++s) {
        const exact_scene &S = scenes[s];
        int rc = check_params(&S.params);
        if (rc != EXACT_OK) return rc;
        if (!S.fp || !S.state || !S.U || !S.noise || !S.waypoints || S.n_wp < 1 || S.n_points < 0 || !S.u_star)
            return EXACT_EINVAL;
        if (S.n_points > 0 && (!S.cloud || ((uintptr_t)S.cloud & 7u) != 0)) return EXACT_EINVAL;
        scratch_off[s] = scratch_total;
        scratch_total += align_up(scene_scratch_bytes(S.params.K, S.params.T, 1), 256);
        // scenes that prune (no d_min output, large cloud) get a spatially ordered cloud copy
        if (!S.dmin && S.n_points >= kPruneMin)
            scratch_total += align_up((size_t)S.n_points * sizeof(float2), 256) + circle_bytes(S.n_points);
        max_stage = std::max(max_stage, std::min(S.n_points, kStage));
    }
    std::vector<int> sort_list;
    for (int s = 0; s < n_scenes; ++s)
        if (!scenes[s].dmin && scenes[s].n_points >= kPruneMin) sort_list.push_back(s);
    const size_t table_bytes = align_up(sizeof(SceneDev) * n_scenes, 256);
    // items and block tables
    std::vector<int> order(n_scenes);
    for (int s = 0; s < n_scenes; ++s) order[s] = s;
    auto cost = [&](int s) {
        const exact_scene &S = scenes[s];
        return (double)S.params.T * std::max(S.n_points, 1) * (double)S.fp->n_pad;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
    std::vector<int2> items, upd, val;
    long long total_k = 0;
    for (int s = 0; s < n_scenes; ++s) total_k += scenes[s].params.K;
    const int sms_now = current_sm_count();
    for (int s : order) {
        const exact_mppi_params &p = scenes[s].params;
        // pairs of samples per item when the whole batch has enough samples
        // to fill the GPU at half the items (and this scene's horizon fits)
        const bool two = pair_samples((int)std::min<long long>(total_k, 1 << 29), p.T, 1, sms_now);
        for (int r = 0; r < p.K; r += two ? 2 : 1)
            items.push_back(make_int2(s, r | (two && r + 1 < p.K ? kItemPair : 0)));
    }
    for (int s = 0; s < n_scenes; ++s) {
        const exact_mppi_params &p = scenes[s].params;
        for (int q = 0; q < upd_blocks_for(p.K, p.T, p.n_u); ++q) upd.push_back(make_int2(s, q));
        for (int q = 0; q < p.T * val_chunks_for(scenes[s].n_points); ++q) val.push_back(make_int2(s, q));
    }
    const size_t items_bytes = align_up(items.size() * sizeof(int2), 256);
    const size_t upd_bytes = align_up(upd.size() * sizeof(int2), 256);
    const size_t val_bytes = align_up(val.size() * sizeof(int2), 256);
    const size_t ctrl_bytes = align_up(kHdrStride * n_scenes + sizeof(unsigned), 256);
    const size_t sort_bytes = align_up(sort_list.size() * sizeof(int) + 1, 256);
    const size_t err_bytes = 256;
    const size_t total =
        2 * table_bytes + items_bytes + upd_bytes + val_bytes + ctrl_bytes + sort_bytes + err_bytes + scratch_total;

    exact_batch *b = new (std::nothrow) exact_batch();
    if (!b) return EXACT_EINVAL;
    if (cudaMalloc(&b->dev, total) != cudaSuccess) { delete b; return EXACT_ECUDA; }
    char *p = static_cast<char *>(b->dev);
    b->d_scenes = reinterpret_cast<SceneDev *>(p); p += table_bytes;
    b->d_tune = reinterpret_cast<SceneDev *>(p); p += table_bytes;
    b->d_items = reinterpret_cast<int2 *>(p); p += items_bytes;
    b->d_upd = reinterpret_cast<int2 *>(p); p += upd_bytes;
    b->d_val = reinterpret_cast<int2 *>(p); p += val_bytes;
    b->d_ctrl = p; p += ctrl_bytes;
    b->d_sort = reinterpret_cast<int *>(p); p += sort_bytes;
    b->n_sort = (int)sort_list.size();
    b->d_err = reinterpret_cast<int *>(p); p += err_bytes;
    char *scratch = p;
    b->ctrl_bytes = ctrl_bytes;
    b->d_queue = reinterpret_cast<unsigned *>(b->d_ctrl + kHdrStride * n_scenes);
    b->n = n_scenes;
    b->n_items = (int)items.size();
    b->n_upd = (int)upd.size();
    b->n_val = (int)val.size();
    b->smem = kFpSlots * sizeof(float4) + (size_t)max_stage * sizeof(float2);
    b->sms = current_sm_count();
    b->uniform = true;
    for (int s = 1; s < n_scenes && b->uniform; ++s)
        b->uniform = memcmp(scenes[s].fp, scenes[0].fp, sizeof(exact_footprint)) == 0;
    if (b->uniform) b->fp = *scenes[0].fp;

    for (int s = 0; s < n_scenes; ++s) {
        const exact_scene &S = scenes[s];
        SceneDev &D = host[s];
        memset(&D, 0, sizeof(D));
        SceneView &V = D.V;
        V.P = to_device_params(&S.params);
        V.state = S.state;
        V.pts = reinterpret_cast<const float2 *>(S.cloud);
        V.mask = S.mask;
        V.N = S.n_points;
        V.wp = S.waypoints;
        V.W = S.n_wp;
        V.U = S.U;
        V.noise = S.noise;
        V.u_star = S.u_star; V.costs = S.costs; V.weights = S.weights; V.U_upd_out = S.U_upd;
        V.dmin = S.dmin; V.valid = S.valid; V.nom_cost = S.nom_cost;
        V.err = b->d_err;
        V.hdr = reinterpret_cast<ArenaHeader *>(b->d_ctrl + kHdrStride * s);
        carve_scene(V, scratch + scratch_off[s], S.params.K, S.params.T, 1);
        D.src_pts = V.pts;
        D.src_mask = V.mask;
        if (!S.dmin && S.n_points >= kPruneMin) {   // the sort kernel fills the copy before each step
            char *q = scratch + scratch_off[s] + align_up(scene_scratch_bytes(S.params.K, S.params.T, 1), 256);
            V.pts = reinterpret_cast<const float2 *>(q);
            D.circ = reinterpret_cast<const float4 *>(q + align_up((size_t)S.n_points * sizeof(float2), 256));
            V.mask = nullptr;
        }
        V.upd_chunk = upd_chunk_for(S.params.K, S.params.T, S.params.n_u);
        V.upd_blocks = upd_blocks_for(S.params.K, S.params.T, S.params.n_u);
        V.val_chunks = val_chunks_for(S.n_points);
        const exact_footprint *fp = S.fp;
        D.kind = fp->kind;
        D.nfp = fp->n_pad;
        D.bc = make_float3(fp->bcx, fp->bcy, fp->brad);
        D.bh = make_float2(fp->bhx, fp->bhy);
        if (fp->kind == EXACT_FP_POLYGON) {
            const int E = fp->n_pad;
            float *eyn = reinterpret_cast<float *>(D.fpc + 3 * E + 1);
            for (int e = 0; e < E; ++e) {
                D.fpc[3 * e] = make_float4(-fp->vx[e], -fp->vx[e], -fp->vy[e], -fp->vy[e]);
                D.fpc[3 * e + 1] = make_float4(fp->exn[e], fp->exn[e], -fp->kx[e], -fp->kx[e]);
                D.fpc[3 * e + 2] = make_float4(-fp->ex[e], -fp->ex[e], -fp->ey[e], -fp->ey[e]);
                eyn[e] = fp->eyn[e];
            }
            D.fpc[3 * E] = D.fpc[0];
        } else {
            for (int j = 0; j < fp->n_pad; ++j) D.fpc[j] = make_float4(fp->cx[j], fp->cy[j], fp->sx[j], fp->sy[j]);
        }
    }
    std::vector<SceneDev> tune = host;
    for (auto &D : tune) D.V.dmin = nullptr;
    int rc = EXACT_OK;
    if (cudaMemcpy(b->d_scenes, host.data(), sizeof(SceneDev) * n_scenes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tune, tune.data(), sizeof(SceneDev) * n_scenes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_upd, upd.data(), upd.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_val, val.data(), val.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        (b->n_sort && cudaMemcpy(b->d_sort, sort_list.data(), sort_list.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                          cudaSuccess) ||
        cudaMemset(b->d_ctrl, 0, ctrl_bytes) != cudaSuccess || cudaMemset(b->d_err, 0, err_bytes) != cudaSuccess ||
        (scratch_total && cudaMemset(scratch, 0, scratch_total) != cudaSuccess))
        rc = EXACT_ECUDA;
    if (rc == EXACT_OK) rc = batch_grid(b);
    if (rc != EXACT_OK) {
        cudaFree(b->dev);
        delete b;
        return rc;
    }
    *out = b;
    return EXACT_OK;
}

extern "C" void exact_batch_destroy(exact_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    cudaFree(b->dev);
    delete b;
}

static int launch_sample(exact_batch *b, const SceneDev *table, cudaStream_t st) {
    if (cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_bytes, st) != cudaSuccess) return EXACT_ECUDA;
    if (b->n_sort > 0) {
        batched_sort_kernel<<<b->n_sort, kSortThreads, 0, st>>>(table, b->d_sort);
        if (cudaGetLastError() != cudaSuccess) return EXACT_ECUDA;
    }
    if (!b->uniform) {
        // behind the cloud-ordering kernel the persistent blocks start early
        // (rollouts first; sample_body waits before it reads a cloud)
        if (b->n_sort > 0)
            return cuda_status(launch_dependent(batched_sample_kernel, (unsigned)b->grid, (unsigned)b->threads, b->smem,
                                                st, table, (const int2 *)b->d_items, b->n_items, b->d_queue, b->pairs));
        batched_sample_kernel<<<b->grid, b->threads, b->smem, st>>>(table, b->d_items, b->n_items, b->d_queue,
                                                                     b->pairs);
        return cuda_status(cudaGetLastError());
    }
    return b->fp.kind == EXACT_FP_POLYGON && b->fp.n_pad > 16 ? launch_uniform_large(b, table, st, false)
                                                               : launch_uniform_small(b, table, st, false);
}

extern "C" int mppi_step_batched(exact_batch *b, void *stream) {
    if (!b) return EXACT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_sample(b, b->d_scenes, st);
    if (rc != EXACT_OK) return rc;
    // update and validation start while their predecessor drains
    // (programmatic dependent launch; the bodies wait where they read its
    // results, as in the single-scene cycle)
    if (launch_dependent(batched_update_kernel, (unsigned)b->n_upd, (unsigned)kUpdBlock, 0, st,
                         (const SceneDev *)b->d_scenes, (const int2 *)b->d_upd) != cudaSuccess)
        return EXACT_ECUDA;
    if (!b->uniform)
        return cuda_status(launch_dependent(batched_validate_kernel, (unsigned)b->n_val, (unsigned)kBlock, 0, st,
                                            (const SceneDev *)b->d_scenes, (const int2 *)b->d_val));
    return b->fp.kind == EXACT_FP_POLYGON && b->fp.n_pad > 16 ? launch_uniform_large(b, b->d_scenes, st, true)
                                                               : launch_uniform_small(b, b->d_scenes, st, true);
}

extern "C" int exact_batch_get_error(exact_batch *b, void *stream) {
    if (!b) return EXACT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int err = 0;
    if (cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(b->d_err, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return EXACT_ECUDA;
    return err;
}

extern "C" int exact_batch_get_tiles(const exact_batch *b, int *threads, int *pairs_per_lane) {
    if (!b) return EXACT_EINVAL;
    if (threads) *threads = b->threads;
    if (pairs_per_lane) *pairs_per_lane = b->pairs;
    return EXACT_OK;
}

extern "C" int exact_batch_set_tiles(exact_batch *b, int threads, int pairs_per_lane) {
    if (!b) return EXACT_EINVAL;
    if (!(threads == 64 || threads == 128 || threads == 256 || threads == 512)) return EXACT_EINVAL;
    if (pairs_per_lane < 1 || pairs_per_lane > 8) return EXACT_EINVAL;
    const int ot = b->threads, op = b->pairs;
    b->threads = threads;
    b->pairs = pairs_per_lane;
    b->grid_c = 0;
    const int rc = batch_grid(b);
    if (rc != EXACT_OK) {
        b->threads = ot;
        b->pairs = op;
        batch_grid(b);
    }
    return rc;
}

extern "C" int exact_batch_autotune(exact_batch *b, int iters, char *json_out, int json_cap, void *stream) {
    if (!b || iters < 1) return EXACT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    static const int kThreads[] = {128, 256, 512};
    static const int kPairs[] = {1, 2, 4, 8};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return EXACT_ECUDA;
    float best_ms = 3.0e38f;
    int best_t = b->threads, best_p = b->pairs;
    std::string json = "{\"candidates\": [";
    bool first = true;
    int rc = EXACT_OK;
    for (int t : kThreads) {
        for (int pl : kPairs) {
            if (exact_batch_set_tiles(b, t, pl) != EXACT_OK) continue;
            if ((rc = launch_sample(b, b->d_tune, st)) != EXACT_OK) break;   // warm-up
            cudaEventRecord(e0, st);
            for (int i = 0; i < iters && rc == EXACT_OK; ++i) rc = launch_sample(b, b->d_tune, st);
            cudaEventRecord(e1, st);
            if (rc != EXACT_OK || cudaEventSynchronize(e1) != cudaSuccess) { rc = EXACT_ECUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= iters;
            char buf[128];
            snprintf(buf, sizeof(buf), "%s{\"threads\": %d, \"pairs_per_lane\": %d, \"ms\": %.6f}", first ? "" : ", ", t,
                     pl, ms);
            json += buf;
            first = false;
            if (ms < best_ms) { best_ms = ms; best_t = t; best_p = pl; }
        }
        if (rc != EXACT_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int src = exact_batch_set_tiles(b, best_t, best_p);
    if (rc == EXACT_OK) rc = src;
    char buf[160];
    snprintf(buf, sizeof(buf), "], \"best\": {\"threads\": %d, \"pairs_per_lane\": %d, \"ms\": %.6f}}", best_t, best_p,
             best_ms);
    json += buf;
    if (json_out && json_cap > 0) {
        strncpy(json_out, json.c_str(), (size_t)json_cap - 1);
        json_out[json_cap - 1] = '\0';
    }
    return rc;
}
