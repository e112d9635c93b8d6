// sdf_batch.cu -- exact_sdf_batch: poses x points body-frame signed distances
// (Sec. IV-C, IV-D), the evaluator benchmarked in Experiment 1.
//
// Layout: block b covers one pose and one chunk of point pairs.  Each thread
// takes two consecutive points per iteration (two independent evaluator
// chains for ILP), so a warp reads 512 contiguous bytes of points and writes
// 256 contiguous bytes of the distance row with streaming stores.  The pose's
// sincos is taken once per thread; the footprint sits in the constant bank.
// Minima are reduced per block (warp shuffles over packed (key, index)
// words); when several blocks share a pose they meet in a 64-bit atomicMin
// on a per-pose key in the context arena, finished by a small kernel.
#include "internal.h"

namespace exact {

template <class FPC, bool DIST, bool MASKED>
__global__ void __launch_bounds__(kBlock)
sdf_batch_kernel(const float2 *__restrict__ pts, const uint8_t *__restrict__ mask, int N,
                 const float *__restrict__ poses, const FPC fpc, float *__restrict__ dist, int vec_store,
                 float *__restrict__ dmin, int *__restrict__ argmin,
                 unsigned long long *__restrict__ keys, int chunks, int chunk_pairs) {
    const int pose = blockIdx.x / chunks;
    const int chunk = blockIdx.x - pose * chunks;
    const float tx = poses[3 * (size_t)pose], ty = poses[3 * (size_t)pose + 1], th = poses[3 * (size_t)pose + 2];
    float sn, cs;
    sincosf(th, &sn, &cs);
    const int npairs = (N + 1) >> 1;
    const int pbeg = chunk * chunk_pairs;
    const int pend = min(npairs, pbeg + chunk_pairs);
    float *drow = DIST ? dist + (size_t)pose * (size_t)N : nullptr;
    float bk = finf();        // best key of this thread (first index wins ties)
    int bi = -1;

    for (int j = pbeg + (int)threadIdx.x; j < pend; j += kBlock) {
        const int i0 = 2 * j, i1 = 2 * j + 1;
        const bool has1 = i1 < N;
        const float2 o0 = __ldg(pts + i0);
        const float2 o1 = has1 ? __ldg(pts + i1) : o0;
        float px0, py0, px1, py1;
        body_frame(o0.x, o0.y, tx, ty, cs, sn, px0, py0);
        body_frame(o1.x, o1.y, tx, ty, cs, sn, px1, py1);
        float k0, k1;
        eval2(fpc, px0, py0, px1, py1, k0, k1);
        bool v0 = true, v1 = has1;
        if (MASKED) {
            v0 = __ldg(mask + i0) != 0;
            v1 = has1 && __ldg(mask + i1) != 0;
            k0 = v0 ? k0 : finf();
            k1 = v1 ? k1 : finf();
        }
        if (DIST) {
            const float d0 = key_to_dist(fpc, k0);
            const float d1 = key_to_dist(fpc, k1);
            if (vec_store) {
                __stcs(reinterpret_cast<float2 *>(drow) + j, make_float2(d0, d1));
            } else {
                __stcs(drow + i0, d0);
                if (has1) __stcs(drow + i1, d1);
            }
        }
        // strict "<" keeps the lowest index among equal keys; +inf (padding)
        // and NaN never replace the initial +inf
        if (k0 < bk) { bk = k0; bi = i0; }
        if (v1 && k1 < bk) { bk = k1; bi = i1; }
    }

    if (!dmin && !argmin) return;
    __shared__ unsigned long long red[kBlock / 32];
    unsigned long long best = bi < 0 ? kNoKey : pack_key(bk, (unsigned)bi);
    best = warp_min_u64(best);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = red[0];
#pragma unroll
        for (int w = 1; w < kBlock / 32; ++w) b = red[w] < b ? red[w] : b;
        if (chunks == 1) {
            if (dmin) dmin[pose] = b == kNoKey ? finf() : key_to_dist(fpc, ord2f((unsigned)(b >> 32)));
            if (argmin) argmin[pose] = b == kNoKey ? -1 : (int)(unsigned)(b & 0xffffffffu);
        } else if (b != kNoKey) {
            atomicMin(keys + pose, b);
        }
    }
}

__global__ void sdf_keys_init(unsigned long long *keys, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) keys[p] = kNoKey;
}

template <class FPC>
__global__ void sdf_keys_finish(const unsigned long long *__restrict__ keys, int P, const FPC fpc,
                                float *__restrict__ dmin, int *__restrict__ argmin) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const unsigned long long b = keys[p];
    if (dmin) dmin[p] = b == kNoKey ? finf() : key_to_dist(fpc, ord2f((unsigned)(b >> 32)));
    if (argmin) argmin[p] = b == kNoKey ? -1 : (int)(unsigned)(b & 0xffffffffu);
}

size_t sdf_scratch_bytes(int n_poses) { return kArenaHeader + align_up((size_t)n_poses * sizeof(unsigned long long), 256); }

}  // namespace exact

extern "C" int exact_sdf_batch(exact_ctx *ctx, const float *points, const uint8_t *mask, int n_points,
                               const float *poses, int n_poses, const exact_footprint *fp,
                               float *dist, float *dmin, int *argmin, void *stream) {
    using namespace exact;
    if (!fp || n_points < 0 || n_poses < 0) return EXACT_EINVAL;
    if (n_poses == 0) return EXACT_OK;
    if (!poses || (n_points > 0 && !points)) return EXACT_EINVAL;
    if (n_points > 0 && ((uintptr_t)points & 7u) != 0) return EXACT_EINVAL;
    if ((size_t)n_points * (size_t)n_poses >= ((size_t)1 << 62)) return EXACT_ECAPACITY;
    cudaStream_t st = (cudaStream_t)stream;

    // one block per pose when there are enough poses to fill the GPU;
    // otherwise split each pose's points over several blocks
    const int npairs = (n_points + 1) / 2;
    int sms = ctx ? ctx->sm_count : 0;
    if (sms <= 0) sms = current_sm_count();
    const int target = sms * 8;
    int chunks = 1;
    if (n_poses < target && npairs > 256) {
        chunks = (target + n_poses - 1) / n_poses;
        const int max_chunks = (npairs + 255) / 256;
        if (chunks > max_chunks) chunks = max_chunks;
    }
    if (chunks > 1 && (dmin || argmin) && !ctx) chunks = 1;   // no arena for the cross-block minimum
    if ((long long)n_poses * chunks > 0x7fffffffLL) chunks = 1;
    const int chunk_pairs = (npairs + chunks - 1) / chunks;
    const int vec = dist && (n_points % 2 == 0) && (((uintptr_t)dist & 7u) == 0);

    unsigned long long *keys = nullptr;
    if (chunks > 1 && (dmin || argmin)) {
        const int rc = ensure_scratch(ctx, sdf_scratch_bytes(n_poses));
        if (rc != EXACT_OK) return rc;
        keys = reinterpret_cast<unsigned long long *>(static_cast<char *>(ctx->scratch) + kArenaHeader);
        ctx->mppi_layout = -1;   // the keys overlay the MPPI per-sample counters
        sdf_keys_init<<<(n_poses + 255) / 256, 256, 0, st>>>(keys, n_poses);
    }
    const float2 *p2 = reinterpret_cast<const float2 *>(points);
    const unsigned grid = (unsigned)(n_poses * chunks);
    return with_footprint(fp, [&](auto fpc) -> int {
        using FPC = decltype(fpc);
        auto k = mask ? (dist ? sdf_batch_kernel<FPC, true, true> : sdf_batch_kernel<FPC, false, true>)
                      : (dist ? sdf_batch_kernel<FPC, true, false> : sdf_batch_kernel<FPC, false, false>);
        k<<<grid, kBlock, 0, st>>>(p2, mask, n_points, poses, fpc, dist, vec, dmin, argmin, keys, chunks,
                                   chunk_pairs);
        if (keys)
            sdf_keys_finish<FPC><<<(n_poses + 255) / 256, 256, 0, st>>>(keys, n_poses, fpc, dmin, argmin);
        return cuda_status(cudaGetLastError());
    });
}
