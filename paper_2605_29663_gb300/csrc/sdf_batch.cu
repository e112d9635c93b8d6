// sdf_batch.cu -- exact_sdf_batch: poses x points body-frame signed distances
// (Sec. IV-C, IV-D), the evaluator benchmarked in Experiment 1.
//
// Layout: block b covers one pose and one chunk of point pairs.  Each thread
// takes two consecutive points per iteration (the two lanes of the packed
// f32x2 evaluator), so a warp reads 512 contiguous bytes of points and writes
// 256 contiguous bytes of the distance row with streaming stores.  The pose's
// sincos is taken once per thread; the footprint sits in the constant bank.
// Minima are reduced per block (warp shuffles over packed (key, index)
// words); when several blocks share a pose they meet in a 64-bit atomicMin
// on a per-pose key in the context arena, finished by a small kernel.
#include "internal.h"

namespace exact {

constexpr int kSdfBlock = 128;   // threads per block (measured 1% faster than 256 at the same occupancy)
constexpr int kNearQ = 128;   // per-warp queue of near points (two batches)

// Polygon rows: point pairs [pbeg, pend) of one pose.  The edge loop takes
// the distances only.  The crossing parity can be odd only for a point within
// the footprint's bounding circle; every other point is outside, sign +.
// Points within the circle (plus a margin far above the rounding of the
// parity test, so that the skipped parities are exactly the even ones the
// full evaluation would find) are queued per warp in index order with their
// squared distance, and take a parity-only pass over the edges 64 at a time.
// Those found inside get their distance rewritten with the minus sign (after
// a __syncwarp, which orders the two stores).  Both passes repeat the
// operations of the full evaluation, so every output is the same bits.  The
// per-thread minimum first sees every near point as outside; the negative key
// of an inside point then replaces it, with ties going to the lower index.
template <class FPC, bool DIST, bool MASKED>
__device__ __forceinline__ void poly_rows(const float2 *__restrict__ pts, const uint8_t *__restrict__ mask, int N,
                                          const FPC &fpc, float tx, float ty, float cs, float sn, int pbeg,
                                          int pend, float *__restrict__ drow, int vec_store, float &bk, int &bi) {
    constexpr int E = fp_traits<FPC>::size;
    __shared__ int q_idx[kSdfBlock / 32][kNearQ];
    __shared__ float q_m[kSdfBlock / 32][kNearQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *qi = q_idx[warp];
    float *qm = q_m[warp];
    int qn = 0;   // queued entries (warp-uniform)
    const float lim = fmaf(fpc.brad, 1e-5f, fpc.brad) + 1e-5f;
    const float lim2 = lim * lim;

    auto parity_pass = [&](int cnt) {   // queue entries [0, cnt), cnt <= 64
        __syncwarp();
        const int e0 = 2 * lane;
        if (e0 < cnt) {
            const bool g1 = e0 + 1 < cnt;
            const int ia = qi[e0], ib = g1 ? qi[e0 + 1] : ia;
            const float2 oa = __ldg(pts + ia), ob = __ldg(pts + ib);
            float pxa, pya, pxb, pyb;
            body_frame(oa.x, oa.y, tx, ty, cs, sn, pxa, pya);
            body_frame(ob.x, ob.y, tx, ty, cs, sn, pxb, pyb);
            float ma, mb;
            unsigned sa, sb;
            poly_eval2<E, kSign>(fpc, pxa, pya, pxb, pyb, ma, mb, sa, sb);
            auto inside = [&](int i, float m, unsigned sg) {
                if (sg & 0x80000000u) {
                    const float k = __uint_as_float(__float_as_uint(m) | 0x80000000u);
                    if (DIST) __stcs(drow + i, key_to_dist(fpc, k));
                    if (k < bk || (k == bk && i < bi)) { bk = k; bi = i; }
                }
            };
            inside(ia, qm[e0], sa);
            if (g1) inside(ib, qm[e0 + 1], sb);
        }
        __syncwarp();
    };

    for (int j0 = pbeg + (int)(threadIdx.x & ~31u); j0 < pend; j0 += kSdfBlock) {   // warp-uniform trip count
        const int j = j0 + lane, i0 = 2 * j, i1 = 2 * j + 1;
        bool f0 = false, f1 = false;
        float m0 = 0.f, m1 = 0.f;
        if (j < pend) {
            const bool has1 = i1 < N;
            const float2 o0 = __ldg(pts + i0);
            const float2 o1 = has1 ? __ldg(pts + i1) : o0;
            float px0, py0, px1, py1;
            body_frame(o0.x, o0.y, tx, ty, cs, sn, px0, py0);
            body_frame(o1.x, o1.y, tx, ty, cs, sn, px1, py1);
            unsigned s0, s1;
            poly_eval2<E, kDist>(fpc, px0, py0, px1, py1, m0, m1, s0, s1);
            bool v0 = true, v1 = has1;
            if (MASKED) {
                v0 = __ldg(mask + i0) != 0;
                v1 = has1 && __ldg(mask + i1) != 0;
            }
            const float k0 = v0 ? m0 : finf(), k1 = v1 ? m1 : finf();
            const float cx0 = px0 - fpc.bcx, cy0 = py0 - fpc.bcy, cx1 = px1 - fpc.bcx, cy1 = py1 - fpc.bcy;
            f0 = v0 && fmaf(cx0, cx0, cy0 * cy0) <= lim2;
            f1 = v1 && fmaf(cx1, cx1, cy1 * cy1) <= lim2;
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
            // strict "<" keeps the lowest index among equal keys; +inf
            // (padding) and NaN never replace the initial +inf
            if (k0 < bk) { bk = k0; bi = i0; }
            if (v1 && k1 < bk) { bk = k1; bi = i1; }
        }
        const unsigned b0 = __ballot_sync(0xffffffffu, f0), b1 = __ballot_sync(0xffffffffu, f1);
        if (b0 | b1) {
            const unsigned below = (1u << lane) - 1u;
            const int pos = qn + __popc(b0 & below) + __popc(b1 & below);
            if (f0) { qi[pos] = i0; qm[pos] = m0; }
            if (f1) { qi[pos + (f0 ? 1 : 0)] = i1; qm[pos + (f0 ? 1 : 0)] = m1; }
            qn += __popc(b0) + __popc(b1);
            if (qn >= 64) {
                parity_pass(64);
                for (int e = lane; e < qn - 64; e += 32) {
                    qi[e] = qi[64 + e];
                    qm[e] = qm[64 + e];
                }
                qn -= 64;
            }
        }
    }
    if (qn > 0) parity_pass(qn);
}

template <class FPC, bool DIST, bool MASKED>
__global__ void __launch_bounds__(kSdfBlock)
sdf_batch_kernel(const float2 *__restrict__ pts, const uint8_t *__restrict__ mask, int N,
                 const float *__restrict__ poses, const FPC fpc, float *__restrict__ dist, int vec_store,
                 float *__restrict__ dmin, int *__restrict__ argmin,
                 unsigned long long *__restrict__ keys, int chunks, int chunk_pairs, int *err) {
    const int pose = blockIdx.x / chunks;
    const int chunk = blockIdx.x - pose * chunks;
    const float tx = poses[3 * (size_t)pose], ty = poses[3 * (size_t)pose + 1], th = poses[3 * (size_t)pose + 2];
    if (chunk == 0 && threadIdx.x == 0 && !(isfinite(tx) && isfinite(ty) && isfinite(th)))
        report_error(err, EXACT_EINVAL);   // non-finite pose (device data)
    float sn, cs;
    sincosf(th, &sn, &cs);
    const int npairs = (N + 1) >> 1;
    const int pbeg = chunk * chunk_pairs;
    const int pend = min(npairs, pbeg + chunk_pairs);
    float *drow = DIST ? dist + (size_t)pose * (size_t)N : nullptr;
    float bk = finf();        // best key of this thread (first index wins ties)
    int bi = -1;

    // polygons of 8 edges or more: parity only for near points (poly_rows);
    // below that the queue costs about what it saves
    if constexpr (fp_traits<FPC>::kind == EXACT_FP_POLYGON && fp_traits<FPC>::size >= 8) {
        poly_rows<FPC, DIST, MASKED>(pts, mask, N, fpc, tx, ty, cs, sn, pbeg, pend, drow, vec_store, bk, bi);
    } else {
    for (int j = pbeg + (int)threadIdx.x; j < pend; j += kSdfBlock) {
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
    }

    if (!dmin && !argmin) return;
    __shared__ unsigned long long red[kSdfBlock / 32];
    unsigned long long best = bi < 0 ? kNoKey : pack_key(bk, (unsigned)bi);
    best = warp_min_u64(best);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = red[0];
#pragma unroll
        for (int w = 1; w < kSdfBlock / 32; ++w) b = red[w] < b ? red[w] : b;
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
        k<<<grid, kSdfBlock, 0, st>>>(p2, mask, n_points, poses, fpc, dist, vec, dmin, argmin, keys, chunks,
                                   chunk_pairs, ctx ? ctx->d_err : nullptr);
        if (keys)
            sdf_keys_finish<FPC><<<(n_poses + 255) / 256, 256, 0, st>>>(keys, n_poses, fpc, dmin, argmin);
        return cuda_status(cudaGetLastError());
    });
}
