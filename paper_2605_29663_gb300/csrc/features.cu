// features.cu -- inputs and outputs of the learned sampling proposal.
//
//   exact_polar_hist        per robot: nearest range per angular bin of its
//                           obstacle points in its body frame
//   exact_proposal_features the network input [hist / r_max, goal (body
//                           frame) / r_max, state (5), previous nominal U]
//   exact_proposal_prepare  per robot: the two candidate nominals, the
//                           proposal's (U + network shift) and the plain one
//   exact_proposal_select   per robot: keep the candidate whose best J~ is
//                           lower (the plain one on ties), i.e. plain MPPI is
//                           the fallback whenever the proposal does worse
#include "internal.h"

namespace exact {

__global__ void __launch_bounds__(256)
polar_hist_kernel(const float2 *__restrict__ clouds, const uint8_t *__restrict__ masks, int N,
                  const float *__restrict__ poses, int nbins, float r_max, float *__restrict__ out) {
    extern __shared__ unsigned bins[];
    const int b = blockIdx.x;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) bins[k] = __float_as_uint(r_max);
    __syncthreads();
    float sn, cs;
    sincosf(poses[3 * b + 2], &sn, &cs);
    const float tx = poses[3 * b], ty = poses[3 * b + 1];
    const float two_pi = 6.283185307179586f, pi = 3.14159265358979f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        if (masks && !masks[(size_t)b * N + i]) continue;
        const float2 o = clouds[(size_t)b * N + i];
        float px, py;
        body_frame(o.x, o.y, tx, ty, cs, sn, px, py);
        const float r = sqrtf(fmaf(px, px, py * py));
        int k = (int)floorf((atan2f(py, px) + pi) / two_pi * (float)nbins);
        k = k < 0 ? 0 : (k > nbins - 1 ? nbins - 1 : k);
        if (r == r) atomicMin(&bins[k], __float_as_uint(r));   // non-negative floats order as their bits
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) out[(size_t)b * nbins + k] = __uint_as_float(bins[k]);
}

// x = [hist / r_max (nbins), goal_body / r_max (2), v_prev, w_prev, |goal| / r_max,
//      cos(bearing), sin(bearing), U_prev (T x 2)]
__global__ void proposal_features_kernel(const float *__restrict__ hist, int nbins, float r_max,
                                         const float *__restrict__ poses, const float *__restrict__ goals,
                                         const float *__restrict__ prev_cmd, const float *__restrict__ U_prev, int T,
                                         int B, float *__restrict__ x) {
    const int b = blockIdx.x;
    if (b >= B) return;
    const int D = nbins + 7 + 2 * T;
    float *xr = x + (size_t)b * D;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) xr[k] = hist[(size_t)b * nbins + k] / r_max;
    for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) xr[nbins + 7 + k] = U_prev[(size_t)b * 2 * T + k];
    if (threadIdx.x == 0) {
        float sn, cs;
        sincosf(poses[3 * b + 2], &sn, &cs);
        float gx, gy;
        body_frame(goals[2 * b], goals[2 * b + 1], poses[3 * b], poses[3 * b + 1], cs, sn, gx, gy);
        const float dist = sqrtf(fmaf(gx, gx, gy * gy));
        xr[nbins + 0] = gx / r_max;
        xr[nbins + 1] = gy / r_max;
        xr[nbins + 2] = prev_cmd[2 * b];
        xr[nbins + 3] = prev_cmd[2 * b + 1];
        xr[nbins + 4] = dist / r_max;
        xr[nbins + 5] = dist > 0.f ? gx / dist : 1.f;
        xr[nbins + 6] = dist > 0.f ? gy / dist : 0.f;
    }
}

__global__ void proposal_prepare_kernel(const float *__restrict__ U_prev, const float *__restrict__ shift,
                                        long long n, float *__restrict__ U_prop, float *__restrict__ U_plain) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float u = U_prev[e];
        U_prop[e] = u + shift[e];
        U_plain[e] = u;
    }
}

// One block per robot: min J~ of both candidates, then copy the chosen
// candidate's (shifted or reset) nominal and command.
__global__ void __launch_bounds__(256)
proposal_select_kernel(const float *__restrict__ costs_prop, const float *__restrict__ costs_plain, int K,
                       const float *__restrict__ U_prop, const float *__restrict__ U_plain,
                       const float *__restrict__ u_prop, const float *__restrict__ u_plain, int TN, int nu,
                       float *__restrict__ U_out, float *__restrict__ u_out, int *__restrict__ chose_prop) {
    __shared__ float s[2][8];
    __shared__ int s_pick;
    const int b = blockIdx.x;
    float mp = finf(), mq = finf();
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
        mp = fminf(mp, costs_prop[(size_t)b * K + r]);
        mq = fminf(mq, costs_plain[(size_t)b * K + r]);
    }
    mp = warp_min_f(mp);
    mq = warp_min_f(mq);
    if ((threadIdx.x & 31) == 0) { s[0][threadIdx.x >> 5] = mp; s[1][threadIdx.x >> 5] = mq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { s[0][0] = fminf(s[0][0], s[0][w]); s[1][0] = fminf(s[1][0], s[1][w]); }
        s_pick = s[0][0] < s[1][0] ? 1 : 0;
        if (chose_prop) chose_prop[b] = s_pick;
    }
    __syncthreads();
    const float *Us = s_pick ? U_prop : U_plain;
    const float *us = s_pick ? u_prop : u_plain;
    for (int e = threadIdx.x; e < TN; e += blockDim.x) U_out[(size_t)b * TN + e] = Us[(size_t)b * TN + e];
    for (int e = threadIdx.x; e < nu; e += blockDim.x) u_out[(size_t)b * nu + e] = us[(size_t)b * nu + e];
}

}  // namespace exact

using namespace exact;

extern "C" int exact_polar_hist(const float *clouds, const uint8_t *masks, int B, int N, const float *poses, int nbins,
                                float r_max, float *out, void *stream) {
    if (B < 0 || N < 0 || nbins < 1 || nbins > 4096 || !(r_max > 0.f) || (B > 0 && (!poses || !out))) return EXACT_EINVAL;
    if (B == 0) return EXACT_OK;
    if (N > 0 && !clouds) return EXACT_EINVAL;
    polar_hist_kernel<<<B, 256, nbins * sizeof(unsigned), (cudaStream_t)stream>>>(
        reinterpret_cast<const float2 *>(clouds), masks, N, poses, nbins, r_max, out);
    return cuda_status(cudaGetLastError());
}

extern "C" int exact_proposal_features(const float *hist, int nbins, float r_max, const float *poses,
                                       const float *goals, const float *prev_cmd, const float *U_prev, int T, int B,
                                       float *x, void *stream) {
    if (B < 0 || nbins < 1 || T < 1 || !(r_max > 0.f)) return EXACT_EINVAL;
    if (B == 0) return EXACT_OK;
    if (!hist || !poses || !goals || !prev_cmd || !U_prev || !x) return EXACT_EINVAL;
    proposal_features_kernel<<<B, 128, 0, (cudaStream_t)stream>>>(hist, nbins, r_max, poses, goals, prev_cmd, U_prev,
                                                                  T, B, x);
    return cuda_status(cudaGetLastError());
}

extern "C" int exact_proposal_prepare(const float *U_prev, const float *shift, long long n, float *U_prop,
                                      float *U_plain, void *stream) {
    if (n < 0 || (n > 0 && (!U_prev || !shift || !U_prop || !U_plain))) return EXACT_EINVAL;
    if (n == 0) return EXACT_OK;
    const long long g = (n + 255) / 256;
    proposal_prepare_kernel<<<(int)(g > 4096 ? 4096 : g), 256, 0, (cudaStream_t)stream>>>(U_prev, shift, n, U_prop,
                                                                                          U_plain);
    return cuda_status(cudaGetLastError());
}

extern "C" int exact_proposal_select(const float *costs_prop, const float *costs_plain, int B, int K,
                                     const float *U_prop, const float *U_plain, const float *u_prop,
                                     const float *u_plain, int T, int nu, float *U_out, float *u_out, int *chose_prop,
                                     void *stream) {
    if (B < 0 || K < 1 || T < 1 || nu < 1) return EXACT_EINVAL;
    if (B == 0) return EXACT_OK;
    if (!costs_prop || !costs_plain || !U_prop || !U_plain || !u_prop || !u_plain || !U_out || !u_out)
        return EXACT_EINVAL;
    proposal_select_kernel<<<B, 256, 0, (cudaStream_t)stream>>>(costs_prop, costs_plain, K, U_prop, U_plain, u_prop,
                                                                u_plain, T * nu, nu, U_out, u_out, chose_prop);
    return cuda_status(cudaGetLastError());
}
