// mlp.cu -- the learned sampling proposal's network on the tensor cores.
//
// y = W3 g(W2 g(W1 x + b1) + b2) + b3 with the exact GELU g(z) = z Phi(z).
// Every product is a BF16 x BF16 -> FP32 tensor-core GEMM (mma.sync
// m16n8k16: the matrices are a few hundred wide, far below the sizes where
// the tcgen05 / TMEM pipeline would pay off).  FP32 master weights and Adam
// moments; BF16 copies of the weights and of every GEMM operand
// (activations, output and hidden gradients); FP32 pre-activations for the
// GELU derivative; FP32 gradients.
//
// One generic tiled GEMM serves all products through strided operand views
// (C[i][j] = sum_k A(i,k) B(k,j), A(i,k) = A[i sar + k sac]), so forward
// (X W^T), input gradients (dZ W) and weight gradients (dZ^T H) are the same
// kernel with different strides and epilogues.  Weight gradients reduce over
// the batch (K = B) into few output tiles; they are split along K over
// gridDim.z into FP32 partial tiles, added in a fixed order afterwards.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace exact {

typedef __nv_bfloat16 bf16;

constexpr int GM = 64, GN = 64, GK = 32, GPAD = 8;   // block tile, k step, smem row padding
constexpr int kMlpInPad = 128;                        // inputs are zero-padded to this width

enum { EPI_PLAIN = 0, EPI_BIAS_GELU = 1, EPI_GELU_GRAD = 2, EPI_BIAS = 3 };

struct GemmArgs {
    int M, N, K;
    const bf16 *A;
    long long sar, sac;
    const bf16 *B;
    long long sbr, sbc;
    float *C;          // FP32 result (row-major, ldc)
    int ldc;
    bf16 *Cb;          // optional BF16 result (row-major, ldcb)
    int ldcb;
    const float *bias; // per column j
    const float *gz;   // pre-activation for EPI_GELU_GRAD (row-major, ldgz)
    int ldgz;
    int epi;
    int kchunk;        // k range of one block along gridDim.z (split-K); K when unsplit
    float *P;          // split-K: FP32 partial tiles P[z][i][j] (M x N each), summed by splitk_sum_kernel
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// 64 x 64 output tile per block (4 warps, 32 x 32 each = 2 x 4 mma tiles of
// 16 x 8), k in steps of 32 staged through shared memory.  A is staged as
// As[i][k], B transposed as Bs[j][k], so both fragments are pairs of
// consecutive k (one 32-bit load each).  Out-of-range elements are zero.
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
    __shared__ __align__(16) bf16 As[GM][GK + GPAD];
    __shared__ __align__(16) bf16 Bs[GN][GK + GPAD];
    const int i0 = blockIdx.y * GM, j0 = blockIdx.x * GN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int gid = lane >> 2, t4 = lane & 3;
    const bf16 zero = __float2bfloat16_rn(0.f);
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

    const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
    for (int k0 = kb; k0 < ke; k0 += GK) {
        for (int e = threadIdx.x; e < GM * GK; e += 128) {
            const int r = e / GK, c = e - r * GK, i = i0 + r, k = k0 + c;
            As[r][c] = (i < g.M && k < ke) ? g.A[(long long)i * g.sar + (long long)k * g.sac] : zero;
        }
        for (int e = threadIdx.x; e < GN * GK; e += 128) {
            const int r = e / GK, c = e - r * GK, j = j0 + r, k = k0 + c;
            Bs[r][c] = (j < g.N && k < ke) ? g.B[(long long)k * g.sbr + (long long)j * g.sbc] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk += 16) {
            uint32_t af[2][4], bfm[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int row = wm * 32 + mi * 16 + gid;
                af[mi][0] = ld_pair(&As[row][kk + 2 * t4]);
                af[mi][1] = ld_pair(&As[row + 8][kk + 2 * t4]);
                af[mi][2] = ld_pair(&As[row][kk + 2 * t4 + 8]);
                af[mi][3] = ld_pair(&As[row + 8][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int col = wn * 32 + ni * 8 + gid;
                bfm[ni][0] = ld_pair(&Bs[col][kk + 2 * t4]);
                bfm[ni][1] = ld_pair(&Bs[col][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfm[ni]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = i0 + wm * 32 + mi * 16 + gid + 8 * h;
                    const int j = j0 + wn * 32 + ni * 8 + 2 * t4 + c;
                    if (i >= g.M || j >= g.N) continue;
                    float v = acc[mi][ni][2 * h + c];
                    if (g.P) {   // split-K: this block's partial, no epilogue
                        g.P[((long long)blockIdx.z * g.M + i) * g.N + j] = v;
                        continue;
                    }
                    float out = v;
                    if (g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU) v += g.bias[j];
                    if (g.epi == EPI_BIAS_GELU) {
                        out = v;                               // pre-activation kept in C
                        if (g.Cb) g.Cb[(long long)i * g.ldcb + j] = __float2bfloat16_rn(gelu_f(v));
                    } else if (g.epi == EPI_GELU_GRAD) {
                        out = v * gelu_grad_f(g.gz[(long long)i * g.ldgz + j]);
                        if (g.Cb) g.Cb[(long long)i * g.ldcb + j] = __float2bfloat16_rn(out);
                    } else {
                        out = v;
                        if (g.Cb) g.Cb[(long long)i * g.ldcb + j] = __float2bfloat16_rn(out);
                    }
                    if (g.C) g.C[(long long)i * g.ldc + j] = out;
                }
}

// C[i][j] (row stride ldc) = sum_z P[z][i][j], z in order (fixed, so the
// result does not depend on scheduling)
__global__ void splitk_sum_kernel(const float *__restrict__ P, int S, int M, int N, float *__restrict__ C, int ldc) {
    const long long n = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int z = 0; z < S; ++z) a += P[z * n + e];
        C[(e / N) * ldc + e % N] = a;
    }
}

// x (B x d_in, FP32) -> Xb (B x 128, BF16, zero-padded)
__global__ void pack_input_kernel(const float *__restrict__ x, int B, int d_in, bf16 *__restrict__ Xb) {
    const long long n = (long long)B * kMlpInPad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / kMlpInPad), d = (int)(e - (long long)b * kMlpInPad);
        Xb[e] = __float2bfloat16_rn(d < d_in ? x[(long long)b * d_in + d] : 0.f);
    }
}

// dY = 2 (Y - target) / (B O) (FP32 and BF16) and the mean squared error
// (one block, fixed reduction order).
__global__ void __launch_bounds__(1024)
mse_grad_kernel(const float *__restrict__ Y, const float *__restrict__ tgt, int B, int O, float *__restrict__ dY,
                bf16 *__restrict__ dYb, float *__restrict__ loss) {
    __shared__ double s[32];
    const long long n = (long long)B * O;
    const float scale = 2.f / (float)n;
    double acc = 0.0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const float d = Y[e] - tgt[e];
        acc += (double)d * (double)d;
        const float gv = d * scale;
        dY[e] = gv;
        dYb[e] = __float2bfloat16_rn(gv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        if (loss) *loss = (float)(t / (double)n);
    }
}

// Bias gradients g[j] = sum_b D[b][j] in two fixed-order stages: slice s of
// kColSlices adds its rows b = s, s + kColSlices, ... (one thread per column,
// coalesced across columns), then colsum_finish adds the slices in order.
constexpr int kColSlices = 32;
__global__ void colsum_kernel(const float *__restrict__ D, int B, int n, float *__restrict__ part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, sl = blockIdx.y;
    if (j >= n) return;
    float a = 0.f;
    for (int b = sl; b < B; b += kColSlices) a += D[(long long)b * n + j];
    part[(long long)sl * n + j] = a;
}
__global__ void colsum_finish_kernel(const float *__restrict__ part, int n, float *__restrict__ g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float a = 0.f;
    for (int sl = 0; sl < kColSlices; ++sl) a += part[(long long)sl * n + j];
    g[j] = a;
}

// Adam (Kingma & Ba) on the packed FP32 parameters; c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// BF16 copy of a row-major FP32 matrix (rows x cols) into a row stride `ld`
// (columns cols..ld-1 are zero).
__global__ void to_bf16_kernel(const float *__restrict__ W, int rows, int cols, int ld, bf16 *__restrict__ Wb) {
    const long long n = (long long)rows * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ld), c = (int)(e - (long long)r * ld);
        Wb[e] = __float2bfloat16_rn(c < cols ? W[(long long)r * cols + c] : 0.f);
    }
}

}  // namespace exact

using namespace exact;

struct exact_mlp {
    int din = 0, H = 0, O = 0, maxB = 0;
    long long nparam = 0;
    long long oW1, ob1, oW2, ob2, oW3, ob3;   // offsets into the packed parameter vector
    void *dev = nullptr;
    float *w, *g, *m, *v;                     // packed FP32 parameters, gradients, moments
    bf16 *W1b, *W2b, *W3b;                    // BF16 weights (W1b rows padded to 128)
    bf16 *Xb, *H1b, *H2b, *dYb, *dZb;         // BF16 operands
    float *Z1, *Z2, *Y, *dY, *dZ, *loss;      // FP32 activations / gradients
    float *ws;                                // split-K partial tiles and column-sum slices
    int t = 0;                                // Adam step
};

// split-K factor of a GEMM whose output tiles would not fill the GPU
constexpr int kSplitMax = 16;
static int splits_for(int M, int N, int K) {
    const int tiles = ((M + GM - 1) / GM) * ((N + GN - 1) / GN);
    int s = 1;
    while (s < kSplitMax && tiles * s * 2 <= 152 && K / (s * 2) >= 2 * GK) s *= 2;
    return s;
}

static int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

static cudaError_t gemm(const GemmArgs &g0, cudaStream_t st, float *ws = nullptr) {
    GemmArgs g = g0;
    // weight gradients (no epilogue, K = the batch) are split along K into
    // partial tiles when their output tiles alone would not fill the GPU
    const int S = (ws && g.epi == EPI_PLAIN && !g.Cb) ? splits_for(g.M, g.N, g.K) : 1;
    g.kchunk = S > 1 ? ((g.K + S - 1) / S + GK - 1) / GK * GK : g.K;
    g.P = S > 1 ? ws : nullptr;
    dim3 grid((g.N + GN - 1) / GN, (g.M + GM - 1) / GM, S);
    gemm_bf16_kernel<<<grid, 128, 0, st>>>(g);
    if (S > 1) {
        const long long n = (long long)g.M * g.N;
        splitk_sum_kernel<<<(int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(ws, S, g.M, g.N, g.C,
                                                                                               g.ldc);
    }
    return cudaGetLastError();
}

static void colsum(const float *D, int B, int n, float *g, float *ws, cudaStream_t st) {
    colsum_kernel<<<dim3((n + 127) / 128, kColSlices), 128, 0, st>>>(D, B, n, ws);
    colsum_finish_kernel<<<(n + 127) / 128, 128, 0, st>>>(ws, n, g);
}

static GemmArgs make_gemm(int M, int N, int K, const bf16 *A, long long sar, long long sac, const bf16 *B, long long sbr,
                          long long sbc, float *C, int ldc, int epi) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.sar = sar; g.sac = sac;
    g.B = B; g.sbr = sbr; g.sbc = sbc;
    g.C = C; g.ldc = ldc;
    g.epi = epi;
    return g;
}

static int refresh_bf16(exact_mlp *m, cudaStream_t st) {
    to_bf16_kernel<<<grid_for((long long)m->H * kMlpInPad, 256), 256, 0, st>>>(m->w + m->oW1, m->H, m->din, kMlpInPad, m->W1b);
    to_bf16_kernel<<<grid_for((long long)m->H * m->H, 256), 256, 0, st>>>(m->w + m->oW2, m->H, m->H, m->H, m->W2b);
    to_bf16_kernel<<<grid_for((long long)m->O * m->H, 256), 256, 0, st>>>(m->w + m->oW3, m->O, m->H, m->H, m->W3b);
    return cuda_status(cudaGetLastError());
}

// forward: Xb -> Z1 (pre-act), H1b -> Z2, H2b -> Y
static int forward(exact_mlp *m, const float *x, int B, float *y, cudaStream_t st) {
    pack_input_kernel<<<grid_for((long long)B * kMlpInPad, 256), 256, 0, st>>>(x, B, m->din, m->Xb);
    const int H = m->H, O = m->O;
    GemmArgs g1 = make_gemm(B, H, kMlpInPad, m->Xb, kMlpInPad, 1, m->W1b, 1, kMlpInPad, m->Z1, H, EPI_BIAS_GELU);
    g1.bias = m->w + m->ob1; g1.Cb = m->H1b; g1.ldcb = H;
    GemmArgs g2 = make_gemm(B, H, H, m->H1b, H, 1, m->W2b, 1, H, m->Z2, H, EPI_BIAS_GELU);
    g2.bias = m->w + m->ob2; g2.Cb = m->H2b; g2.ldcb = H;
    GemmArgs g3 = make_gemm(B, O, H, m->H2b, H, 1, m->W3b, 1, H, y, O, EPI_BIAS);
    g3.bias = m->w + m->ob3;
    if (gemm(g1, st) != cudaSuccess || gemm(g2, st) != cudaSuccess || gemm(g3, st) != cudaSuccess) return EXACT_ECUDA;
    return EXACT_OK;
}

// loss and gradients into m->g (packed like the parameters)
static int backward(exact_mlp *m, const float *x, const float *target, int B, cudaStream_t st) {
    int rc = forward(m, x, B, m->Y, st);
    if (rc != EXACT_OK) return rc;
    const int H = m->H, O = m->O, D = m->din;
    mse_grad_kernel<<<1, 1024, 0, st>>>(m->Y, target, B, O, m->dY, m->dYb, m->loss);
    // layer 3: gW3 = dY^T H2, gb3 = sum dY, dZ2 = (dY W3) * g'(Z2)
    GemmArgs a = make_gemm(O, H, B, m->dYb, 1, O, m->H2b, H, 1, m->g + m->oW3, H, EPI_PLAIN);
    colsum(m->dY, B, O, m->g + m->ob3, m->ws, st);
    GemmArgs b = make_gemm(B, H, O, m->dYb, O, 1, m->W3b, H, 1, m->dZ, H, EPI_GELU_GRAD);
    b.gz = m->Z2; b.ldgz = H; b.Cb = m->dZb; b.ldcb = H;
    if (gemm(a, st, m->ws) != cudaSuccess || gemm(b, st) != cudaSuccess) return EXACT_ECUDA;
    // layer 2: gW2 = dZ2^T H1, gb2 = sum dZ2, dZ1 = (dZ2 W2) * g'(Z1)
    GemmArgs c = make_gemm(H, H, B, m->dZb, 1, H, m->H1b, H, 1, m->g + m->oW2, H, EPI_PLAIN);
    colsum(m->dZ, B, H, m->g + m->ob2, m->ws, st);
    if (gemm(c, st, m->ws) != cudaSuccess) return EXACT_ECUDA;
    // dZ1 overwrites dZ / dZb only after gW2 and gb2 have consumed them (stream order)
    GemmArgs d = make_gemm(B, H, H, m->dZb, H, 1, m->W2b, H, 1, m->Z2, H, EPI_GELU_GRAD);
    d.gz = m->Z1; d.ldgz = H; d.Cb = m->H2b; d.ldcb = H;   // Z2 / H2b are free after layer 2's backward
    if (gemm(d, st) != cudaSuccess) return EXACT_ECUDA;
    // layer 1: gW1 = dZ1^T X (only the d_in real columns), gb1 = sum dZ1
    GemmArgs e = make_gemm(H, D, B, m->H2b, 1, H, m->Xb, kMlpInPad, 1, m->g + m->oW1, D, EPI_PLAIN);
    colsum(m->Z2, B, H, m->g + m->ob1, m->ws, st);
    if (gemm(e, st, m->ws) != cudaSuccess) return EXACT_ECUDA;
    return cuda_status(cudaGetLastError());
}

extern "C" int exact_mlp_create(int d_in, int hidden, int d_out, int max_batch, exact_mlp **out) {
    if (!out) return EXACT_EINVAL;
    *out = nullptr;
    if (d_in < 1 || hidden < 1 || d_out < 1 || max_batch < 1) return EXACT_EINVAL;
    if (d_in > kMlpInPad || hidden > 1024 || d_out > 256 || max_batch > (1 << 20)) return EXACT_ECAPACITY;
    exact_mlp *m = new (std::nothrow) exact_mlp();
    if (!m) return EXACT_EINVAL;
    m->din = d_in; m->H = hidden; m->O = d_out; m->maxB = max_batch;
    const long long H = hidden, D = d_in, O = d_out, B = max_batch;
    m->oW1 = 0; m->ob1 = H * D; m->oW2 = m->ob1 + H; m->ob2 = m->oW2 + H * H; m->oW3 = m->ob2 + H;
    m->ob3 = m->oW3 + O * H;
    m->nparam = m->ob3 + O;
    std::vector<size_t> sz = {
        (size_t)m->nparam * 4, (size_t)m->nparam * 4, (size_t)m->nparam * 4, (size_t)m->nparam * 4,   // w g m v
        (size_t)(H * kMlpInPad) * 2, (size_t)(H * H) * 2, (size_t)(O * H) * 2,                          // W1b W2b W3b
        (size_t)(B * kMlpInPad) * 2, (size_t)(B * H) * 2, (size_t)(B * H) * 2, (size_t)(B * O) * 2,      // Xb H1b H2b dYb
        (size_t)(B * H) * 2,                                                                             // dZb
        (size_t)(B * H) * 4, (size_t)(B * H) * 4, (size_t)(B * O) * 4, (size_t)(B * O) * 4,              // Z1 Z2 Y dY
        (size_t)(B * H) * 4, 256,                                                                        // dZ loss
        (size_t)kSplitMax * (size_t)std::max(H * std::max(H, D), O * H) * 4};                           // ws
    size_t total = 0;
    for (auto s : sz) total += align_up(s, 256);
    if (cudaMalloc(&m->dev, total) != cudaSuccess) { delete m; return EXACT_ECUDA; }
    if (cudaMemset(m->dev, 0, total) != cudaSuccess) { cudaFree(m->dev); delete m; return EXACT_ECUDA; }
    char *p = static_cast<char *>(m->dev);
    void **slots[] = {(void **)&m->w, (void **)&m->g, (void **)&m->m, (void **)&m->v, (void **)&m->W1b,
                      (void **)&m->W2b, (void **)&m->W3b, (void **)&m->Xb, (void **)&m->H1b, (void **)&m->H2b,
                      (void **)&m->dYb, (void **)&m->dZb, (void **)&m->Z1, (void **)&m->Z2, (void **)&m->Y,
                      (void **)&m->dY, (void **)&m->dZ, (void **)&m->loss, (void **)&m->ws};
    for (size_t i = 0; i < sz.size(); ++i) {
        *slots[i] = p;
        p += align_up(sz[i], 256);
    }
    *out = m;
    return EXACT_OK;
}

extern "C" void exact_mlp_destroy(exact_mlp *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->dev);
    delete m;
}

extern "C" long long exact_mlp_num_params(const exact_mlp *m) { return m ? m->nparam : -1; }

extern "C" int exact_mlp_set_params(exact_mlp *m, const float *host_params) {
    if (!m || !host_params) return EXACT_EINVAL;
    for (long long k = 0; k < m->nparam; ++k)
        if (!isfinite(host_params[k])) return EXACT_EINVAL;
    if (cudaMemcpy(m->w, host_params, (size_t)m->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess) return EXACT_ECUDA;
    if (cudaMemset(m->m, 0, (size_t)m->nparam * 4) != cudaSuccess ||
        cudaMemset(m->v, 0, (size_t)m->nparam * 4) != cudaSuccess)
        return EXACT_ECUDA;
    m->t = 0;
    const int rc = refresh_bf16(m, 0);
    if (rc != EXACT_OK) return rc;
    return cuda_status(cudaDeviceSynchronize());
}

extern "C" int exact_mlp_get_params(const exact_mlp *m, float *host_params) {
    if (!m || !host_params) return EXACT_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return EXACT_ECUDA;
    return cuda_status(cudaMemcpy(host_params, m->w, (size_t)m->nparam * 4, cudaMemcpyDeviceToHost));
}

extern "C" int exact_mlp_get_state(const exact_mlp *m, float *host_params, float *host_m, float *host_v,
                                   long long *step) {
    if (!m || !host_params || !host_m || !host_v || !step) return EXACT_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return EXACT_ECUDA;
    const size_t bytes = (size_t)m->nparam * 4;
    if (cudaMemcpy(host_params, m->w, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host_m, m->m, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host_v, m->v, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return EXACT_ECUDA;
    *step = m->t;
    return EXACT_OK;
}

extern "C" int exact_mlp_set_state(exact_mlp *m, const float *host_params, const float *host_m, const float *host_v,
                                   long long step) {
    if (!m || !host_params || !host_m || !host_v || step < 0 || step > (1ll << 30)) return EXACT_EINVAL;
    for (long long k = 0; k < m->nparam; ++k)
        if (!isfinite(host_params[k]) || !isfinite(host_m[k]) || !(host_v[k] >= 0.f) || !isfinite(host_v[k]))
            return EXACT_EINVAL;
    const size_t bytes = (size_t)m->nparam * 4;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(m->w, host_params, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->m, host_m, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->v, host_v, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return EXACT_ECUDA;
    m->t = (int)step;
    const int rc = refresh_bf16(m, 0);
    if (rc != EXACT_OK) return rc;
    return cuda_status(cudaDeviceSynchronize());
}

extern "C" int exact_mlp_forward(exact_mlp *m, const float *x, int B, float *y, void *stream) {
    if (!m || !x || !y || B < 0) return EXACT_EINVAL;
    if (B == 0) return EXACT_OK;
    if (B > m->maxB) return EXACT_ECAPACITY;
    return forward(m, x, B, y, (cudaStream_t)stream);
}

extern "C" int exact_mlp_loss_grad(exact_mlp *m, const float *x, const float *target, int B, float *loss,
                                   float *grads, void *stream) {
    if (!m || !x || !target || B < 1) return EXACT_EINVAL;
    if (B > m->maxB) return EXACT_ECAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    const int rc = backward(m, x, target, B, st);
    if (rc != EXACT_OK) return rc;
    if (loss && cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return EXACT_ECUDA;
    if (grads && cudaMemcpyAsync(grads, m->g, (size_t)m->nparam * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return EXACT_ECUDA;
    return EXACT_OK;
}

extern "C" int exact_mlp_train_step(exact_mlp *m, const float *x, const float *target, int B, float lr, float *loss,
                                    void *stream) {
    if (!m || !x || !target || B < 1 || !(lr > 0.f)) return EXACT_EINVAL;
    if (B > m->maxB) return EXACT_ECAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = backward(m, x, target, B, st);
    if (rc != EXACT_OK) return rc;
    m->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, m->t)), c2 = (float)(1.0 - pow(b2, m->t));
    adam_kernel<<<grid_for(m->nparam, 256), 256, 0, st>>>(m->w, m->g, m->m, m->v, m->nparam, lr, (float)b1, (float)b2,
                                                          1e-8f, c1, c2);
    if ((rc = refresh_bf16(m, st)) != EXACT_OK) return rc;
    if (loss && cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return EXACT_ECUDA;
    return cuda_status(cudaGetLastError());
}
