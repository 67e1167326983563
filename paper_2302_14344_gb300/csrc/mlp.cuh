// Kernels of the warm-start network: a fully connected GELU network in BF16 with FP32
// accumulation (forward, backward, Adam).  The matrix products run on the tensor cores
// through warp-level mma.sync (m16n8k16, BF16 inputs, FP32 accumulators); the layers are
// small (32..256 wide), so a 64 x 64 block tile staged through shared memory is enough.
#pragma once

#include <cuda_bf16.h>

namespace wsn {

// C = op(A) op(B) with A(m, k) = A[m sam + k sak] and B(k, n) = B[k sbk + n sbn] (BF16),
// M x N x K; the epilogue decides what is written (see Epi).
struct Gemm {
    const __nv_bfloat16 *A, *B;
    long long sam, sak, sbk, sbn;
    int M, N, K;
    const float *bias;        // per column (BIAS, BIAS_GELU)
    const float *scale;       // per column, BIAS only: out = (C + bias) * scale (NULL: 1)
    float *out;               // FP32 output (ldo = N): C, C + bias, or the pre-activation
    __nv_bfloat16 *act;       // BF16 output (ldo = N): GELU(C + bias), or C * GELU'(pre)
    const float *pre;         // pre-activation read by GELU_BWD (ldo = N)
};

enum Epi { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float u)
{
    return 0.5f * (1.0f + erff(u * 0.70710678118654752f)) + u * 0.39894228040143268f * expf(-0.5f * u * u);
}

__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, const unsigned *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int TM = 64, TN = 64, TK = 32, PAD = 8;

// 4 warps in a 2 x 2 arrangement, each computing a 32 x 32 block of C as 2 x 4 tiles of
// m16n8.  Shared tiles: As[m][k] and Bs[n][k], k contiguous, rows padded by 8 BF16 so the
// 32-bit fragment loads of a warp hit 32 distinct banks.
template <int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(Gemm g)
{
    __shared__ __align__(16) __nv_bfloat16 As[TM][TK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[TN][TK + PAD];
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = 0; k0 < g.K; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 128) {
            const int r = e / TK, c = e - r * TK;
            const int m = m0 + r, n = n0 + r, k = k0 + c;
            As[r][c] = (m < g.M && k < g.K) ? g.A[m * g.sam + k * g.sak] : zero;
            Bs[r][c] = (n < g.N && k < g.K) ? g.B[k * g.sbk + n * g.sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm + 16 * i + gq;
                a[i][0] = *reinterpret_cast<const unsigned *>(&As[row][kk + 2 * tq]);
                a[i][1] = *reinterpret_cast<const unsigned *>(&As[row + 8][kk + 2 * tq]);
                a[i][2] = *reinterpret_cast<const unsigned *>(&As[row][kk + 2 * tq + 8]);
                a[i][3] = *reinterpret_cast<const unsigned *>(&As[row + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = wn + 8 * j + gq;
                b[j][0] = *reinterpret_cast<const unsigned *>(&Bs[col][kk + 2 * tq]);
                b[j][1] = *reinterpret_cast<const unsigned *>(&Bs[col][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    // accumulator (i, j, q): row wm + 16 i + gq (+ 8 for q >= 2), column wn + 8 j + 2 tq + (q & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + 16 * i + gq + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tq + (q & 1);
                if (m >= g.M || n >= g.N) continue;
                const long long o = (long long)m * g.N + n;
                const float c = acc[i][j][q];
                if (EPI == EPI_STORE) {
                    g.out[o] = c;
                } else if (EPI == EPI_BIAS) {
                    g.out[o] = g.scale ? (c + g.bias[n]) * g.scale[n] : c + g.bias[n];
                } else if (EPI == EPI_BIAS_GELU) {
                    const float u = c + g.bias[n];
                    g.out[o] = u;
                    g.act[o] = __float2bfloat16(gelu_f(u));
                } else {
                    g.act[o] = __float2bfloat16(c * gelu_grad_f(g.pre[o]));
                }
            }
        }
    }
}

// x (FP32) -> BF16 ((x - mean) / std per column)
__global__ void normalize_kernel(const float *x, long long ldx, const float *mean,
                                 const float *inv_std, __nv_bfloat16 *xb, int B, int D)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * D;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / D;
        const int d = (int)(i - b * D);
        xb[i] = __float2bfloat16((x[b * ldx + d] - mean[d]) * inv_std[d]);
    }
}

// output gradient g = mask (y - t / scale) / B (BF16) and the loss sum of
// mask (y - t / scale)^2 / (2B)
__global__ void output_grad_kernel(const float *y, const float *t, const float *mask,
                                   const float *scale, __nv_bfloat16 *g, int B, int N,
                                   float *loss)
{
    float part = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * N;
         i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i % N);
        const float r = y[i] - t[i] / scale[n];
        const float d = mask[i] * r;
        g[i] = __float2bfloat16(d / (float)B);
        part += d * r;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, 0.5f * part / (float)B);
}

// Per-column statistics of a B x D FP32 matrix (leading dimension ld), one block of 256
// threads per column, FP64 partial sums reduced in a fixed tree order (deterministic).
// mode 1: mean and 1 / std (std < 1e-6 gives 1); mode 0: scale = root mean square (0 -> 1).
__global__ void column_stats_kernel(const float *x, long long ld, int B, int D, float *mean,
                                    float *second, int mode)
{
    __shared__ double s1[256], s2[256];
    const int d = blockIdx.x;
    if (d >= D) return;
    double a = 0.0, q = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const double v = (double)x[(long long)b * ld + d];
        a += v;
        q += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = q;
    __syncthreads();
    for (int w = blockDim.x / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mu = s1[0] / B, ms = s2[0] / B;
        if (mode == 1) {
            const double var = ms - mu * mu;
            const double sd = var > 1e-12 ? sqrt(var) : 1.0;
            mean[d] = (float)mu;
            second[d] = (float)(1.0 / sd);
        } else {
            const double rms = sqrt(ms);
            second[d] = rms > 0.0 ? (float)rms : 1.0f;
        }
    }
}

// column sums of a B x N BF16 matrix into FP32 (bias gradients).  A block of 32 x 8 threads
// takes 32 columns: each of its 8 row groups sums rows g, g + 8, ... in order, then the 8
// partial sums are added in group order (a fixed order: deterministic).
__global__ void __launch_bounds__(256) column_sum_kernel(const __nv_bfloat16 *g, int B, int N, float *out)
{
    __shared__ float part[8][33];
    const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + c;
    float s = 0.0f;
    if (n < N)
        for (int b = r; b < B; b += 8) s += __bfloat162float(g[(long long)b * N + n]);
    part[r][c] = s;
    __syncthreads();
    if (r == 0 && n < N) {
        float t = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += part[q][c];
        out[n] = t;
    }
}

// Adam (bias-corrected) on the FP32 master parameters; refreshes their BF16 copies
__global__ void adam_kernel(float *p, __nv_bfloat16 *pb, const float *grad, float *m, float *v,
                            long long n, float lr, float beta1, float beta2, float eps, float c1,
                            float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float mi = beta1 * m[i] + (1.0f - beta1) * gr;
        const float vi = beta2 * v[i] + (1.0f - beta2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = w;
        if (pb) pb[i] = __float2bfloat16(w);
    }
}

__global__ void to_bf16_kernel(const float *x, __nv_bfloat16 *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

}  // namespace wsn
