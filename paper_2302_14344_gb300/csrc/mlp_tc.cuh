// Fused inference of the warm-start network (32 -> 256 -> 256 -> 256 -> 7, GELU) on the
// 5th-generation tensor cores: one persistent launch runs all four layers for 128 interfaces
// at a time.  Per tile the normalised inputs are written to shared memory as BF16 (the
// 128-byte swizzled K-major layout the MMA reads); for each layer one thread streams the
// layer's packed weights through a two-stage ring by TMA (cp.async.bulk.tensor) and issues
// tcgen05.mma kind::f16 (BF16 operands, FP32 accumulator in tensor memory, M = 128); four
// warps then read the accumulator (tcgen05.ld), add the bias, apply GELU and write the BF16
// activations into the other shared-memory buffer, which the next layer reads; the last layer
// adds its bias, applies the output scale and stores FP32 outputs.  The numerics are those of
// the layer-by-layer path: BF16 weights and activations, FP32 accumulation, exact GELU.
//
// Every wait is bounded (1 s): a wait that runs out raises the error word and the block
// stops; tensor memory is freed on every path.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wsn {

constexpr int kMlpIn = 32, kMlpInPad = 64, kMlpHidden = 256, kMlpOut = 7, kMlpOutPad = 16;
constexpr int kMlpRows = 128;                          // interfaces per tile (MMA M)
constexpr int kMlpActBytes = kMlpRows * kMlpHidden * 2;        // 64 KB: one activation buffer
constexpr int kMlpStageBytes = kMlpHidden * 128;               // 32 KB: 256 rows x 64 BF16
constexpr int kMlpSmem = 2 * kMlpActBytes + 2 * kMlpStageBytes + 1024;
constexpr int kMlpThreads = 128;
constexpr unsigned long long kMlpWaitNs = 1000000000ull;

struct MlpArgs {
    const float *x;        // inputs, batch x ldx
    long long ldx;
    int batch;
    const float *mean, *inv_std;   // input normalisation
    const float *bias[4];  // FP32 biases of the layers
    const float *scale;    // output scale
    float *y;              // outputs, batch x 7
    int *err;
};

__device__ __forceinline__ uint32_t mlp_s32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long mlp_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mlp_wait(uint64_t *b, unsigned parity, volatile int *abort_flag)
{
    unsigned ok;
    const unsigned long long t0 = mlp_ns();
    for (;;) {
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(mlp_s32(b)), "r"(parity) : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (mlp_ns() - t0 > kMlpWaitNs) return false;
    }
}

// shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t mlp_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) |
           ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, K-major, M = 128, N = n
__device__ __forceinline__ uint32_t mlp_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kMlpRows >> 4) << 24);
}

__device__ __forceinline__ float mlp_gelu(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }

// eight BF16 values into row r, K offset k0 (a multiple of 8) of a swizzled K-major buffer
// of 64-wide K blocks (each 128 rows x 128 bytes)
__device__ __forceinline__ void mlp_put8(unsigned char *buf, int r, int k0, uint4 v)
{
    const int kb = k0 >> 6, c = (k0 & 63) >> 3;
    *reinterpret_cast<uint4 *>(buf + kb * (kMlpRows * 128) + r * 128 + ((c ^ (r & 7)) << 4)) = v;
}

__device__ __forceinline__ uint32_t mlp_pack2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <int N>
__device__ __forceinline__ void mlp_tmem_ld(uint32_t taddr, float *v);

template <>
__device__ __forceinline__ void mlp_tmem_ld<32>(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

template <>
__device__ __forceinline__ void mlp_tmem_ld<16>(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// packed weights: layer l as (N_l rows of K_l BF16, K-major): Wt[n][k] = W_l[k][n]
__global__ void mlp_pack_kernel(const __nv_bfloat16 *pb, long long o0, long long o1, long long o2,
                                long long o3, __nv_bfloat16 *w0, __nv_bfloat16 *w1,
                                __nv_bfloat16 *w2, __nv_bfloat16 *w3)
{
    const int total = kMlpHidden * kMlpInPad + 2 * kMlpHidden * kMlpHidden + kMlpOutPad * kMlpHidden;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int q = i;
        if (q < kMlpHidden * kMlpInPad) {
            const int n = q / kMlpInPad, k = q % kMlpInPad;
            w0[q] = k < kMlpIn ? pb[o0 + (long long)k * kMlpHidden + n] : __float2bfloat16(0.0f);
            continue;
        }
        q -= kMlpHidden * kMlpInPad;
        if (q < 2 * kMlpHidden * kMlpHidden) {
            const int l = q / (kMlpHidden * kMlpHidden), r = q % (kMlpHidden * kMlpHidden);
            const int n = r / kMlpHidden, k = r % kMlpHidden;
            (l ? w2 : w1)[r] = pb[(l ? o2 : o1) + (long long)k * kMlpHidden + n];
            continue;
        }
        q -= 2 * kMlpHidden * kMlpHidden;
        const int n = q / kMlpHidden, k = q % kMlpHidden;
        w3[q] = n < kMlpOut ? pb[o3 + (long long)k * kMlpOut + n] : __float2bfloat16(0.0f);
    }
}

__global__ void __launch_bounds__(kMlpThreads, 1)
mlp_fused_kernel(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
                 const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap m3,
                 const MlpArgs a)
{
    extern __shared__ unsigned char mlp_raw[];
    __shared__ __align__(8) uint64_t full[2], empty[2], acc;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(mlp_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *act[2] = {smem, smem + kMlpActBytes};
    unsigned char *stage[2] = {smem + 2 * kMlpActBytes, smem + 2 * kMlpActBytes + kMlpStageBytes};
    const CUtensorMap *maps[4] = {&m0, &m1, &m2, &m3};
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mlp_s32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mlp_s32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mlp_s32(&acc)) : "memory");
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(mlp_s32(&tmem_base)), "r"(kMlpHidden) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    unsigned fcnt[2] = {0, 0}, ecnt[2] = {0, 0}, acnt = 0;   // completions issued so far
    const int tiles = (a.batch + kMlpRows - 1) / kMlpRows;
    for (int tile = blockIdx.x; tile < tiles && !abort_flag; tile += gridDim.x) {
        const int row = tile * kMlpRows + tid;
        // ---- inputs: (x - mean) / std in BF16, K padded to 64 with zeros
        {
            float v[kMlpInPad];
#pragma unroll
            for (int k = 0; k < kMlpInPad; ++k) v[k] = 0.0f;
            if (row < a.batch) {
                const float *xr = a.x + (long long)row * a.ldx;
#pragma unroll
                for (int k = 0; k < kMlpIn; ++k) v[k] = (xr[k] - a.mean[k]) * a.inv_std[k];
            }
#pragma unroll
            for (int k = 0; k < kMlpInPad; k += 8)
                mlp_put8(act[0], tid, k, make_uint4(mlp_pack2(v[k], v[k + 1]), mlp_pack2(v[k + 2], v[k + 3]),
                                                    mlp_pack2(v[k + 4], v[k + 5]), mlp_pack2(v[k + 6], v[k + 7])));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        for (int l = 0; l < 4; ++l) {
            const int K = l == 0 ? kMlpInPad : kMlpHidden, N = l == 3 ? kMlpOutPad : kMlpHidden;
            const int nk = K / 64;
            unsigned char *ain = act[l & 1], *aout = act[(l + 1) & 1];
            const unsigned bytes = (unsigned)N * 128;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool ok = true;
                auto load = [&](int kc) {
                    const int s = kc & 1;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 ::"r"(mlp_s32(&full[s])), "r"(bytes) : "memory");
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];"
                                 ::"r"(mlp_s32(stage[s])), "l"(reinterpret_cast<uint64_t>(maps[l])),
                                   "r"(kc * 64), "r"(0), "r"(mlp_s32(&full[s])) : "memory");
                    ++fcnt[s];
                };
                load(0);
                if (nk > 1) load(1);
                for (int kc = 0; kc < nk && ok; ++kc) {
                    const int s = kc & 1;
                    if (!mlp_wait(&full[s], (fcnt[s] - 1) & 1u, &abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ad = mlp_desc(mlp_s32(ain + kc * (kMlpRows * 128)));
                    const uint64_t bd = mlp_desc(mlp_s32(stage[s]));
                    const uint32_t idesc = mlp_idesc(N);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t accum = (kc > 0 || j > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\t"
                                     "setp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     ::"r"(tmem), "l"(ad + 2 * j), "l"(bd + 2 * j), "r"(idesc), "r"(accum)
                                     : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(mlp_s32(&empty[s])) : "memory");
                    ++ecnt[s];
                    if (kc + 2 < nk) {
                        if (!mlp_wait(&empty[s], (ecnt[s] - 1) & 1u, &abort_flag)) { ok = false; break; }
                        load(kc + 2);
                    }
                }
                if (!ok) { abort_flag = 1; atomicExch(a.err, 1); }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(mlp_s32(&acc)) : "memory");
            }
            ++acnt;
            __syncwarp();
            const bool got = mlp_wait(&acc, (acnt - 1) & 1u, &abort_flag);
            if (!__all_sync(0xffffffffu, got)) { abort_flag = 1; atomicExch(a.err, 1); }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            if (l < 3) {
                const float *bias = a.bias[l];
                for (int cb = 0; cb < kMlpHidden; cb += 32) {
                    float v[32];
                    mlp_tmem_ld<32>(trow + (uint32_t)cb, v);
#pragma unroll
                    for (int k = 0; k < 32; k += 8) {
                        float g[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) g[q] = mlp_gelu(v[k + q] + bias[cb + k + q]);
                        mlp_put8(aout, tid, cb + k, make_uint4(mlp_pack2(g[0], g[1]), mlp_pack2(g[2], g[3]),
                                                               mlp_pack2(g[4], g[5]), mlp_pack2(g[6], g[7])));
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            } else {
                float v[16];
                mlp_tmem_ld<16>(trow, v);
                if (row < a.batch)
#pragma unroll
                    for (int n = 0; n < kMlpOut; ++n)
                        a.y[(long long)row * kMlpOut + n] = (v[n] + a.bias[3][n]) * a.scale[n];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (abort_flag) break;
        }
    }
    // teardown: nothing may still write shared or tensor memory
    if (tid == 0) {
        volatile int never = 0;
        for (int s = 0; s < 2; ++s) {
            if (fcnt[s]) mlp_wait(&full[s], (fcnt[s] - 1) & 1u, &never);
            if (ecnt[s]) mlp_wait(&empty[s], (ecnt[s] - 1) & 1u, &never);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"(kMlpHidden) : "memory");
}

}  // namespace wsn
