// Gram matrices on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Per step and subsystem the v-step's affine map needs D = W^T W and c = W^T g with
// W = L^-1 J^T and g = L^-1 b (Algorithm 1's per-step factorise, carried through to the
// constraint space; Eq. admm-1i reassociated as x = c + D w).  With the right-hand side b
// appended as W's last column, [D c; c^T g^T g] is one Gram matrix G = W^T W of the
// (m + 1) columns of W: a dense contraction over the n DOF of the subsystem, the only
// GEMM-shaped work of the step.  These kernels form G on the tensor cores:
//
//   gram_prep_kernel  W (n x ldw, DOF-major: the layout the triangular solves write) is
//                     transposed into a stacked, K-major buffer of TF32 pairs: each value
//                     x = hi + lo with hi = x rounded to TF32 and lo = x - hi (exact in
//                     FP32), every job's rows padded with zeros to a multiple of 128 and
//                     its K extent with zeros to the buffer's row length.
//   gram_tc_kernel    a persistent kernel, one 128 x 128 tile of G at a time (upper
//                     triangle only; the lower one is mirrored on store).  A TMA warp
//                     stages 32-wide K chunks of the tile's row panels (hi and lo of both
//                     operands, 128-byte swizzled) into a ring of shared-memory stages; an
//                     MMA warp issues tcgen05.mma kind::tf32 (M = N = 128, K = 8) with the
//                     accumulators in tensor memory: hi*hi + hi*lo + lo*hi per K step, the
//                     split-TF32 product, whose error is about 2^-21 relative per term.  The
//                     tensor core's own FP32 accumulation truncates, so the K chunks go round
//                     robin into four accumulators (all 512 columns of tensor memory), each
//                     summing a quarter of K at a quarter of the magnitude; four epilogue warps
//                     read them (tcgen05.ld), add them in FP32, and store D, c and the
//                     mirrored tile.
//
// The same kernel is the Schur update of the blocked Cholesky factorisation (chol.cu): the
// panel kernel writes the panel's rows below its diagonal tile as TF32 pairs straight into
// the stacked buffers (no transpose), and the epilogue subtracts the Gram matrix of those
// rows from the lower triangle of the trailing tiles, C -= P P^T, while the block's step flag
// says that its factorisation is the blocked one.
//
// All waits are bounded: a wait that runs out raises the launch's error word and the roles
// stop; the kernel then waits (bounded) for its own copies and MMAs and frees its tensor
// memory before it returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gram.h"

namespace subadmm {

__device__ __forceinline__ uint32_t gram_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gram_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void gram_mbar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gram_smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool gram_mbar_test(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(gram_smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for the completion of phase `parity`; false if it did not come within kGramWaitNs or
// the block's abort word was raised meanwhile.
__device__ __forceinline__ bool gram_wait(uint64_t *b, unsigned parity, volatile int *abort_flag)
{
    if (gram_mbar_test(b, parity)) return true;
    const unsigned long long t0 = gram_ns();
    for (;;) {
        for (int k = 0; k < 256; ++k)
            if (gram_mbar_test(b, parity)) return true;
        if (*abort_flag) return false;
        if (gram_ns() - t0 > kGramWaitNs) return false;
    }
}

__device__ __forceinline__ void gram_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gram_smem_u32(b)) : "memory");
}

__device__ __forceinline__ void gram_expect_tx(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(gram_smem_u32(b)), "r"(bytes) : "memory");
}

// 2-D tiled TMA load of a (32 x 128)-element box at (x, y) into 128-byte swizzled shared
// memory; completes `bytes` on the barrier
__device__ __forceinline__ void gram_tma_load(void *dst, const CUtensorMap *map, int x, int y,
                                              uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(gram_smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
                   "r"(gram_smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzled layout:
// rows of 128 bytes, groups of 8 rows 1024 bytes apart (stride byte offset), the leading
// byte offset unused, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t gram_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M = N = 128.
constexpr uint32_t kGramIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(kGramTile >> 3) << 17) |
                                ((uint32_t)(kGramTile >> 4) << 24);

__device__ __forceinline__ void gram_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(a), "l"(b), "r"(kGramIdesc), "r"(acc)
                 : "memory");
}

// arrive on `bar` once every tcgen05 operation this thread issued so far has completed
__device__ __forceinline__ void gram_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(gram_smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void gram_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void gram_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this thread's lane (its tile row)
__device__ __forceinline__ void gram_tmem_ld32(uint32_t taddr, float *v)
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

// ---- W (DOF-major) -> stacked K-major TF32 pairs
// one 32 x 32 tile per block (32 x 8 threads): rows t of the job (columns of W) by DOF p
__global__ void __launch_bounds__(256) gram_prep_kernel(const GramJob *jobs, int njobs,
                                                        const int *tile_prefix, float *hi,
                                                        float *lo, int ldt)
{
    __shared__ float tile[32][33];
    const int b = blockIdx.x;
    int j = 0;
    while (j + 1 < njobs && tile_prefix[j + 1] <= b) ++j;
    const GramJob J = jobs[j];
    const int local = b - tile_prefix[j];
    const int pt = ldt / 32;                      // DOF tiles per row of the buffer
    const int tr = local / pt, tp = local - tr * pt;
    const int t0 = tr * 32, p0 = tp * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // read W[p][t] with lanes along t (coalesced), write rows t with lanes along p
    for (int k = ty; k < 32; k += 8) {
        const int p = p0 + k, t = t0 + tx;
        tile[k][tx] = (p < J.k && t < J.rows) ? J.W[(size_t)p * J.ldw + t] : 0.0f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int t = t0 + k, p = p0 + tx;
        const float x = tile[tx][k];
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        const float xh = __uint_as_float(h);
        const size_t o = (size_t)(J.row_off + t) * ldt + p;
        hi[o] = xh;
        lo[o] = x - xh;
    }
    // zero D's padding columns [m, mpad) of the rows this tile covers (first DOF tile only)
    if (tp == 0 && J.D) {
        const int m = J.rows - 1;
        for (int k = ty; k < 32; k += 8) {
            const int t = t0 + k;
            if (t < m)
                for (int u = m + tx; u < J.mpad; u += 32) J.D[(size_t)t * J.ldd + u] = 0.0f;
        }
    }
}

// tile number -> (job, row block, column block), row block <= column block
__device__ __forceinline__ void gram_tile_of(const GramJob *jobs, int njobs, int tile, int &j,
                                             int &bi, int &bj)
{
    j = 0;
    while (j + 1 < njobs && jobs[j + 1].tile0 <= tile) ++j;
    int l = tile - jobs[j].tile0;
    const int T = (jobs[j].rows + kGramTile - 1) / kGramTile;
    bi = 0;
    while (l >= T - bi) { l -= T - bi; ++bi; }
    bj = bi + l;
}

__device__ __forceinline__ void gram_store(const GramJob &J, int r, int c, float v, bool mirror)
{
    if (J.S) {                                  // Schur update: lower triangle, row c
        if (r < J.rows && c < J.rows) J.S[(size_t)c * J.lds + r] -= v;
        return;
    }
    const int m = J.rows - 1;
    if (J.G) {
        if (r < J.rows && c < J.rows) {
            J.G[(size_t)r * J.ldg + c] = v;
            if (mirror) J.G[(size_t)c * J.ldg + r] = v;
        }
        return;
    }
    if (r < m && c < m && J.D) {
        J.D[(size_t)r * J.ldd + c] = v;
        if (mirror) J.D[(size_t)c * J.ldd + r] = v;
    } else if (c == m && r < m && J.c) {
        J.c[r] = v;
    }
}

__global__ void __launch_bounds__(kGramThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
               const GramJob *jobs, int njobs, int ntiles, int *err)
{
    extern __shared__ unsigned char gram_raw[];
    __shared__ __align__(8) uint64_t full[kGramStages], empty[kGramStages], acc_full, acc_empty,
        mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(gram_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGramStages; ++s) {
            gram_mbar_init(&full[s], 1);
            gram_mbar_init(&empty[s], 1);
        }
        gram_mbar_init(&acc_full, 1);
        gram_mbar_init(&acc_empty, 128);
        gram_mbar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(gram_smem_u32(&tmem_base)), "r"(kGramAcc * kGramTile) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    gram_fence_before();
    __syncthreads();
    gram_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        // ---- TMA producer: the K chunks of every tile of this block, through the ring
        if (lane == 0) {
            unsigned it = 0;
            for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
                int j, bi, bj;
                gram_tile_of(jobs, njobs, tile, j, bi, bj);
                const GramJob &J = jobs[j];
                const int ya = J.row_off + bi * kGramTile, yb = J.row_off + bj * kGramTile;
                const int nk = (J.k + kGramKChunk - 1) / kGramKChunk;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kGramStages;
                    const unsigned ph = (it / kGramStages) & 1u;
                    if (!gram_wait(&empty[s], ph ^ 1u, &abort_flag)) { abort_flag = 1; atomicExch(err, 1); break; }
                    unsigned char *st = smem + (size_t)s * kGramStageBytes;
                    gram_expect_tx(&full[s], kGramStageBytes);
                    const int x = kc * kGramKChunk;
                    gram_tma_load(st, &map_hi, x, ya, &full[s]);
                    gram_tma_load(st + kGramPanelBytes, &map_lo, x, ya, &full[s]);
                    gram_tma_load(st + 2 * kGramPanelBytes, &map_hi, x, yb, &full[s]);
                    gram_tma_load(st + 3 * kGramPanelBytes, &map_lo, x, yb, &full[s]);
                }
            }
            // teardown: every issued stage must have landed before the block exits
            for (unsigned k = 0; k < kGramStages && k < it; ++k) {
                const unsigned i = it - 1 - k;
                volatile int never = 0;
                gram_wait(&full[i % kGramStages], (i / kGramStages) & 1u, &never);
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer: hi*hi + hi*lo + lo*hi over each tile's K, accumulator in TMEM
        if (lane == 0) {
            unsigned it = 0, tph = 0;
            for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, tph ^= 1u) {
                int j, bi, bj;
                gram_tile_of(jobs, njobs, tile, j, bi, bj);
                const int nk = (jobs[j].k + kGramKChunk - 1) / kGramKChunk;
                // the epilogue of the previous tile has read the accumulator
                if (!gram_wait(&acc_empty, tph ^ 1u, &abort_flag)) { abort_flag = 1; atomicExch(err, 1); break; }
                gram_fence_after();
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kGramStages;
                    const unsigned ph = (it / kGramStages) & 1u;
                    if (!gram_wait(&full[s], ph, &abort_flag)) { ok = false; break; }
                    gram_fence_after();
                    const uint32_t st = gram_smem_u32(smem + (size_t)s * kGramStageBytes);
                    const uint64_t ah = gram_desc(st), al = gram_desc(st + kGramPanelBytes);
                    const uint64_t bh = gram_desc(st + 2 * kGramPanelBytes);
                    const uint64_t bl = gram_desc(st + 3 * kGramPanelBytes);
                    const uint32_t acc = tmem + (uint32_t)((kc % kGramAcc) * kGramTile);
#pragma unroll
                    for (int k = 0; k < kGramKChunk / 8; ++k) {
                        const uint64_t dk = (uint64_t)(2 * k);   // 32 bytes of K per step
                        gram_mma(acc, ah + dk, bh + dk, (kc >= kGramAcc || k > 0) ? 1u : 0u);
                        gram_mma(acc, ah + dk, bl + dk, 1u);
                        gram_mma(acc, al + dk, bh + dk, 1u);
                    }
                    gram_commit(&empty[s]);            // the stage is free once these finish
                }
                if (!ok) { abort_flag = 1; atomicExch(err, 1); break; }
                gram_commit(&acc_full);                // the tile's accumulator is complete
            }
            // teardown: a barrier of its own marks every MMA issued so far complete (on
            // acc_full it could complete a second phase right after the last tile's, which
            // an epilogue warp still polling that tile's parity might then never see)
            gram_commit(&mma_done);
        }
    } else {
        // ---- epilogue (warps 0-3): accumulator -> D, c (row r = the thread's TMEM lane)
        unsigned tph = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, tph ^= 1u) {
            int j, bi, bj;
            gram_tile_of(jobs, njobs, tile, j, bi, bj);
            const GramJob &J = jobs[j];
            const bool got = gram_wait(&acc_full, tph, &abort_flag);
            if (!__all_sync(0xffffffffu, got)) { abort_flag = 1; atomicExch(err, 1); break; }
            gram_fence_after();
            // a diagonal tile stores its upper triangle and mirrors it (the MMA forms (i, j)
            // and (j, i) with the split's two correction terms in swapped order, so they may
            // differ in the last bit); an off-diagonal tile is mirrored whole
            const int r = bi * kGramTile + warp * 32 + lane;
            const bool diag = bi == bj;
            const bool live = !J.gate || *(volatile const int *)J.gate == J.gate_val;
            const int nk = (J.k + kGramKChunk - 1) / kGramKChunk;
            const int nacc = nk < kGramAcc ? nk : kGramAcc;      // accumulators written
            for (int cb = 0; cb < kGramTile; cb += 32) {
                float v[32];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
                gram_tmem_ld32(ta, v);
                for (int a = 1; a < nacc; ++a) {
                    float w[32];
                    gram_tmem_ld32(ta + (uint32_t)(a * kGramTile), w);
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] += w[k];
                }
                const int c0 = bj * kGramTile + cb;
                if (c0 >= J.rows || !live) continue;
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (!diag || c0 + k >= r) gram_store(J, r, c0 + k, v[k], c0 + k != r);
            }
            gram_fence_before();
            gram_arrive(&acc_empty);
        }
    }
    // all roles done (or stopped): the MMA issuer's last commit marks every MMA complete
    __syncwarp();
    __syncthreads();
    if (warp == 5 && lane == 0) {
        volatile int never = 0;
        gram_wait(&mma_done, 0u, &never);
    }
    gram_fence_before();
    __syncthreads();
    gram_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"(kGramAcc * kGramTile) : "memory");
}

}  // namespace subadmm
