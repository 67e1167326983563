// Blocked Cholesky factorisation of the large blocks' K_i = A_i + beta_i J_i^T J_i
// (Algorithm 1, factorise; Eq. admm-1i), with the Schur updates on the tensor cores.
//
// Right-looking over panels of 128 columns.  For panel kb (columns r0 .. r0 + 127):
//
//   chol_panel_kernel   one block per matrix: the diagonal tile K_kk = L_kk L_kk^T in shared
//                       memory (sub-blocks of 32 columns: a warp factorises the 32 x 32 block,
//                       the threads solve the tile's rows below it and apply the rank-32 update
//                       to the rest of the tile), then every row below the tile that the panel
//                       reaches, L_ik = K_ik L_kk^-T (a thread per row, chunks of 256 rows in
//                       shared memory).  The rows below go back into L and, as TF32 pairs
//                       (hi = x rounded to TF32, lo = x - hi), into the Schur update's operand.
//   gram_tc_kernel      the trailing update K_ij -= L_ik L_jk^T for every tile pair below the
//                       panel (i >= j > kb, both rows reached by the panel): the Gram matrix of
//                       the panel's rows below the tile, subtracted into the lower triangle.
//
// The envelope of K_i (fill stays inside it) decides which tiles take part: a tile of rows
// takes part in panel kb when its first row's envelope starts at or before the panel's last
// column, since the envelope is nondecreasing.  Entries of those tiles left of the envelope
// are zeros and stay zeros (every product that reaches them has a zero factor).
//
// The panel kernel and the Schur update of a matrix whose step flag is not 4 (a stiff block
// factorised in FP64 by the setup, or a failed factorisation) do nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "chol.h"

namespace subadmm {

namespace {

// k -> (a, b) over the lower triangle a >= b >= 0, row by row
__device__ __forceinline__ void chol_tri(int k, int &a, int &b)
{
    int r = (int)((sqrtf(8.0f * (float)k + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > k) --r;
    while ((r + 1) * (r + 2) / 2 <= k) ++r;
    a = r;
    b = k - r * (r + 1) / 2;
}

__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo)
{
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    lo = x - hi;
}

}  // namespace

__global__ void __launch_bounds__(kCholThreads, 1) chol_panel_kernel(const CholPanelJob *jobs)
{
    extern __shared__ __align__(16) float chol_smem[];
    float *const Dg = chol_smem;                         // diagonal tile
    float *const X = Dg + kCholTile * kCholPad;          // a chunk of rows below it
    float *const idg = X + kCholThreads * kCholPad;      // 1 / L_cc
    __shared__ int s_live, s_bad;
    const CholPanelJob J = jobs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_live = *(volatile int *)J.pending == 4;
        s_bad = 0;
    }
    __syncthreads();
    if (!s_live) return;
    const int n = J.n, r0 = J.r0, nb = min(kCholTile, n - r0);
    float *const A = J.L;

    // the diagonal tile's lower triangle (the upper one as zeros)
    for (int k = tid; k < kCholTile * kCholTile; k += kCholThreads) {
        const int i = k / kCholTile, j = k - i * kCholTile;
        float v = 0.0f;
        if (i < nb && j <= i) v = A[(size_t)(r0 + i) * n + r0 + j];
        Dg[i * kCholPad + j] = v;
    }
    __syncthreads();

    // ---- K_kk = L_kk L_kk^T, 32 columns at a time
    for (int c0 = 0; c0 < nb; c0 += 32) {
        const int w = min(32, nb - c0);
        if (warp == 0) {
            // the w x w block at (c0, c0): lane l holds row c0 + l
            float *const B = Dg + c0 * kCholPad + c0;
            for (int c = 0; c < w; ++c) {
                const float d = B[c * kCholPad + c];            // the same for every lane
                if (!(d > 0.0f) || !isfinite(d)) {
                    if (lane == 0) s_bad = 1;
                    break;
                }
                const float s = rsqrtf(d);
                __syncwarp();
                if (lane > c && lane < w) B[lane * kCholPad + c] *= s;
                if (lane == c) {
                    B[c * kCholPad + c] = d * s;
                    idg[c0 + c] = s;
                }
                __syncwarp();
                if (lane > c && lane < w) {
                    const float lc = B[lane * kCholPad + c];
                    for (int q = c + 1; q <= lane; ++q) B[lane * kCholPad + q] -= lc * B[q * kCholPad + c];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_bad) break;
        // rows of the tile below the block: x L_bb^T = a (a thread per row)
        {
            const int i = c0 + w + tid;
            if (i < nb) {
                float *const xr = Dg + i * kCholPad + c0;
                const float *const Lb = Dg + c0 * kCholPad + c0;
                for (int c = 0; c < w; ++c) {
                    float s0 = xr[c], s1 = 0.0f;
                    int q = 0;
                    for (; q + 1 < c; q += 2) {
                        s0 -= xr[q] * Lb[c * kCholPad + q];
                        s1 -= xr[q + 1] * Lb[c * kCholPad + q + 1];
                    }
                    if (q < c) s0 -= xr[q] * Lb[c * kCholPad + q];
                    xr[c] = (s0 + s1) * idg[c0 + c];
                }
            }
        }
        __syncthreads();
        // the rest of the tile: rank-w update of its lower triangle
        {
            const int t0 = c0 + w, m = nb - t0, tri = m * (m + 1) / 2;
            for (int k = tid; k < tri; k += kCholThreads) {
                int a, b;
                chol_tri(k, a, b);
                const float *pa = Dg + (t0 + a) * kCholPad + c0;
                const float *pb = Dg + (t0 + b) * kCholPad + c0;
                float s0 = 0.0f, s1 = 0.0f;
                int c = 0;
                for (; c + 1 < w; c += 2) {
                    s0 += pa[c] * pb[c];
                    s1 += pa[c + 1] * pb[c + 1];
                }
                if (c < w) s0 += pa[c] * pb[c];
                Dg[(t0 + a) * kCholPad + t0 + b] -= s0 + s1;
            }
        }
        __syncthreads();
    }
    if (s_bad) {
        if (tid == 0) {
            *(volatile int *)J.pending = 0;
            if (J.subflag) *(volatile int *)J.subflag = 0;
            atomicExch(J.status, J.fail_status);
        }
        return;
    }

    // ---- rows below the tile: L_ik = K_ik L_kk^-T, a chunk of 256 rows at a time
    for (int base = r0 + nb; base < J.rend; base += kCholThreads) {
        const int rows = min(kCholThreads, J.rend - base);
        for (int k = tid; k < rows * kCholTile; k += kCholThreads) {
            const int t = k / kCholTile, c = k - t * kCholTile;
            X[t * kCholPad + c] = A[(size_t)(base + t) * n + r0 + c];
        }
        __syncthreads();
        if (tid < rows) {
            float *const xr = X + tid * kCholPad;
            for (int c = 0; c < kCholTile; ++c) {
                const float *const Lc = Dg + c * kCholPad;
                float s0 = xr[c], s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
                int q = 0;
                for (; q + 3 < c; q += 4) {
                    s0 -= xr[q] * Lc[q];
                    s1 -= xr[q + 1] * Lc[q + 1];
                    s2 -= xr[q + 2] * Lc[q + 2];
                    s3 -= xr[q + 3] * Lc[q + 3];
                }
                for (; q < c; ++q) s0 -= xr[q] * Lc[q];
                xr[c] = ((s0 + s1) + (s2 + s3)) * idg[c];
            }
        }
        __syncthreads();
        const size_t op = (size_t)(base - r0 - nb) * kCholTile;     // operand row of `base`
        for (int k = tid; k < rows * kCholTile; k += kCholThreads) {
            const int t = k / kCholTile, c = k - t * kCholTile;
            const float x = X[t * kCholPad + c];
            A[(size_t)(base + t) * n + r0 + c] = x;
            if (J.hi) {
                float h, l;
                tf32_split(x, h, l);
                J.hi[op + k] = h;
                J.lo[op + k] = l;
            }
        }
        __syncthreads();
    }

    // ---- the diagonal tile back, 1 / L_pp on the diagonal (read by the solves)
    for (int k = tid; k < nb * kCholTile; k += kCholThreads) {
        const int i = k / kCholTile, j = k - i * kCholTile;
        if (j < i) A[(size_t)(r0 + i) * n + r0 + j] = Dg[i * kCholPad + j];
        else if (j == i) A[(size_t)(r0 + i) * n + r0 + i] = idg[i];
    }
}

cudaError_t chol_plan_build(CholPlan &P, const std::vector<CholMatrix> &mats, int *status,
                            int fail_status)
{
    chol_plan_free(P);
    cudaError_t e = cudaGetDevice(&P.device);
    if (e != cudaSuccess) return e;
    int tmax = 0;
    for (const CholMatrix &m : mats) {
        if (m.n < 1 || (int)m.env.size() != m.n) return cudaErrorInvalidValue;
        tmax = std::max(tmax, (m.n + kCholTile - 1) / kCholTile);
    }
    P.panels.resize(tmax);
    for (int kb = 0; kb < tmax; ++kb) {
        const int r0 = kb * kCholTile;
        std::vector<CholPanelJob> jobs;
        std::vector<GramJob> upd;
        std::vector<int> upd_of;
        for (const CholMatrix &m : mats) {
            if (r0 >= m.n) continue;
            // the last tile of rows that the panel reaches
            int il = kb;
            while ((il + 1) * kCholTile < m.n && m.env[(il + 1) * kCholTile] / kCholTile <= kb) ++il;
            CholPanelJob J{};
            J.L = m.L;
            J.n = m.n;
            J.r0 = r0;
            J.rend = std::min(m.n, (il + 1) * kCholTile);
            J.pending = m.pending;
            J.subflag = m.subflag;
            J.status = status;
            J.fail_status = fail_status;
            const int below = J.rend - std::min(m.n, r0 + kCholTile);
            if (below > 0) {
                GramJob g{};
                g.rows = below;
                g.k = kCholTile;
                g.S = m.L + (size_t)(r0 + kCholTile) * m.n + r0 + kCholTile;
                g.lds = m.n;
                g.gate = m.pending;
                g.gate_val = 4;
                upd.push_back(g);
                upd_of.push_back((int)jobs.size());
            }
            jobs.push_back(J);
        }
        CholPanel &pn = P.panels[kb];
        if (!upd.empty()) {
            if ((e = gram_plan_build(pn.syrk, upd)) != cudaSuccess) return e;
            if (pn.syrk.ldt != kCholTile) return cudaErrorInvalidValue;
            for (size_t q = 0; q < upd.size(); ++q) {
                CholPanelJob &J = jobs[upd_of[q]];
                J.hi = pn.syrk.hi + (size_t)upd[q].row_off * kCholTile;
                J.lo = pn.syrk.lo + (size_t)upd[q].row_off * kCholTile;
            }
        }
        pn.njobs = (int)jobs.size();
        if (pn.njobs == 0) continue;
        if ((e = cudaMalloc((void **)&pn.d_jobs, sizeof(CholPanelJob) * jobs.size())) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(pn.d_jobs, jobs.data(), sizeof(CholPanelJob) * jobs.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute((const void *)chol_panel_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmem);
}

cudaError_t chol_plan_run(const CholPlan &P, cudaStream_t st, int *err)
{
    for (const CholPanel &pn : P.panels) {
        if (pn.njobs == 0) continue;
        chol_panel_kernel<<<pn.njobs, kCholThreads, kCholSmem, st>>>(pn.d_jobs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (pn.syrk.njobs > 0 && (e = gram_plan_run(pn.syrk, st, err)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void chol_plan_free(CholPlan &P)
{
    for (CholPanel &pn : P.panels) {
        cudaFree(pn.d_jobs);
        gram_plan_free(pn.syrk);
    }
    P = CholPlan{};
}

}  // namespace subadmm
