// Host side of the tensor-core Gram kernel, and its standalone C-ABI entry point.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "subadmm.h"
#include "gram_tc.cuh"
#include "tmap.h"
#include "device_guard.h"

namespace subadmm {

namespace {

// a 2-D FP32 tensor of `rows` rows of `ld` elements, boxes of 32 x 128, 128-byte swizzle
cudaError_t encode(CUtensorMap *map, float *base, int ld, int rows)
{
    return tmap_encode_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), base, ld, rows,
                          kGramKChunk, kGramTile);
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

}  // namespace

cudaError_t gram_plan_build(GramPlan &P, std::vector<GramJob> &jobs)
{
    gram_plan_free(P);
    cudaError_t e = cudaGetDevice(&P.device);
    if (e != cudaSuccess) return e;
    P.njobs = (int)jobs.size();
    if (P.njobs == 0) return cudaSuccess;
    int maxk = 1, rows = 0, tiles = 0;
    for (const GramJob &J : jobs) maxk = std::max(maxk, J.k);
    P.prep = jobs[0].W != nullptr;
    for (const GramJob &J : jobs)
        if ((J.W != nullptr) != P.prep) return cudaErrorInvalidValue;
    P.ldt = round_up(maxk, kGramKChunk);
    std::vector<int> prefix;
    int prep = 0;
    for (GramJob &J : jobs) {
        if (J.rows < 1 || J.k < 1) return cudaErrorInvalidValue;
        const int T = (J.rows + kGramTile - 1) / kGramTile;
        J.row_off = rows;
        J.tile0 = tiles;
        rows += T * kGramTile;
        tiles += T * (T + 1) / 2;
        prefix.push_back(prep);
        prep += (T * kGramTile / 32) * (P.ldt / 32);
    }
    P.rows_total = rows;
    P.ntiles = tiles;
    P.prep_blocks = prep;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P.device);
    if (e != cudaSuccess) return e;
    P.grid = std::max(1, std::min(tiles, sms));
    const size_t bytes = sizeof(float) * (size_t)rows * P.ldt;
    if ((e = cudaMalloc((void **)&P.hi, bytes)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&P.lo, bytes)) != cudaSuccess) return e;
    if (!P.prep) {
        if ((e = cudaMemset(P.hi, 0, bytes)) != cudaSuccess) return e;
        if ((e = cudaMemset(P.lo, 0, bytes)) != cudaSuccess) return e;
    }
    if ((e = cudaMalloc((void **)&P.d_jobs, sizeof(GramJob) * jobs.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&P.d_prep_prefix, sizeof(int) * prefix.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&P.d_err, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemset(P.d_err, 0, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(P.d_jobs, jobs.data(), sizeof(GramJob) * jobs.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(P.d_prep_prefix, prefix.data(), sizeof(int) * prefix.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = encode(&P.map_hi, P.hi, P.ldt, rows)) != cudaSuccess) return e;
    if ((e = encode(&P.map_lo, P.lo, P.ldt, rows)) != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)gram_tc_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kGramSmem);
}

cudaError_t gram_plan_run(const GramPlan &P, cudaStream_t st, int *err)
{
    if (P.njobs == 0) return cudaSuccess;
    if (P.prep) {
        gram_prep_kernel<<<P.prep_blocks, 256, 0, st>>>(P.d_jobs, P.njobs, P.d_prep_prefix,
                                                        P.hi, P.lo, P.ldt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    gram_tc_kernel<<<P.grid, kGramThreads, kGramSmem, st>>>(P.map_hi, P.map_lo, P.d_jobs,
                                                            P.njobs, P.ntiles,
                                                            err ? err : P.d_err);
    return cudaGetLastError();
}

cudaError_t gram_plan_error(const GramPlan &P, int *out)
{
    *out = 0;
    if (!P.d_err) return cudaSuccess;
    cudaError_t e = cudaMemcpy(out, P.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(P.d_err, 0, sizeof(int));
    return e;
}

void gram_plan_free(GramPlan &P)
{
    cudaFree(P.hi); cudaFree(P.lo); cudaFree(P.d_jobs); cudaFree(P.d_prep_prefix);
    cudaFree(P.d_err);
    P = GramPlan{};
}

}  // namespace subadmm

extern "C" int sim_gram_tc(int device, int njobs, const float *const *W, const int *n,
                           const int *cols, const int *ldw, float *const *G, const int *ldg,
                           int reps, float *ms_per_run)
{
    using namespace subadmm;
    if (njobs < 1 || !W || !n || !cols || !ldw || !G || !ldg || reps < 1) return SIM_EINVAL;
    std::vector<GramJob> jobs(njobs);
    for (int j = 0; j < njobs; ++j) {
        if (!W[j] || !G[j] || n[j] < 1 || cols[j] < 1 || ldw[j] < cols[j] || ldg[j] < cols[j])
            return SIM_EINVAL;
        GramJob &J = jobs[j];
        J = GramJob{};
        J.W = W[j];
        J.ldw = ldw[j];
        J.rows = cols[j];
        J.k = n[j];
        J.G = G[j];
        J.ldg = ldg[j];
    }
    DeviceGuard on_device(device);
    if (on_device.err != cudaSuccess) return SIM_ECUDA;
    GramPlan P;
    cudaError_t e = gram_plan_build(P, jobs);
    if (e == cudaErrorMemoryAllocation) { gram_plan_free(P); return SIM_ENOMEM; }
    if (e != cudaSuccess) { gram_plan_free(P); return SIM_ECUDA; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    e = gram_plan_run(P, 0);                    // first run (not timed)
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    for (int r = 1; r < reps && e == cudaSuccess; ++r) e = gram_plan_run(P, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess && reps > 1) e = cudaEventElapsedTime(&ms, e0, e1);
    int err = 0;
    if (e == cudaSuccess) e = gram_plan_error(P, &err);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gram_plan_free(P);
    if (e != cudaSuccess) return SIM_ECUDA;
    if (ms_per_run) *ms_per_run = reps > 1 ? ms / (reps - 1) : 0.0f;
    return err ? SIM_ETIMEOUT : SIM_OK;
}
