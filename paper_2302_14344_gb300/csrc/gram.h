// Host side of the tensor-core Gram kernel (gram_tc.cuh): a plan holds a batch of Gram jobs
// (one per subsystem), the stacked K-major TF32-pair buffers they are transposed into, the
// two TMA tensor maps over those buffers and the launch geometry.  Internal to libsubadmm.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "gram_tc.cuh"

namespace subadmm {

struct GramPlan {
    int device = -1;
    int njobs = 0;
    int ntiles = 0;            // upper-triangle 128 x 128 output tiles of the batch
    int prep_blocks = 0;       // 32 x 32 transpose tiles of the batch
    int ldt = 0;               // row length of the stacked buffers (a multiple of 32)
    int rows_total = 0;        // rows of the stacked buffers (each job padded to 128)
    int grid = 0;              // blocks of the Gram launch
    float *hi = nullptr, *lo = nullptr;
    GramJob *d_jobs = nullptr;
    int *d_prep_prefix = nullptr;
    int *d_err = nullptr;      // raised by a wait that ran out
    CUtensorMap map_hi{}, map_lo{};
};

// Lays out the jobs (W, ldw, rows, k and the outputs of each must be set; row_off and tile0
// are filled in), allocates the buffers and encodes the tensor maps on the current device.
// Returns cudaSuccess or the first error.
cudaError_t gram_plan_build(GramPlan &P, std::vector<GramJob> jobs);

// Enqueues the transpose and the Gram kernel on `st`.
cudaError_t gram_plan_run(const GramPlan &P, cudaStream_t st);

// Reads (and clears) the plan's error word: 1 if a wait of the last runs ran out.
cudaError_t gram_plan_error(const GramPlan &P, int *out);

void gram_plan_free(GramPlan &P);

}  // namespace subadmm
