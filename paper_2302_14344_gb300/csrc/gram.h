// Host side of the tensor-core Gram kernel (gram_tc.cuh): a plan holds a batch of Gram jobs
// (one per subsystem), the stacked K-major TF32-pair buffers they are transposed into, the
// two TMA tensor maps over those buffers and the launch geometry.  Internal to libsubadmm.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include <vector>

namespace subadmm {

constexpr int kGramTile = 128;          // M = N of one MMA and one output tile
constexpr int kGramKChunk = 32;         // FP32 elements of K per stage (128 bytes)
constexpr int kGramStages = 3;          // shared-memory ring depth
constexpr int kGramPanelBytes = kGramTile * kGramKChunk * 4;      // 16 KB
constexpr int kGramStageBytes = 4 * kGramPanelBytes;             // A hi, A lo, B hi, B lo
constexpr int kGramSmem = kGramStages * kGramStageBytes + 1024;  // + alignment slack
constexpr int kGramThreads = 192;       // warps 0-3 epilogue, 4 TMA, 5 MMA
constexpr int kGramAcc = 4;             // accumulators in tensor memory (K chunk kc adds into
                                        // accumulator kc % 4; the epilogue sums them)
constexpr unsigned long long kGramWaitNs = 1000000000ull;       // 1 s per wait

// One Gram matrix of the batch.
struct GramJob {
    const float *W;   // W[p * ldw + t], p < k (DOF), t < rows (= m + 1 columns, last = g)
    int ldw;
    int rows;         // m + 1
    int k;            // n
    int row_off;      // first row of this job in the stacked buffer (a multiple of 128)
    int tile0;        // first upper-triangle tile of this job in the launch's numbering
    float *D;         // G[t][u] for t, u < m at D[t * ldd + u] (null: not stored)
    int ldd;
    int mpad;         // D rows are zero-padded from m to mpad
    float *c;         // G[t][m] for t < m at c[t] (null: not stored)
    float *G;         // the whole (m + 1) x (m + 1) matrix at G[t * ldg + u] (null: not stored)
    int ldg;
    // Schur-update form (the blocked Cholesky's trailing update): S[u * lds + t] -= G[t][u]
    // for t <= u, the lower triangle of a row-major matrix (null: not this form).  The operand
    // rows are written into the plan's buffers by their producer (W is null: no transpose).
    float *S;
    int lds;
    const int *gate;  // stores happen only while *gate == gate_val (null: always)
    int gate_val;
};


struct GramPlan {
    int device = -1;
    int njobs = 0;
    int ntiles = 0;            // upper-triangle 128 x 128 output tiles of the batch
    int prep_blocks = 0;       // 32 x 32 transpose tiles of the batch
    int ldt = 0;               // row length of the stacked buffers (a multiple of 32)
    int rows_total = 0;        // rows of the stacked buffers (each job padded to 128)
    int grid = 0;              // blocks of the Gram launch
    bool prep = true;          // W given: the transpose kernel fills the buffers (else their
                               // producer writes them; padding rows stay zero)
    float *hi = nullptr, *lo = nullptr;
    GramJob *d_jobs = nullptr;
    int *d_prep_prefix = nullptr;
    int *d_err = nullptr;      // raised by a wait that ran out
    CUtensorMap map_hi{}, map_lo{};
};

// Lays out the jobs (W, ldw, rows, k and the outputs of each must be set; row_off and tile0
// are filled in), allocates the buffers and encodes the tensor maps on the current device.
// Either every job has its W or none (the Schur-update form: the buffers start zeroed and
// job j's operand row t goes to row row_off + t of hi and lo).  Returns cudaSuccess or the
// first error.
cudaError_t gram_plan_build(GramPlan &P, std::vector<GramJob> &jobs);

// Enqueues the transpose and the Gram kernel on `st`; a wait that runs out raises *err
// (the plan's own error word when err is null).
cudaError_t gram_plan_run(const GramPlan &P, cudaStream_t st, int *err = nullptr);

// Reads (and clears) the plan's error word: 1 if a wait of the last runs ran out.
cudaError_t gram_plan_error(const GramPlan &P, int *out);

void gram_plan_free(GramPlan &P);

}  // namespace subadmm
