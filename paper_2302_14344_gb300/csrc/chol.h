// Host side of the blocked Cholesky factorisation with tensor-core Schur updates (chol.cu):
// per 128-wide panel, one launch of the panel kernel (the diagonal tile's factor and the
// rows below it, on the CUDA cores) and one of the Gram kernel in its Schur-update form
// (C -= P P^T over the trailing tiles the panel reaches, tcgen05 split-TF32).  Internal to
// libsubadmm.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "gram.h"

namespace subadmm {

constexpr int kCholTile = kGramTile;        // panel width = the Gram kernel's tile
constexpr int kCholThreads = 256;           // threads of the panel kernel (a row each)
constexpr int kCholPad = kCholTile + 1;     // shared-memory row stride (floats)
// the diagonal tile, one chunk of rows below it, and 1 / L_cc
constexpr int kCholSmem = (kCholTile + kCholThreads) * kCholPad * 4 + kCholTile * 4;

// One panel of one matrix.
struct CholPanelJob {
    float *L;          // row-major n x n: the lower triangle holds K (with the updates of the
                       // earlier panels) on entry; this panel's columns of the factor on exit
                       // (L_pq below the diagonal, 1 / L_pp on it)
    int n;
    int r0;            // first row and column of the panel
    int rend;          // the panel's rows end here (the last row any of its columns reaches,
                       // rounded up to a whole tile)
    int *pending;      // the matrix's step flag: the panel is factorised only while it is 4
    int *subflag;      // kept-factor flag, cleared on failure (null: none)
    int *status;       // set to the failure status on a non-positive pivot
    int fail_status;
    float *hi, *lo;    // rows r0 + 128 .. rend of the panel as TF32 pairs, 128 per row (the
                       // Schur update's operand); null when no row lies below the tile
};

// A matrix to factorise: its storage, its envelope and its flags.
struct CholMatrix {
    float *L;
    int n;
    std::vector<int> env;   // first column of row p inside the envelope, nondecreasing in p;
                            // the lower triangle holds zeros left of env[p] from the first
                            // column of the envelope's tile of row p's tile row on
    int *pending;
    int *subflag;
};

struct CholPanel {
    int njobs = 0;
    CholPanelJob *d_jobs = nullptr;
    GramPlan syrk;          // the panel's Schur update (no jobs: none)
};

struct CholPlan {
    int device = -1;
    std::vector<CholPanel> panels;
};

// Lays out the panels of every matrix (a tile of rows takes part in panel kb if its first row's
// envelope starts inside panel kb's columns or before), allocates the Schur-update operands and
// uploads the jobs, on the current device.
cudaError_t chol_plan_build(CholPlan &P, const std::vector<CholMatrix> &mats, int *status,
                            int fail_status);

// Enqueues every panel's kernel and Schur update on `st`; a wait of the Gram kernel that runs
// out raises *err.
cudaError_t chol_plan_run(const CholPlan &P, cudaStream_t st, int *err);

void chol_plan_free(CholPlan &P);

}  // namespace subadmm
