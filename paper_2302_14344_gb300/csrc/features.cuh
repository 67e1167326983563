// Per-interface inputs and targets of the warm-start network, and its initial duals.
//
// Features (32 per interface, in public interface order), from the state at the start of a
// step: [0:4] projection type one-hot (equality, hard, soft, contact); [4:7] anchor point of
// side a minus that of side b (world); [7:11] relative orientation q_a^-1 q_b (w, x, y, z;
// identity for nodes and the world); [11:14] anchor velocity of a minus that of b; [14:17]
// angular velocity of a minus that of b (world); [17:23] the previous step's lambda (first 6
// rows); [23:26] the constraint's error terms e (first 3 rows); [26] mu; [27] s = sum 1/beta
// of its sides (previous step's beta); [28] contact gap; [29] beta_a / beta_b (1 for one
// side); [30:32] zero.
#pragma once

#include "rigid_model.cuh"

namespace subadmm {

constexpr int kFeatures = 32;
constexpr int kDualOut = 7;       // network outputs: 6 dual corrections, log2 beta scale
constexpr int kDualRows = 6;

__device__ __forceinline__ void quat_conj_mul(const double *a, const double *b, double *o)
{
    // conj(a) (x) b, quaternions (w, x, y, z)
    const double aw = a[0], ax = -a[1], ay = -a[2], az = -a[3];
    o[0] = aw * b[0] - ax * b[1] - ay * b[2] - az * b[3];
    o[1] = aw * b[1] + ax * b[0] + ay * b[3] - az * b[2];
    o[2] = aw * b[2] - ax * b[3] + ay * b[0] + az * b[1];
    o[3] = aw * b[3] + ax * b[2] - ay * b[1] + az * b[0];
}

// point, velocity of the point and angular velocity (world) of one side of a model
// constraint: a body record (p at 4, q at 7, v at 11, body-frame w at 14), a node record
// (x, v), or the world (anc is then a world point at rest)
__device__ __forceinline__ void side_motion(int kind, const double *rec, const double *anc,
                                           double *P, double *Vp, double *W, double *q)
{
    for (int d = 0; d < 3; ++d) { Vp[d] = 0.0; W[d] = 0.0; }
    q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
    if (kind == 0) {                           // world
        for (int d = 0; d < 3; ++d) P[d] = anc[d];
        return;
    }
    if (kind == 1) {                           // node
        for (int d = 0; d < 3; ++d) { P[d] = rec[d]; Vp[d] = rec[3 + d]; }
        return;
    }
    const Rot R = quat_rot(rec + 7);
    double r[3], wr[3], wxa[3];
    mul(R, anc, r);
    for (int d = 0; d < 3; ++d) P[d] = rec[4 + d] + r[d];
    cross(rec + 14, anc, wxa);                 // w x anc in the body frame
    mul(R, wxa, wr);
    mul(R, rec + 14, W);
    for (int d = 0; d < 3; ++d) Vp[d] = rec[11 + d] + wr[d];
    for (int k = 0; k < 4; ++k) q[k] = rec[7 + k];
}

__global__ void interface_features_kernel(const StepParams P, const int *pub2dev,
                                          const int *con_scene, int nif, float *X)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nif; i += gridDim.x * blockDim.x) {
        float f[kFeatures];
        for (int k = 0; k < kFeatures; ++k) f[k] = 0.0f;
        const int j = pub2dev[i];
        const ConDesc c = P.cons[j];
        const SceneDesc &S = P.scenes[con_scene[j]];
        f[c.type] = 1.0f;
        const int rg = S.row_g0 + c.row0;
        for (int r = 0; r < c.rows && r < kDualRows; ++r) f[17 + r] = (float)P.lam[rg + r];
        // beta of the last step (zero before the first step: then s = 0 and the ratio 1)
        double s = 0.0;
        for (int q = 0; q < c.ns; ++q) {
            const double b = P.beta[S.sub0 + c.sub[q]];
            s += b > 0.0 ? 1.0 / b : 0.0;
        }
        f[27] = (float)s;
        // the sizes the best beta depends on (the rho search prefers larger scales for large
        // scenes): the scene's side-rows and the DOF of side a's subsystem, as log2(1 + x)
        f[30] = log2f(1.0f + (float)S.nsr);
        f[31] = log2f(1.0f + (float)P.subs[S.sub0 + c.sub[0]].n);
        const double b0 = P.beta[S.sub0 + c.sub[0]], b1 = c.ns >= 2 ? P.beta[S.sub0 + c.sub[1]] : 0.0;
        f[29] = (b0 > 0.0 && b1 > 0.0) ? (float)(b0 / b1) : 1.0f;
        const double *prm = P.pool + c.par_off;
        if (c.src <= SRC_CONTACT) {
            for (int r = 0; r < c.rows && r < 3; ++r) f[23 + r] = (float)prm[3 + r];
            f[26] = (float)prm[2];
        } else {
            double Ja[30], Jb[30], ee[5], kk = 0.0, al = 0.0;
            model_rows(c, prm, P.bodies, P.nodes, P.h, P.gamma, Ja, Jb, ee, &kk, &al);
            for (int r = 0; r < c.rows && r < 3; ++r) f[23 + r] = (float)ee[r];
            const double *ra = c.node_a ? P.nodes + (size_t)c.gb_a * SUBADMM_NODE
                                        : P.bodies + (size_t)c.gb_a * SUBADMM_BODY;
            double pa[3], va[3], wa[3], qa[4], pb[3], vb[3], wb[3], qb[4], qr[4];
            side_motion(c.node_a ? 1 : 2, ra, prm + 0, pa, va, wa, qa);
            if (c.gb_b >= 0) {
                const double *rb = c.node_b ? P.nodes + (size_t)c.gb_b * SUBADMM_NODE
                                            : P.bodies + (size_t)c.gb_b * SUBADMM_BODY;
                side_motion(c.node_b ? 1 : 2, rb, prm + 3, pb, vb, wb, qb);
            } else {
                side_motion(0, nullptr, prm + 3, pb, vb, wb, qb);
            }
            if (c.src == SRC_PLANE) {
                // b is the foot of a's centre on the plane n . x = plane_z
                const double *n = prm + 9;
                const double off = n[0] * pa[0] + n[1] * pa[1] + n[2] * pa[2] - prm[21];
                for (int d = 0; d < 3; ++d) pb[d] = pa[d] - off * n[d];
                f[26] = (float)prm[22];
                f[28] = (float)(off - prm[12]);
            } else if (c.src == SRC_SPHERE) {
                const double d[3] = {pa[0] - pb[0], pa[1] - pb[1], pa[2] - pb[2]};
                f[26] = (float)prm[22];
                f[28] = (float)(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - prm[12] - prm[15]);
            }
            quat_conj_mul(qa, qb, qr);
            for (int d = 0; d < 3; ++d) {
                f[4 + d] = (float)(pa[d] - pb[d]);
                f[11 + d] = (float)(va[d] - vb[d]);
                f[14 + d] = (float)(wa[d] - wb[d]);
            }
            for (int k = 0; k < 4; ++k) f[7 + k] = (float)qr[k];
        }
        for (int k = 0; k < kFeatures; ++k) X[(size_t)i * kFeatures + k] = isfinite(f[k]) ? f[k] : 0.0f;
    }
}

// training targets after a step: t = lambda* - lambda_prev (the previous lambda read back from
// the features taken before the step), mask 1 on the interface's rows (first 6), 0 elsewhere;
// column 6 (log2 beta scale) 0 with mask 1
__global__ void interface_targets_kernel(const StepParams P, const int *pub2dev,
                                         const int *con_scene, int nif, const float *X,
                                         float *T, float *M)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nif; i += gridDim.x * blockDim.x) {
        const int j = pub2dev[i];
        const ConDesc &c = P.cons[j];
        const int rg = P.scenes[con_scene[j]].row_g0 + c.row0;
        for (int r = 0; r < kDualRows; ++r) {
            const bool on = r < c.rows;
            T[(size_t)i * kDualOut + r] = on ? (float)(P.lam[rg + r] - (double)X[(size_t)i * kFeatures + 17 + r]) : 0.0f;
            M[(size_t)i * kDualOut + r] = on ? 1.0f : 0.0f;
        }
        // the seventh output, log2 of the beta scale: 0 (the trace rule) unless the caller
        // writes the best scale a search found
        T[(size_t)i * kDualOut + kDualRows] = 0.0f;
        M[(size_t)i * kDualOut + kDualRows] = 1.0f;
    }
}

// learned initial duals: lambda0 = lambda_prev + the network's correction on the first 6
// rows of each interface; other rows keep lambda_prev
__global__ void learned_duals_kernel(const StepParams P, const int *pub2dev, const int *con_scene,
                                     int nif, const float *Y, double *lam0)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nif; i += gridDim.x * blockDim.x) {
        const int j = pub2dev[i];
        const ConDesc &c = P.cons[j];
        const int rg = P.scenes[con_scene[j]].row_g0 + c.row0;
        for (int r = 0; r < c.rows; ++r)
            lam0[rg + r] = P.lam[rg + r] + (r < kDualRows ? (double)Y[(size_t)i * kDualOut + r] : 0.0);
    }
}

// learned beta scale, accumulation: every interface adds the network's seventh output (log2
// of the scale it proposes) to its scene's sum; acc holds nscenes sums, then nscenes counts,
// zeroed before
__global__ void learned_beta_accumulate_kernel(const int *con_scene, int nif, const int *pub2dev,
                                               const float *Y, float *acc, int nscenes)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nif; i += gridDim.x * blockDim.x) {
        const int sc = con_scene[pub2dev[i]];
        const float y = Y[(size_t)i * kDualOut + kDualRows];
        atomicAdd(&acc[sc], isfinite(y) ? y : 0.0f);
        atomicAdd(&acc[nscenes + sc], 1.0f);
    }
}

// learned beta scale of every subsystem of a scene: 2^k with k the mean proposal of the
// scene's interfaces rounded to an integer in [-3, 3] (whole powers of two, so a kept factor
// is refactorised only when the proposal moves by a whole step; one scale per scene, as the
// rho search that labels the training data picks one per scene); 1 without interfaces
__global__ void learned_beta_scale_kernel(const SceneDesc *scenes, const float *acc, int nscenes,
                                          double *scale)
{
    for (int sc = blockIdx.x * blockDim.x + threadIdx.x; sc < nscenes; sc += gridDim.x * blockDim.x) {
        const float n = acc[nscenes + sc];
        float k = n > 0.0f ? rintf(acc[sc] / n) : 0.0f;
        k = fminf(3.0f, fmaxf(-3.0f, k));
        const double s = exp2((double)k);
        for (int i = 0; i < scenes[sc].nsub; ++i) scale[scenes[sc].sub0 + i] = s;
    }
}

}  // namespace subadmm
