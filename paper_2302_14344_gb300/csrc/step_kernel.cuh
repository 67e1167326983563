// One time step of subsystem-based ADMM (Algorithm 1) for a batch of independent scenes,
// one thread block per scene, with the whole per-step working set in shared memory.
//
// Per step and scene:
//   assemble   A_i, b_i, J_ci, e (rigid model or generic blocks)           (Eq. sdyn, Sec. II-A)
//   beta_i     Tr(A_i)/Tr(J_ci^T J_ci) or rho                               (Sec. III-D)
//   factor     K_i = A_i + beta_i J_ci^T J_ci = L_i L_i^T                   (Algorithm 1, factorise)
//   map        W_i = L_i^-1 J_ci^T, g_i = L_i^-1 b_i,
//              D_i = W_i^T W_i = J_ci K_i^-1 J_ci^T, c_i = W_i^T g_i = J_ci K_i^-1 b_i
//   iterate    x_i = c_i + D_i (beta_i z_i - u_i)                           (Eq. admm-1i, then x = J v)
//              y_i = beta_i x_i + u_i ; theta                               (Eq. surrogate, residual)
//              lambda_j by type, beta_i z_ij = y_ij + lambda_j              (Eq. admm-2j)
//              u_i = -lambda (the u-step of Eq. admm-3, simplified by Eq. surrogate)
//   recover    v_i = L_i^-T (g_i + W_i (beta_i z_i - u_i)) for the last iterate (Eq. admm-1i)
//   update     rigid state from v-hat                                       (Eq. ddyn)
//
// The v-step is evaluated through the per-step affine map x = c + D w instead of two
// triangular solves and two products with J per iteration: it is the same linear map,
// reassociated, so every iteration is a small dense mat-vec whose rows run in parallel.
// The u-step uses the identity u^{l+1} = y^{l+1} - beta z^{l+1} = -lambda^{l+1} (from
// Eq. admm-3 and Eq. surrogate), so each row keeps one lambda shared by all its sides.
#pragma once
#include "layout.h"
#include "rigid_model.cuh"

namespace subadmm {

__device__ __forceinline__ double nanmax(double a, double b) { return (a != a || a > b) ? a : b; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// per-side-row integer tables kept in shared memory for the whole launch
struct SrTables {
    int *row;    // scene row of the side-row (lambda, e index)
    int *sub;    // scene-local subsystem
    int *drow;   // shared-memory offset of its row of D
    int *coff;   // shared-memory offset of its entry of c
    int *wbase;  // first side-row of its subsystem
    int *mlen;   // side-rows of its subsystem
};

__device__ void scene_tables(const StepParams &P, const SceneDesc &S, double *sm, SrTables &T)
{
    int *ib = reinterpret_cast<int *>(sm + S.o_int);
    T.row = ib;
    T.sub = ib + S.nsr;
    T.drow = ib + 2 * S.nsr;
    T.coff = ib + 3 * S.nsr;
    T.wbase = ib + 4 * S.nsr;
    T.mlen = ib + 5 * S.nsr;
    for (int j = threadIdx.x; j < S.ncon; j += blockDim.x) {
        const ConDesc &c = P.cons[S.con0 + j];
        for (int s = 0; s < c.ns; ++s) {
            const SubDesc &u = P.subs[S.sub0 + c.sub[s]];
            for (int r = 0; r < c.rows; ++r) {
                const int t = c.sr[s] + r;
                const int lr = t - u.sr0;
                T.row[t] = c.row0 + r;
                T.sub[t] = c.sub[s];
                T.drow[t] = u.o_D + lr * u.m;
                T.coff[t] = u.o_c + lr;
                T.wbase[t] = u.sr0;
                T.mlen[t] = u.m;
            }
        }
    }
}

// Parameters k, alpha, mu of a constraint (model kinds derive them from their drive gains)
__device__ __forceinline__ void con_params(const ConDesc &c, const double *pool, double h,
                                           double &k, double &alpha, double &mu)
{
    const double *p = pool + c.par_off;
    k = 0.0; alpha = 0.0; mu = 0.0;
    if (c.src <= SRC_CONTACT) {
        k = p[0]; alpha = p[1]; mu = p[2];
    } else if (c.src == SRC_ANGLE_PD) {
        k = p[18]; alpha = p[19] / p[18] + 0.5 * h;
    } else if (c.src == SRC_PLANE) {
        mu = p[22];
    }
}

// Step (assemble .. factor .. map) for all subsystems of the scene.  Returns via s_status.
__device__ void scene_setup(const StepParams &P, const SceneDesc &S, double *sm, int *s_status)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // zero W and K of rigid subsystems (their rows only fill body columns); generic blocks
    // are copied whole
    for (int i = warp; i < S.nsub; i += SUBADMM_WARPS) {
        const SubDesc &u = P.subs[S.sub0 + i];
        double *W = sm + u.o_W, *K = sm + u.o_L;
        if (u.kind == KIND_RIGID) {
            for (int q = lane; q < u.m * u.n; q += 32) W[q] = 0.0;
            for (int q = lane; q < u.n * u.n; q += 32) K[q] = 0.0;
        } else {
            const double *A = P.pool + u.gen_off;
            for (int q = lane; q < u.n * u.n; q += 32) K[q] = A[q];
            for (int q = lane; q < u.n; q += 32) sm[u.o_b + q] = A[u.n * u.n + q];
        }
    }
    __syncthreads();
    // rigid bodies: diagonal A = (2/h) M and b (lane per body)
    for (int i = warp; i < S.nsub; i += SUBADMM_WARPS) {
        const SubDesc &u = P.subs[S.sub0 + i];
        if (u.kind != KIND_RIGID) continue;
        for (int k = lane; k < u.nb; k += 32) {
            double Ad[6], bb[6];
            body_dynamics(P.bodies + (size_t)(u.body0 + k) * SUBADMM_BODY, P.h, P.g0, P.g1, P.g2,
                          Ad, bb);
            double *K = sm + u.o_L;
            for (int d = 0; d < 6; ++d) {
                const int q = 6 * k + d;
                K[q * u.n + q] = Ad[d];
                sm[u.o_b + q] = bb[d];
            }
        }
    }
    // constraint rows into W (as rows of J_ci) and e (thread per constraint)
    for (int j = tid; j < S.ncon; j += blockDim.x) {
        const ConDesc &c = P.cons[S.con0 + j];
        double *e = sm + S.o_e + c.row0;
        if (c.src <= SRC_CONTACT) {
            const double *p = P.pool + c.par_off + 3;
            for (int r = 0; r < c.rows; ++r) e[r] = p[r];
            const double *J = p + c.rows;
            for (int s = 0; s < c.ns; ++s) {
                const SubDesc &u = P.subs[S.sub0 + c.sub[s]];
                for (int r = 0; r < c.rows; ++r) {
                    double *Wr = sm + u.o_W + (c.sr[s] + r - u.sr0) * u.n;
                    for (int q = 0; q < u.n; ++q) Wr[q] = J[r * u.n + q];
                }
                J += c.rows * u.n;
            }
        } else {
            double Ja[30], Jb[30], ee[5], kk = 0.0, al = 0.0;
            model_rows(c, P.pool + c.par_off, P.bodies, P.h, P.gamma, Ja, Jb, ee, &kk, &al);
            for (int r = 0; r < c.rows; ++r) e[r] = ee[r];
            {
                const SubDesc &u = P.subs[S.sub0 + c.sub[0]];
                for (int r = 0; r < c.rows; ++r) {
                    double *Wr = sm + u.o_W + (c.sr[0] + r - u.sr0) * u.n + 6 * c.ba;
                    for (int q = 0; q < 6; ++q) Wr[q] = Ja[6 * r + q];
                }
            }
            if (c.side_b >= 0) {
                const SubDesc &u = P.subs[S.sub0 + c.sub[c.side_b]];
                for (int r = 0; r < c.rows; ++r) {
                    double *Wr = sm + u.o_W + (c.sr[c.side_b] + r - u.sr0) * u.n + 6 * c.bb;
                    for (int q = 0; q < 6; ++q) Wr[q] = Jb[6 * r + q];
                }
            }
        }
    }
    __syncthreads();
    // per subsystem (one warp each): beta, K += beta J^T J, Cholesky, W, g, D, c
    for (int i = warp; i < S.nsub; i += SUBADMM_WARPS) {
        const SubDesc &u = P.subs[S.sub0 + i];
        const int n = u.n, m = u.m;
        double *W = sm + u.o_W, *K = sm + u.o_L, *D = sm + u.o_D, *b = sm + u.o_b, *cc = sm + u.o_c;
        // beta_i = Tr(A_i) / Tr(J_ci^T J_ci)  (Sec. III-D)
        double trA = 0.0, trJ = 0.0;
        for (int q = lane; q < n; q += 32) trA += K[q * n + q];
        for (int q = lane; q < m * n; q += 32) trJ += W[q] * W[q];
        trA = warp_sum(trA);
        trJ = warp_sum(trJ);
        const double beta = P.beta_fixed ? P.rho : (trJ > 0.0 ? trA / trJ : 1.0);
        if (lane == 0) {
            sm[S.o_beta + i] = beta;
            P.beta[S.sub0 + i] = beta;
        }
        // K_i = A_i + beta_i J_ci^T J_ci (lower triangle)
        for (int t = lane; t < n * n; t += 32) {
            const int p = t / n, q = t - p * n;
            if (q > p) continue;
            double acc = 0.0;
            for (int r = 0; r < m; ++r) acc += W[r * n + p] * W[r * n + q];
            K[t] += beta * acc;
        }
        __syncwarp();
        // right-looking Cholesky, in place (lower triangle)
        bool ok = true;
        for (int k = 0; k < n; ++k) {
            const double d = K[k * n + k];
            if (!(d > 0.0) || !isfinite(d)) { ok = false; break; }
            const double lkk = sqrt(d);
            __syncwarp();
            for (int r = k + lane; r < n; r += 32) K[r * n + k] = (r == k) ? lkk : K[r * n + k] / lkk;
            __syncwarp();
            for (int r = k + 1 + lane; r < n; r += 32) {
                const double lrk = K[r * n + k];
                for (int q = k + 1; q <= r; ++q) K[r * n + q] -= lrk * K[q * n + k];
            }
            __syncwarp();
        }
        if (!ok) {
            if (lane == 0) *s_status = ST_NOTSPD;
            continue;
        }
        // W rows <- L^-1 J rows ; g = L^-1 b (forward substitution, lane per right-hand side)
        for (int t = lane; t <= m; t += 32) {
            double *x = (t < m) ? W + t * n : b;
            for (int p = 0; p < n; ++p) {
                double s = x[p];
                for (int q = 0; q < p; ++q) s -= K[p * n + q] * x[q];
                x[p] = s / K[p * n + p];
            }
        }
        __syncwarp();
        // D = W^T W (as rows of W), c = W^T g
        for (int t = lane; t < m * m + m; t += 32) {
            if (t < m * m) {
                const int r = t / m, s = t - r * m;
                if (s > r) continue;
                double acc = 0.0;
                for (int p = 0; p < n; ++p) acc += W[r * n + p] * W[s * n + p];
                D[r * m + s] = acc;
                D[s * m + r] = acc;
            } else {
                const int r = t - m * m;
                double acc = 0.0;
                for (int p = 0; p < n; ++p) acc += W[r * n + p] * b[p];
                cc[r] = acc;
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(SUBADMM_THREADS) step_kernel(StepParams P)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ double red[2][4][SUBADMM_WARPS];
    __shared__ int s_status;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int sc = blockIdx.x; sc < P.nscenes; sc += gridDim.x) {
        const SceneDesc S = P.scenes[sc];
        SrTables T;
        scene_tables(P, S, sm, T);
        double *X = sm + S.o_x, *Y = sm + S.o_y, *Z = sm + S.o_z, *LAM = sm + S.o_lam;
        double *E = sm + S.o_e, *BETA = sm + S.o_beta;
        double *Wv[2] = {sm + S.o_w0, sm + S.o_w1};
        __syncthreads();

        for (int step = 0; step < P.n_steps; ++step) {
            if (tid == 0) s_status = ST_OK;
            __syncthreads();
            scene_setup(P, S, sm, &s_status);
            const int status0 = s_status;
            if (status0 != ST_OK) {
                // K_i not SPD: report, leave the state untouched (as the step is undefined)
                if (tid == 0) {
                    double *o = P.res + 6 * sc;
                    o[0] = o[1] = o[2] = __longlong_as_double(0x7ff8000000000000LL);
                    o[3] = 0.0; o[4] = 0.0; o[5] = (double)status0;
                }
                __syncthreads();
                continue;
            }
            // initial z, u = -lambda (cold: zeros; warm: the previous step's)
            for (int r = tid; r < S.nrow; r += blockDim.x)
                LAM[r] = P.warm_prev ? P.lam[S.row_g0 + r] : 0.0;
            for (int t = tid; t < S.nsr; t += blockDim.x) {
                const double beta = BETA[T.sub[t]];
                const double z = P.warm_prev ? P.z[S.sr_g0 + t] : 0.0;
                const double l = P.warm_prev ? P.lam[S.row_g0 + T.row[t]] : 0.0;
                Z[t] = z;
                X[t] = 0.0;
                Y[t] = beta * z - l;           // y^0 = beta z^0 + u^0
                Wv[0][t] = beta * z + l;       // w^0 = beta z^0 - u^0
            }
            __syncthreads();

            int par = 0, last_par = 0, iters = 0, conv = 0, status = ST_OK;
            double th = INFINITY, rp = INFINITY, rd = INFINITY, rz = INFINITY;
            for (int l = 0; l < P.max_iters; ++l) {
                // v-step through the affine map, then y and the theta partial
                const double *w = Wv[par];
                double tpart = 0.0;
                for (int t = tid; t < S.nsr; t += blockDim.x) {
                    const double *Dr = sm + T.drow[t];
                    const double *wb = w + T.wbase[t];
                    const int m = T.mlen[t];
                    double acc = sm[T.coff[t]];
                    for (int s = 0; s < m; ++s) acc += Dr[s] * wb[s];
                    const double ynew = BETA[T.sub[t]] * acc - LAM[T.row[t]];
                    const double d = ynew - Y[t];
                    tpart += d * d;
                    Y[t] = ynew;
                    X[t] = acc;
                }
                tpart = warp_sum(tpart);
                if (lane == 0) red[l & 1][0][warp] = tpart;
                __syncthreads();
                th = 0.0;
                for (int q = 0; q < SUBADMM_WARPS; ++q) th += red[l & 1][0][q];
                last_par = par;
                iters = l + 1;
                if (P.stop_theta && l >= 1 && th < P.theta_th) { conv = 1; break; }
                // z-step per constraint (Sec. III-C), u = -lambda, residual partials
                double *wn = Wv[par ^ 1];
                double rpp = 0.0, rzp = 0.0, rdp = 0.0;
                for (int j = tid; j < S.ncon; j += blockDim.x) {
                    const ConDesc &c = P.cons[S.con0 + j];
                    double invb[SUBADMM_MAXS], bet[SUBADMM_MAXS];
                    double s = 0.0;
                    for (int si = 0; si < c.ns; ++si) {
                        bet[si] = BETA[c.sub[si]];
                        invb[si] = 1.0 / bet[si];
                        s += invb[si];
                    }
                    double kk, al, mu;
                    con_params(c, P.pool, P.h, kk, al, mu);
                    double lamv[8];
                    if (c.type == TYPE_CONTACT) {
                        double qv[3];
                        for (int r = 0; r < 3; ++r) {
                            double q = 0.0;
                            for (int si = 0; si < c.ns; ++si) q += Y[c.sr[si] + r] * invb[si];
                            qv[r] = q + E[c.row0 + r];
                        }
                        const double ln = -qv[0] / s, l1 = -qv[1] / s, l2 = -qv[2] / s;
                        if (ln <= 0.0) {
                            lamv[0] = lamv[1] = lamv[2] = 0.0;
                        } else {
                            const double tn = sqrt(l1 * l1 + l2 * l2);
                            const double lim = mu * ln;
                            lamv[0] = ln;
                            if (tn > lim) { const double f = lim / tn; lamv[1] = l1 * f; lamv[2] = l2 * f; }
                            else { lamv[1] = l1; lamv[2] = l2; }
                        }
                    } else {
                        for (int r = 0; r < c.rows; ++r) {
                            double q = 0.0;
                            for (int si = 0; si < c.ns; ++si) q += Y[c.sr[si] + r] * invb[si];
                            const double e = E[c.row0 + r];
                            double lv;
                            if (c.type == TYPE_EQUALITY) lv = -(q + e) / s;
                            else if (c.type == TYPE_HARD) { lv = -(q + e) / s; lv = lv > 0.0 ? lv : 0.0; }
                            else lv = -kk * (e + al * q) / (1.0 + s * al * kk);
                            lamv[r] = lv;
                        }
                    }
                    for (int r = 0; r < c.rows; ++r) LAM[c.row0 + r] = lamv[r];
                    for (int si = 0; si < c.ns; ++si) {
                        for (int r = 0; r < c.rows; ++r) {
                            const int t = c.sr[si] + r;
                            const double zn = (Y[t] + lamv[r]) / bet[si];
                            const double dz = fabs(zn - Z[t]);
                            rzp = nanmax(rzp, dz);
                            rdp = nanmax(rdp, bet[si] * dz);
                            rpp = nanmax(rpp, fabs(X[t] - zn));
                            Z[t] = zn;
                            wn[t] = bet[si] * zn + lamv[r];
                        }
                    }
                }
                rpp = warp_max(rpp);
                rzp = warp_max(rzp);
                rdp = warp_max(rdp);
                if (lane == 0) {
                    red[l & 1][1][warp] = rpp;
                    red[l & 1][2][warp] = rzp;
                    red[l & 1][3][warp] = rdp;
                }
                __syncthreads();
                rp = 0.0; rz = 0.0; rd = 0.0;
                for (int q = 0; q < SUBADMM_WARPS; ++q) {
                    rp = nanmax(rp, red[l & 1][1][q]);
                    rz = nanmax(rz, red[l & 1][2][q]);
                    rd = nanmax(rd, red[l & 1][3][q]);
                }
                par ^= 1;
                if (!isfinite(rp) || !isfinite(th) || !isfinite(rz)) { status = ST_NAN; break; }
                if (!P.stop_theta && P.tol > 0.0 && rp <= P.tol && rz <= P.tol) { conv = 1; break; }
            }

            // v-hat of the last v-step: v = L^-T (g + W w)  (warp per subsystem)
            for (int i = warp; i < S.nsub; i += SUBADMM_WARPS) {
                const SubDesc &u = P.subs[S.sub0 + i];
                const int n = u.n, m = u.m;
                const double *W = sm + u.o_W, *Lf = sm + u.o_L;
                double *g = sm + u.o_b;
                const double *w = Wv[last_par] + u.sr0;
                for (int p = lane; p < n; p += 32) {
                    double acc = g[p];
                    for (int r = 0; r < m; ++r) acc += W[r * n + p] * w[r];
                    g[p] = acc;
                }
                __syncwarp();
                for (int p = n - 1; p >= 0; --p) {
                    const double vp = g[p] / Lf[p * n + p];
                    __syncwarp();
                    if (lane == 0) g[p] = vp;
                    for (int q = lane; q < p; q += 32) g[q] -= Lf[p * n + q] * vp;
                    __syncwarp();
                }
                for (int p = lane; p < n; p += 32) P.vhat[u.v_off + p] = g[p];
            }
            __syncthreads();
            // state update of rigid bodies (Algorithm 1, last line)
            for (int i = warp; i < S.nsub; i += SUBADMM_WARPS) {
                const SubDesc &u = P.subs[S.sub0 + i];
                if (u.kind != KIND_RIGID) continue;
                for (int k = lane; k < u.nb; k += 32)
                    body_update(P.bodies + (size_t)(u.body0 + k) * SUBADMM_BODY, sm + u.o_b + 6 * k, P.h);
            }
            // warm-start state and reports
            for (int r = tid; r < S.nrow; r += blockDim.x) P.lam[S.row_g0 + r] = LAM[r];
            for (int t = tid; t < S.nsr; t += blockDim.x) P.z[S.sr_g0 + t] = Z[t];
            if (tid == 0) {
                double *o = P.res + 6 * sc;
                o[0] = rp; o[1] = rd; o[2] = th; o[3] = (double)iters; o[4] = (double)conv;
                o[5] = (double)status;
                long long *st = P.stats + 4 * sc;
                st[0] += iters;
                if (iters > st[1]) st[1] = iters;
                st[2] += conv ? 0 : 1;
                st[3] += 1;
            }
            __syncthreads();
        }
    }
}

}  // namespace subadmm
