// One time step of subsystem-based ADMM (Algorithm 1) for a batch of independent scenes,
// one thread block per scene, with the whole per-step working set in shared memory.
//
// Per step and scene:
//   assemble   A_i, b_i, J_ci, e (rigid model or generic blocks)           (Eq. sdyn, Sec. II-A)
//   beta_i     Tr(A_i)/Tr(J_ci^T J_ci) or rho                               (Sec. III-D)
//   factor     K_i = A_i + beta_i J_ci^T J_ci = L_i L_i^T in FP64          (Algorithm 1, factorise)
//   map        W_i = L_i^-1 J_ci^T, g_i = L_i^-1 b_i,
//              D_i = W_i^T W_i = J_ci K_i^-1 J_ci^T, c_i = W_i^T g_i = J_ci K_i^-1 b_i
//   iterate    x_i = c_i + D_i (beta_i z_i - u_i)                           (Eq. admm-1i, x = J v)
//              y_i = beta_i x_i + u_i                                       (Eq. surrogate)
//              lambda_j by type, beta_i z_ij = y_ij + lambda_j              (Eq. admm-2j)
//              u_i = -lambda (the u-step of Eq. admm-3, simplified by Eq. surrogate)
//   recover    v_i = K_i^-1 (b_i + J_ci^T (beta_i z_i - u_i)) in FP64 for the last v-step
//   update     rigid state from v-hat                                       (Eq. ddyn)
//
// The v-step is evaluated through the per-step affine map x = c + D w instead of two
// triangular solves and two products with J per iteration: it is the same linear map,
// reassociated, so every iteration is a small dense mat-vec whose rows run in parallel.
// The u-step uses u^{l+1} = y^{l+1} - beta z^{l+1} = -lambda^{l+1} (Eq. admm-3 with
// Eq. surrogate), so each row keeps one lambda shared by its sides and w = y + 2 lambda.
//
// T is the iteration type.  T = double: the map and the iterations in FP64.  T = float (the
// mixed form): assembly stays FP64; K and its Cholesky factor are FP32 for well-conditioned
// blocks and FP64 for stiff or high-mass-ratio ones (spread of diag K above 1e3); W, g, D,
// c are formed in FP32 and the iterations run in FP32.  (In a grid scene, the FP32 factor of
// a refactorised block of >= 128 DOF is left to the blocked factorisation with tensor-core
// Schur updates that runs between the grid kernel's launches.)  When the FP32 stop test
// passes, v-hat is recovered in FP64 and the primal residual re-evaluated as
// max |J v-hat - z| in FP64; if that misses the tolerance, c is corrected by the FP64 - FP32
// difference of x at the current iterate (iterative refinement) and the iterations resume.
//
// On GB300 an FP64 warp instruction costs about 64 issue cycles of a sub-partition however
// few lanes are active, so FP64 work is kept out of the loop of the mixed form and the loop
// keeps each thread's coefficients, y and z in registers for the whole step.
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

// 16-byte vectors of the iteration type and residual bit patterns.  Residuals are
// non-negative, so their IEEE bit patterns order like their values and a NaN (sign bit
// cleared by fabs) orders above +inf: maxima reduce on the integer pipe.
template <typename T> struct VecOf;
template <> struct VecOf<float> { using V = float4; using U = unsigned; static constexpr int N = 4; };
template <> struct VecOf<double> { using V = double2; using U = unsigned long long; static constexpr int N = 2; };

__device__ __forceinline__ float vdot(const float4 a, const float4 b, float acc)
{
    acc = fmaf(a.x, b.x, acc); acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc); acc = fmaf(a.w, b.w, acc);
    return acc;
}
__device__ __forceinline__ double vdot(const double2 a, const double2 b, double acc)
{
    acc = fma(a.x, b.x, acc); acc = fma(a.y, b.y, acc);
    return acc;
}
__device__ __forceinline__ unsigned rbits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long rbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned umax(unsigned a, unsigned b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned warp_umax(unsigned v) { return __reduce_max_sync(0xffffffffu, v); }
__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v)
{
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}
__device__ __forceinline__ unsigned tol_bits(float, double tol) { return __float_as_uint(__double2float_rd(tol)); }
__device__ __forceinline__ unsigned long long tol_bits(double, double tol) { return rbits(tol); }
__device__ __forceinline__ unsigned inf_bits(float) { return 0x7f800000u; }
__device__ __forceinline__ unsigned long long inf_bits(double) { return 0x7ff0000000000000ull; }
// D chunks (16-byte vectors) a lane keeps in registers in the cached iteration
template <typename T> struct CachedChunks;
template <> struct CachedChunks<float> { static constexpr int value = 4; };
template <> struct CachedChunks<double> { static constexpr int value = 6; };
template <typename T> struct VecZero;
template <> struct VecZero<float> { __device__ static float4 get() { return make_float4(0.f, 0.f, 0.f, 0.f); } };
template <> struct VecZero<double> { __device__ static double2 get() { return make_double2(0.0, 0.0); } };
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// Sum (a) and maxima (b, c) of three per-thread doubles over the block.
__device__ __forceinline__ void block_reduce3(double (*red)[SUBADMM_MAXWARPS], double &a,
                                              double &b, double &c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a); b = warp_max(b); c = warp_max(c);
    __syncthreads();
    if (lane == 0) { red[0][warp] = a; red[1][warp] = b; red[2][warp] = c; }
    __syncthreads();
    a = 0.0; b = 0.0; c = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        a += red[0][q]; b = nanmax(b, red[1][q]); c = nanmax(c, red[2][q]);
    }
    __syncthreads();
}

// Phase tracer: thread 0 of a scene's block accumulates clock64 deltas per phase in
// registers and adds them to P.phase once per step (flush), so tracing stays off the
// critical path of the iterations.
struct PhaseClock {
    long long *out;
    long long t;
    long long a[8];
    __device__ __forceinline__ PhaseClock(long long *o) : out(threadIdx.x == 0 ? o : nullptr), t(0)
    {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = 0;
        if (out) t = clock64();
    }
    __device__ __forceinline__ void mark(int phase)
    {
        if (out) {
            const long long n = clock64();
            a[phase] += n - t;
            t = n;
        }
    }
    // attribute the time up to `when` (a clock64 value) to `phase`
    __device__ __forceinline__ void mark_at(int phase, long long when)
    {
        if (out) {
            a[phase] += when - t;
            t = when;
        }
    }
    __device__ __forceinline__ void flush(int iters, int steps = 1)
    {
        if (out) {
            a[PHASE_ITERS] = iters;
            a[PHASE_STEPS] = steps;
#pragma unroll
            for (int q = 0; q < 8; ++q) out[q] += a[q];
        }
    }
};

// shared-memory views of one scene
template <typename T>
struct View {
    double *db;          // double region (shared memory): scene arrays
    T *tb;               // T region (shared memory): scene arrays
    double *sdb;         // per-subsystem double arrays: shared memory, or global for a
    T *stb;              // scene too large to hold them on chip; likewise for T
    T *htb;              // per-subsystem iteration arrays (D, c): shared memory unless the
                         // scene cannot hold even those
    int *row, *sub, *drow, *coff, *wbase, *mlen;   // per side-row tables
    Item *item;
    int *list;
};

template <typename T>
__device__ View<T> scene_view(const StepParams &P, const SceneDesc &S, unsigned char *raw)
{
    View<T> V;
    V.db = reinterpret_cast<double *>(raw);
    V.tb = reinterpret_cast<T *>(raw + S.t_base);
    if (S.sub_global) {
        unsigned char *w = reinterpret_cast<unsigned char *>(P.work) + S.g_base;
        V.sdb = reinterpret_cast<double *>(w);
        V.stb = reinterpret_cast<T *>(w + S.g_tbase);
    } else {
        V.sdb = V.db;
        V.stb = V.tb;
    }
    V.htb = S.hot_global ? V.stb : V.tb;
    int *ib = reinterpret_cast<int *>(raw + S.i_base);
    V.row = ib;
    V.sub = ib + S.nsr;
    V.drow = ib + 2 * S.nsr;
    V.coff = ib + 3 * S.nsr;
    V.wbase = ib + 4 * S.nsr;
    V.mlen = ib + 5 * S.nsr;
    V.item = reinterpret_cast<Item *>(ib + 6 * S.nsr);
    V.list = ib + 6 * S.nsr + 4 * S.nitem;
    return V;
}

// Work distribution of one scene's step: the threads of a block (block kernel: one block
// per scene) or of the whole grid (grid kernel: one scene over every SM).  Loops over
// subsystems take a warp each, loops over rows and constraints a thread each; sync() is a
// barrier over all of them.
struct BlockDist {
    // a scene's own block: its per-warp loops take the subsystems largest first, and the
    // chunks of W wait on per-subsystem flags instead of a barrier after the factor loop (a
    // scene over the whole grid has far more warps than subsystems, and its pollers would
    // load the L2 that its factorisations run through)
    static constexpr bool kSpread = true;
    int tid, nthreads, warp, nwarps;
    __device__ __forceinline__ BlockDist()
        : tid(threadIdx.x), nthreads(blockDim.x), warp(threadIdx.x >> 5), nwarps(blockDim.x >> 5) {}
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ void fence() const { __threadfence_block(); }
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier over the `expected` blocks of a cooperative launch.  Thread 0 of each block adds
// one to a counter that only grows (zeroed before the launch); the barrier of round r is
// complete when the counter reaches (r + 1) expected, which each block reads off its own
// arrival (arrivals of round r fall in [r expected, (r + 1) expected)).  The waiters poll
// the counter itself, so the last arrival completes the barrier with its one atomic.  A
// wait longer than limit_ns, or an error raised by another block, sets / sees the error
// flag and returns at once, here and at every later barrier, so the grid always runs to its
// end.  (`gen` is unused: kept for the scratch layout.)
__device__ __noinline__ void grid_barrier(unsigned *count, unsigned *gen, int *err,
                                          unsigned expected, unsigned long long limit_ns)
{
    (void)gen;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vcount = count;
        volatile int *verr = err;
        if (!*verr) {
            __threadfence();
            const unsigned my = atomicAdd(count, 1u);
            const unsigned target = (my / expected + 1u) * expected;
            if ((int)(*vcount - target) < 0) {
                const unsigned long long t0 = global_ns();
                while ((int)(*vcount - target) < 0) {
                    if (*verr) break;
                    if (global_ns() - t0 > limit_ns) { atomicExch(err, 1); break; }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
}

// Warps are numbered block-interleaved (warp k of block b is k * blocks + b): per-subsystem
// work (one warp each, FP64-bound in the setup and the recovery) then spreads over one warp
// per block, i.e. over the SMs and their FP64 pipes, instead of filling the first blocks.
struct GridDist {
    static constexpr bool kSpread = false;
    int tid, nthreads, warp, nwarps;
    unsigned *count, *gen;
    int *err;
    __device__ __forceinline__ GridDist(unsigned *c, unsigned *g, int *e)
        : tid(blockIdx.x * blockDim.x + threadIdx.x), nthreads(gridDim.x * blockDim.x),
          warp((int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x),
          nwarps((gridDim.x * blockDim.x) >> 5), count(c), gen(g), err(e) {}
    __device__ __forceinline__ void sync() const
    {
        grid_barrier(count, gen, err, gridDim.x, 20000000000ull);
    }
    __device__ __forceinline__ void fence() const { __threadfence(); }
};

template <typename T, typename Dist>
__device__ void scene_tables(const StepParams &P, const SceneDesc &S, const View<T> &V,
                             const Dist &d)
{
    for (int t = d.tid; t < S.nsr; t += d.nthreads) {
        V.row[t] = 0; V.sub[t] = 0; V.drow[t] = 0; V.coff[t] = 0; V.wbase[t] = 0; V.mlen[t] = 0;
    }
    d.sync();
    for (int j = d.tid; j < S.ncon; j += d.nthreads) {
        const ConDesc &c = P.cons[S.con0 + j];
        for (int s = 0; s < c.ns; ++s) {
            const SubDesc &u = P.subs[S.sub0 + c.sub[s]];
            for (int r = 0; r < c.rows; ++r) {
                const int t = c.sr[s] + r;
                const int lr = t - u.sr0;
                V.row[t] = c.row0 + r;
                V.sub[t] = c.sub[s];
                V.drow[t] = u.ot_D + lr * u.ldd;
                V.coff[t] = u.ot_c + lr;
                V.wbase[t] = u.sr0;
                V.mlen[t] = u.m;
            }
        }
    }
    for (int i = d.tid; i < S.nitem; i += d.nthreads) V.item[i] = P.items[S.item_g0 + i];
    for (int i = d.tid; i < S.nlist; i += d.nthreads) V.list[i] = P.lists[S.list_g0 + i];
}

// k, alpha, mu of a constraint (model kinds derive them from their drive gains)
__device__ __forceinline__ void con_params(const ConDesc &c, const double *pool, double h,
                                           double &k, double &alpha, double &mu)
{
    const double *p = pool + c.par_off;
    k = 0.0; alpha = 0.0; mu = 0.0;
    if (c.src <= SRC_CONTACT) {
        k = p[0]; alpha = p[1]; mu = p[2];
    } else if (c.src == SRC_ANGLE_PD) {
        k = p[18]; alpha = p[19] / p[18] + 0.5 * h;
    } else if (c.src == SRC_PLANE || c.src == SRC_SPHERE) {
        mu = p[22];
    }
}

// index (r, s), s <= r, of entry t of a lower triangle stored row by row
__device__ __forceinline__ void tri_index(int t, int &r, int &s)
{
    r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    s = t - r * (r + 1) / 2;
}

// Profile of a subsystem's K_i and the column spans of its J rows (built by the host from
// the structure of A_i and J_i): env[p] first column of row p inside the envelope, lastr[k]
// last row whose envelope reaches column k, [jlo[t], jhi[t]) the columns of J row t.
struct SubEnv {
    const int *env, *lastr, *jlo, *jhi;
    const int *grp;        // first rows of the row groups (ngrp + 1 entries)
    int ngrp;
};

__device__ __forceinline__ SubEnv sub_env(const StepParams &P, const SubDesc &u)
{
    SubEnv e;
    e.env = P.ipool + u.env_off;
    e.lastr = e.env + u.n;
    e.jlo = e.lastr + u.n;
    e.jhi = e.jlo + u.m;
    e.grp = P.ipool + u.grp_off;
    e.ngrp = u.ngrp;
    return e;
}

// A constant K_i whose factor from an earlier step is still held: in the workspace (it
// outlives the launch) or in shared memory from an earlier step of this launch.  With
// keep_factors 0 every step refactors (the same matrix; results agree to rounding).  A
// changed beta scale refactors too (K_i = A_i + beta_i J^T J changed).  A tc_phase 1 launch (the host issues it only for steps that refactor) refactors every tc
// subsystem.
__device__ __forceinline__ bool factor_kept(const StepParams &P, const SceneDesc &S,
                                            const SubDesc &u, int gsub, int step)
{
    if (P.tc_phase == 1 && u.tc) return false;
    return P.keep_factors && u.cst && (step > 0 || S.sub_global) && (P.subflag[gsub] & 1) &&
           P.beta_scale[gsub] == P.beta_used[gsub];
}

// K += beta J^T J on the lower triangle (row-major n x n), a row group at a time (rows
// with one column span [lo, lo + w)): lanes across the span's triangle entries, each summing
// its products over the group's rows with independent loads, then one update of K per
// entry and group (groups share entries, so they are added in turn)
template <typename F>
__device__ void add_jtj(F *K, int n, const double *J, const SubEnv &e, F beta)
{
    const int lane = threadIdx.x & 31;
    for (int g = 0; g < e.ngrp; ++g) {
        const int r0 = e.grp[g], r1 = e.grp[g + 1];
        const int lo = e.jlo[r0], w = e.jhi[r0] - lo;
        const double *J0 = J + (size_t)r0 * n + lo;
        for (int k = lane; k < w * (w + 1) / 2; k += 32) {
            int a, b;
            tri_index(k, a, b);
            F acc = (F)0;
            for (int t = 0; t < r1 - r0; ++t) acc += (F)J0[(size_t)t * n + a] * (F)J0[(size_t)t * n + b];
            K[(lo + a) * n + lo + b] += beta * acc;
        }
        __syncwarp();
    }
}

// Right-looking Cholesky inside the envelope, in place on the lower triangle of K (one
// warp).  Column k below the diagonal is scaled, then the triangle k < q <= r <= lastr[k]
// it reaches is updated with the lanes across its entries: a band of width w costs
// w (w + 1) / 64 warp instructions per column rather than w (on GB300 an FP64 warp
// instruction occupies its pipe however few lanes are active).  Every entry receives the
// same updates in the same order (k ascending).  INV_DIAG: the diagonal ends as 1/L_kk
// (the T factor); otherwise as L_kk with 1/L_kk in idg.  False on a non-positive pivot.
template <typename F, bool INV_DIAG>
__device__ bool env_cholesky(F *K, int n, const SubEnv &e, double *idg)
{
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < n; ++k) {
        const F d = K[k * n + k];
        if (!(d > (F)0) || !isfinite(d)) return false;
        const F ilkk = rsq(d);
        const int R = e.lastr[k];
        __syncwarp();
        for (int q = k + 1 + lane; q <= R; q += 32) K[q * n + k] *= ilkk;
        if (lane == 0) {
            if (INV_DIAG) {
                K[k * n + k] = ilkk;
            } else {
                K[k * n + k] = d * ilkk;
                idg[k] = (double)ilkk;
            }
        }
        __syncwarp();
        const int w = R - k, tri = w * (w + 1) / 2;
        for (int t = lane; t < tri; t += 32) {
            int a, b;
            tri_index(t, a, b);
            const int r = k + 1 + a, q = k + 1 + b;
            K[r * n + q] -= K[r * n + k] * K[q * n + k];
        }
        __syncwarp();
    }
    return true;
}

// Columns c0 .. c0 + 31 of W = L^-1 [J^T b] (column-major, W[p ldw + t]; a lane per
// column): column t < m is row t of J, column m is b, columns m < t < ldw are padding
// (zero).  Row t of J is zero outside its span [jlo[t], jhi[t]), so column t of W is zero
// above jlo[t]: the warp starts at the first such row among its columns and reads J's span
// directly (no separate transposed fill).  Rows above that start are written as zeros only
// when `whole` (a reader that takes W whole: the tensor-core Gram kernel); the map's
// items skip them.  The diagonal of LT holds 1/L_pp.
template <typename F>
__device__ void solve_w_chunk(const F *LT, F *W, const double *J, const double *b, int n,
                              int m, int ldw, int c0, const SubEnv &e, bool whole)
{
    const int lane = threadIdx.x & 31;
    const int t = c0 + lane;
    const bool act = t <= m;                       // a column of J^T or b
    const bool pad = t > m && t < ldw;             // zero padding
    const int lo = !act ? n : (t == m ? 0 : e.jlo[t]);
    const int hi = !act ? n : (t == m ? n : e.jhi[t]);
    int p0 = lo;
#pragma unroll
    for (int o = 16; o; o >>= 1) p0 = min(p0, __shfl_xor_sync(0xffffffffu, p0, o));
    if (pad)
        for (int p = 0; p < n; ++p) W[(size_t)p * ldw + t] = (F)0;
    if (whole && act)
        for (int p = 0; p < p0; ++p) W[(size_t)p * ldw + t] = (F)0;
    F *x = W + (act ? t : c0);                     // idle lanes read column c0, write nothing
    const double *Jt = J + (size_t)(act && t < m ? t : 0) * n;
    for (int p = p0; p < n; ++p) {
        const F *Lp = LT + (size_t)p * n;
        F s0 = (F)0, s1 = (F)0, s2 = (F)0, s3 = (F)0;
        if (p >= lo && p < hi) s0 = (F)(t == m ? b[p] : Jt[p]);
        int q = max(e.env[p], p0);                 // x[q] = 0 above p0
        for (; q + 3 < p; q += 4) {
            s0 -= Lp[q] * x[(size_t)q * ldw];
            s1 -= Lp[q + 1] * x[(size_t)(q + 1) * ldw];
            s2 -= Lp[q + 2] * x[(size_t)(q + 2) * ldw];
            s3 -= Lp[q + 3] * x[(size_t)(q + 3) * ldw];
        }
        for (; q < p; ++q) s0 -= Lp[q] * x[(size_t)q * ldw];
        if (act) x[(size_t)p * ldw] = ((s0 + s1) + (s2 + s3)) * Lp[p];
    }
}

// The range of a prefix table pre[0 .. nsub] (pre[0] = 0, nondecreasing) that holds item w
// < pre[nsub]: the i with pre[i] <= w < pre[i + 1]
__device__ __forceinline__ int pre_find(const int *pre, int nsub, int w)
{
    int lo = 0, hi = nsub;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

// x[q ldx] -= a[q lda] f for q0 <= q < q1 (warp, lanes across q).  Whole passes of 8 x 32
// entries load their a and x before writing any x (x and a may share a type, so the
// compiler could not move a load of a above a store to x, and each entry would cost a
// round trip); the remainder takes one more such pass if it is long, else one pass of 2 x 32
// or 32.  The passes are warp-uniform: a short range issues no predicated-off
// instructions (an FP64 one occupies its pipe all the same).
template <int K, typename F, typename G>
__device__ __forceinline__ void axpy_pass(F *x, int ldx, const G *a, int lda, int q, int q1, F f)
{
    G av[K];
    F xv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int qq = q + 32 * k;
        av[k] = qq < q1 ? a[qq * lda] : (G)0;
        xv[k] = qq < q1 ? x[qq * ldx] : (F)0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int qq = q + 32 * k;
        if (qq < q1) x[qq * ldx] = xv[k] - (F)av[k] * f;
    }
}

// (indices: q lda and q ldx stay below 2^31 for the supported sizes, n, m <= 2048)
template <typename F, typename G>
__device__ __forceinline__ void warp_axpy_neg(F *x, int ldx, const G *a, int lda, int q0, int q1,
                                              F f)
{
    const int lane = threadIdx.x & 31;
    if (q1 - q0 <= 32) {                     // one entry per lane at most
        const int q = q0 + lane;
        if (q < q1) x[q * ldx] -= (F)a[q * lda] * f;
        return;
    }
    int base = q0;
    for (; base + 256 <= q1; base += 256) axpy_pass<8>(x, ldx, a, lda, base + lane, q1, f);
    if (q1 - base > 64) {                    // a long range's remainder in one pass
        axpy_pass<8>(x, ldx, a, lda, base + lane, q1, f);
        return;
    }
    // at most 64 entries left
    if (q1 - base > 32) axpy_pass<2>(x, ldx, a, lda, base + lane, q1, f);
    else if (q1 > base) axpy_pass<1>(x, ldx, a, lda, base + lane, q1, f);
}

// y <- L^-1 y for one vector (stride ldy), column by column: lanes update the rows below p
template <typename F>
__device__ void env_forward_vec(const F *LT, F *y, int n, int ldy, const int *lastr)
{
    const int lane = threadIdx.x & 31;
    for (int p = 0; p < n; ++p) {
        const F yp = y[p * ldy] * LT[p * n + p];
        __syncwarp();
        if (lane == 0) y[p * ldy] = yp;
        warp_axpy_neg(y, ldy, LT + p, n, p + 1, lastr[p] + 1, yp);
        __syncwarp();
    }
}

// One work item of the map D = W^T W, c = W^T g of a subsystem (W = L^-1 [J^T b], column m
// is g; W column t is zero above row jlo[t]; D rows ldd apart, zero-padded from m to mp), for
// items spread over many threads: item k < nb (nb + 1) / 2 is the 4 x 4 block k of D's lower
// triangle (mirrored; per row p of W a thread loads 4 + 4 values for 16 FMAs); item
// nb (nb + 1) / 2 + q gives c and the zero padding of D for rows 4q .. 4q + 3.

template <typename F>
__device__ void map_item(const F *W, int n, int m, int mp, int ldd, int ldw, const int *jlo,
                         F *D, F *cc, int k, bool with_D)
{
    const int nb = (m + 3) / 4, ntri = nb * (nb + 1) / 2;
    if (k < ntri) {
        if (!with_D) return;
        int bi, bj;
        tri_index(k, bi, bj);
        const int r0 = 4 * bi, s0 = 4 * bj;
        int pr = n, ps = n;
        for (int q = 0; q < 4; ++q) {
            if (r0 + q < m) pr = min(pr, jlo[r0 + q]);
            if (s0 + q < m) ps = min(ps, jlo[s0 + q]);
        }
        F acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = (F)0;
        for (int p = max(pr, ps); p < n; ++p) {
            const F *Wp = W + (size_t)p * ldw;
            F wr[4], ws[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { wr[q] = Wp[r0 + q]; ws[q] = Wp[s0 + q]; }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += wr[a] * ws[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int r = r0 + a, s = s0 + b;
                if (r < m && s < m && s <= r) {
                    D[r * ldd + s] = acc[a][b];
                    D[s * ldd + r] = acc[a][b];
                }
            }
        }
        return;
    }
    const int q0 = 4 * (k - ntri);
    for (int r = q0; r < q0 + 4 && r < m; ++r) {
        F a0 = (F)0, a1 = (F)0;
        int p = jlo[r];
        for (; p + 1 < n; p += 2) {
            a0 += W[p * ldw + r] * W[p * ldw + m];
            a1 += W[(p + 1) * ldw + r] * W[(p + 1) * ldw + m];
        }
        if (p < n) a0 += W[p * ldw + r] * W[p * ldw + m];
        cc[r] = a0 + a1;
        if (with_D)
            for (int t = m; t < mp; ++t) D[r * ldd + t] = (F)0;
    }
}

// K_i = A_i + beta_i J_i^T J_i in FP32 for the blocks whose factorisation is left to the
// blocked tensor-core factorisation (step flag 4, set before the barrier that precedes this),
// a warp per row over every warp of the scene: the lower triangle from the first column of
// the envelope's tile of the row's tile row on (zeros left of the envelope: that
// factorisation reads whole tiles), then, for every row group whose span holds the row's
// column p (ascending), the group's products summed over its rows and added times beta: the
// arithmetic of add_jtj, entry by entry.
template <typename T, typename Dist>
__device__ void deferred_fill(const StepParams &P, const SceneDesc &S, const View<T> &V,
                              const Dist &d)
{
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < S.nsub; ++i) {
        if (P.pending[S.sub0 + i] != 4) continue;
        const SubDesc &u = P.subs[S.sub0 + i];
        const int n = u.n;
        const SubEnv e = sub_env(P, u);
        const double *K = V.sdb + u.od_L, *J = V.sdb + u.od_J;
        T *LT = V.stb + u.ot_L;
        const T beta = (T)V.db[S.od_beta + i];
        for (int p = d.warp; p < n; p += d.nwarps) {
            const int ep = e.env[p], q0 = e.env[p & ~127] & ~127;
            T *Lp = LT + (size_t)p * n;
            for (int q = q0 + lane; q <= p; q += 32) Lp[q] = q < ep ? (T)0 : (T)K[(size_t)p * n + q];
            __syncwarp();
            for (int g0 = 0; g0 < e.ngrp; g0 += 32) {
                bool cov = false;
                if (g0 + lane < e.ngrp) {
                    const int r0 = e.grp[g0 + lane];
                    cov = e.jlo[r0] <= p && p < e.jhi[r0];
                }
                for (unsigned mask = __ballot_sync(0xffffffffu, cov); mask; mask &= mask - 1) {
                    const int g = g0 + __ffs(mask) - 1;
                    const int r0 = e.grp[g], r1 = e.grp[g + 1], lo = e.jlo[r0];
                    for (int q = lo + lane; q <= p; q += 32) {
                        T acc = (T)0;
                        for (int r = r0; r < r1; ++r)
                            acc += (T)J[(size_t)r * n + p] * (T)J[(size_t)r * n + q];
                        Lp[q] += beta * acc;
                    }
                    __syncwarp();
                }
            }
        }
    }
}

// W = L^-1 [J^T b] of the subsystems whose step flag is `want` (3: factorised by the setup;
// 4: by the blocked tensor-core factorisation), in chunks of 32 columns, a warp per chunk over
// every warp of the scene, so that one large subsystem does not hold a single warp (and the
// scene) for all of its columns.  With flags still being set (want 3 in the setup, the spread
// distribution: no barrier after the factor loop) a chunk waits for its own subsystem's flag,
// and the chunks run smallest subsystem first (the largest are factorised first and take
// longest), so the chunks of the others overlap the largest factorisations.  Each warp ends
// its factor tasks before it takes a chunk, so every wait ends; it is bounded all the same (a
// wait that runs out marks the scene ST_TIMEOUT and skips the chunk).
template <typename T, typename Dist>
__device__ void w_chunks(const StepParams &P, const SceneDesc &S, const View<T> &V,
                         int *s_status, const Dist &d, int want)
{
    const int lane = threadIdx.x & 31;
    const double *sdb = V.sdb;
    T *stb = V.stb;
    {
        const int *wpre = P.ipool + S.pre_off, *ord = P.ipool + S.ord_off;
        const int total = __ldg(wpre + S.nsub);
        for (int w = d.warp; w < total; w += d.nwarps) {
            const int pos = pre_find(wpre, S.nsub, w);
            const int i = __ldg(ord + S.nsub - 1 - pos);
            int flag = 0;
            if (lane == 0 && !Dist::kSpread) {
                flag = P.pending[S.sub0 + i];     // set before the barrier above
            } else if (lane == 0) {
                volatile int *vf = &P.pending[S.sub0 + i];
                flag = *vf;
                for (long long spin = 0; flag == -1; ++spin) {
                    if (spin > (1ll << 26)) { *s_status = ST_TIMEOUT; break; }
                    __nanosleep(64);
                    flag = *vf;
                }
                d.fence();                        // the factor after its flag
            }
            flag = __shfl_sync(0xffffffffu, flag, 0);
            if (flag != want) continue;
            const SubDesc &u = P.subs[S.sub0 + i];
            const int ldw = (u.m + 1 + 3) / 4 * 4;
            solve_w_chunk<T>(stb + u.ot_L, stb + u.ot_W, sdb + u.od_J, sdb + u.od_b, u.n, u.m,
                             ldw, 32 * (w - __ldg(wpre + pos)), sub_env(P, u),
                             (P.tc_phase == 1 || P.tc_phase == 3) && u.tc);
        }
    }
}

// assemble .. factor .. map, and the per-step constants of the z-step
template <typename T, typename Dist>
__device__ long long scene_setup(const StepParams &P, const SceneDesc &S, const View<T> &V,
                                 int *s_status, int step, const Dist &d)
{
    const int lane = threadIdx.x & 31;
    constexpr bool MIXED = sizeof(T) == 4;
    double *db = V.db, *sdb = V.sdb;
    T *tb = V.tb, *stb = V.stb, *htb = V.htb;
    for (int i = d.warp; i < S.nsub; i += d.nwarps) {
        const SubDesc &u = P.subs[S.sub0 + i];
        const SubEnv e = sub_env(P, u);
        const bool keep = factor_kept(P, S, u, S.sub0 + i, step);
        double *J = sdb + u.od_J, *K = sdb + u.od_L;
        // J's rows are read only inside their column spans (model rows are written there,
        // explicit rows whole): zero the spans
        for (int g = 0; g < e.ngrp; ++g) {
            const int r0 = e.grp[g], r1 = e.grp[g + 1], lo = e.jlo[r0], w = e.jhi[r0] - lo;
            for (int k = lane; k < (r1 - r0) * w; k += 32)
                J[(size_t)(r0 + k / w) * u.n + lo + k % w] = 0.0;
        }
        if (u.kind == KIND_GENERIC) {
            const double *A = P.pool + u.gen_off;
            for (int q = lane; q < u.n * u.n; q += 32) K[q] = A[q];
            for (int q = lane; q < u.n; q += 32) sdb[u.od_b + q] = A[u.n * u.n + q];
            continue;
        }
        if (!keep) {
            // the band [env[p], lastr[p]] of every row holds A (both triangles)
            for (int p = 0; p < u.n; ++p)
                for (int q = e.env[p] + lane; q <= e.lastr[p]; q += 32) K[p * u.n + q] = 0.0;
        }
        if (u.kind == KIND_LINEAR) {
            // A = (2/h) M + (h/2) K_el (K_el sparse, scattered into the band);
            // b from the node state (Eq. ddyn, elastic force at the midpoint)
            __syncwarp();
            const double *mass = P.pool + u.gen_off;
            const double *f = mass + u.nb, *X0 = f + u.n, *Kval = X0 + u.n;
            const int *rowp = P.ipool + u.csr_off, *col = rowp + u.n + 1;
            const double gv[3] = {P.g0, P.g1, P.g2};
            const double *nodes = P.nodes + (size_t)u.body0 * SUBADMM_NODE;
            if (u.ne > 0) {
                // co-rotational: (2/h) M on the diagonal and b without the elastic force here;
                // the elements add (h/2) R K_e R^T and their forces in the pass below
                for (int p = lane; p < u.n; p += 32) {
                    const double m = mass[p / 3];
                    K[p * u.n + p] = (2.0 / P.h) * m;
                    sdb[u.od_b + p] = (2.0 / P.h) * m * nodes[(p / 3) * SUBADMM_NODE + 3 + p % 3] +
                                      f[p] + m * gv[p % 3];
                }
                __syncwarp();
                continue;
            }
            double *ux = sdb + u.od_v;               // x - X0 (v-hat is rewritten later)
            for (int p = lane; p < u.n; p += 32) ux[p] = nodes[(p / 3) * SUBADMM_NODE + p % 3] - X0[p];
            if (!keep) {
                for (int p = lane; p < u.n; p += 32) {
                    const int q1 = rowp[p + 1];
#pragma unroll 4
                    for (int q = rowp[p]; q < q1; ++q) K[p * u.n + col[q]] = 0.5 * P.h * Kval[q];
                }
                __syncwarp();
                for (int p = lane; p < u.n; p += 32) K[p * u.n + p] += (2.0 / P.h) * mass[p / 3];
            }
            __syncwarp();
            for (int p = lane; p < u.n; p += 32)
                sdb[u.od_b + p] = linear_b(p, mass, f, ux, Kval, rowp, col, nodes, P.h, gv);
        }
    }
    d.sync();
    // co-rotational blocks: every element's rotated stiffness and force, the elements of all
    // such blocks of the scene spread over every thread
    {
        int total = 0;
        for (int i = 0; i < S.nsub; ++i) total += P.subs[S.sub0 + i].ne;
        for (int w = d.tid; w < total; w += d.nthreads) {
            int el = w, i = 0;
            for (; i < S.nsub; ++i) {
                const int ne = P.subs[S.sub0 + i].ne;
                if (el < ne) break;
                el -= ne;
            }
            const SubDesc &u = P.subs[S.sub0 + i];
            const double *X0 = P.pool + u.gen_off + u.nb + u.n;
            corot_element(P.ipool + u.tet_off + 4 * el, P.pool + u.ke_off + 144 * (size_t)el, X0,
                          P.nodes + (size_t)u.body0 * SUBADMM_NODE, P.h, u.n, sdb + u.od_L,
                          sdb + u.od_b);
        }
    }
    // rigid bodies: diagonal A = (2/h) M and b (lane per body)
    for (int i = d.warp; i < S.nsub; i += d.nwarps) {
        const SubDesc &u = P.subs[S.sub0 + i];
        if (u.kind != KIND_RIGID) continue;
        for (int k = lane; k < u.nb; k += 32) {
            double Ad[6], bb[6];
            body_dynamics(P.bodies + (size_t)(u.body0 + k) * SUBADMM_BODY, P.h, P.g0, P.g1, P.g2,
                          Ad, bb);
            double *K = sdb + u.od_L;
            for (int d = 0; d < 6; ++d) {
                const int q = 6 * k + d;
                K[q * u.n + q] = Ad[d];
                sdb[u.od_b + q] = bb[d];
            }
        }
    }
    // constraint rows into J (FP64) and e; constraints in the host's assembly order, which
    // groups kinds by warp so a warp runs one kind's code path
    T *E = tb + S.ot_e;
    for (int a = d.tid; a < S.nasm; a += d.nthreads) {
        const int j = P.asm_order[S.asm_g0 + a];
        if (j < 0) continue;
        const ConDesc &c = P.cons[S.con0 + j];
        if (c.src <= SRC_CONTACT) {
            const double *p = P.pool + c.par_off + 3;
            for (int r = 0; r < c.rows; ++r) E[c.row0 + r] = (T)p[r];
            const double *Jp = p + c.rows;
            for (int s = 0; s < c.ns; ++s) {
                const SubDesc &u = P.subs[S.sub0 + c.sub[s]];
                for (int r = 0; r < c.rows; ++r) {
                    double *Jr = sdb + u.od_J + (c.sr[s] + r - u.sr0) * u.n;
                    for (int q = 0; q < u.n; ++q) Jr[q] = Jp[r * u.n + q];
                }
                Jp += c.rows * u.n;
            }
        } else {
            double Ja[30], Jb[30], ee[5], kk = 0.0, al = 0.0;
            model_rows(c, P.pool + c.par_off, P.bodies, P.nodes, P.h, P.gamma, Ja, Jb, ee, &kk, &al);
            for (int r = 0; r < c.rows; ++r) E[c.row0 + r] = (T)ee[r];
            {
                // a body side fills 6 columns at 6 * index, a node side 3 columns at 3 * index
                const SubDesc &u = P.subs[S.sub0 + c.sub[0]];
                const int wa = c.node_a ? 3 : 6;
                for (int r = 0; r < c.rows; ++r) {
                    double *Jr = sdb + u.od_J + (c.sr[0] + r - u.sr0) * u.n + wa * c.ba;
                    for (int q = 0; q < wa; ++q) Jr[q] = Ja[6 * r + q];
                }
            }
            if (c.side_b >= 0) {
                const SubDesc &u = P.subs[S.sub0 + c.sub[c.side_b]];
                const int wb = c.node_b ? 3 : 6;
                for (int r = 0; r < c.rows; ++r) {
                    double *Jr = sdb + u.od_J + (c.sr[c.side_b] + r - u.sr0) * u.n + wb * c.bb;
                    for (int q = 0; q < wb; ++q) Jr[q] += Jb[6 * r + q];
                }
            }
        }
    }
    // factor-ready flags of this step (see the factor loop): -1 until a subsystem is done
    for (int i = d.tid; i < S.nsub; i += d.nthreads) P.pending[S.sub0 + i] = -1;
    d.sync();
    const long long t_asm = clock64();
    // per subsystem (one warp each): beta, K = A + beta J^T J and its Cholesky factor, then
    // the map W = L^-1 [J^T b], D = W^T W, c.  The FP64 form and the stiff blocks of the mixed
    // form factorise K in FP64 (rounded into the T copy); the other mixed blocks factorise in
    // FP32, keeping the FP64 A, b and J for the recovery and refinement of v-hat.
    for (int k = d.warp; k < S.nsub; k += d.nwarps) {
        const int i = Dist::kSpread ? __ldg(P.ipool + S.ord_off + k) : k;   // largest first
        const SubDesc &u = P.subs[S.sub0 + i];
        const int gsub = S.sub0 + i;
        // W's leading dimension: m + 1 columns rounded up to 4 (map_item reads 4-column blocks)
        const int n = u.n, m = u.m, ldw = (m + 1 + 3) / 4 * 4;
        const SubEnv e = sub_env(P, u);
        double *J = sdb + u.od_J, *K = sdb + u.od_L, *b = sdb + u.od_b, *idg = sdb + u.od_id;
        T *LT = stb + u.ot_L, *W = stb + u.ot_W;
        if (factor_kept(P, S, u, gsub, step)) {
            // constant K_i: only g = L^-1 b and c change (and D when the launch lost it)
            if (step == 0 && lane == 0) {
                db[S.od_beta + i] = P.beta[gsub];
                db[S.od_flag + i] = (P.subflag[gsub] & 2) ? 1.0 : 0.0;
            }
            for (int p = lane; p < n; p += 32) W[p * ldw + m] = (T)b[p];
            __syncwarp();
            env_forward_vec<T>(LT, W + m, n, ldw, e.lastr);
            // c (and D if the launch lost it) below, over every thread of the scene
            __syncwarp();
            if (lane == 0) {
                d.fence();
                *(volatile int *)&P.pending[gsub] = (step == 0 && !S.hot_global) ? 2 : 1;
            }
            __syncwarp();
            continue;
        }
        // beta_i = Tr(A_i) / Tr(J_ci^T J_ci)  (Sec. III-D)
        double beta;
        if (!MIXED) {
            double trA = 0.0, trJ = 0.0;
            for (int q = lane; q < n; q += 32) trA += K[q * n + q];
            for (int g = 0; g < e.ngrp; ++g) {            // J's rows inside their spans
                const int r0 = e.grp[g], r1 = e.grp[g + 1], lo = e.jlo[r0], w = e.jhi[r0] - lo;
                for (int k = lane; k < (r1 - r0) * w; k += 32) {
                    const double x = J[(size_t)(r0 + k / w) * n + lo + k % w];
                    trJ += x * x;
                }
            }
            trA = warp_sum(trA);
            trJ = warp_sum(trJ);
            beta = P.beta_fixed ? P.rho : (trJ > 0.0 ? trA / trJ : 1.0);
        } else {
            T trA = (T)0, trJ = (T)0;
            for (int q = lane; q < n; q += 32) trA += (T)K[q * n + q];
            for (int g = 0; g < e.ngrp; ++g) {
                const int r0 = e.grp[g], r1 = e.grp[g + 1], lo = e.jlo[r0], w = e.jhi[r0] - lo;
                for (int k = lane; k < (r1 - r0) * w; k += 32) {
                    const T jq = (T)J[(size_t)(r0 + k / w) * n + lo + k % w];
                    trJ += jq * jq;
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                trA += __shfl_xor_sync(0xffffffffu, trA, o);
                trJ += __shfl_xor_sync(0xffffffffu, trJ, o);
            }
            beta = (double)(P.beta_fixed ? (T)P.rho : (trJ > (T)0 ? trA / trJ : (T)1));
        }
        beta *= P.beta_scale[gsub];
        if (P.pj) beta = 0.0;                       // Projected Jacobi: K_i = A_i
        if (lane == 0) {
            db[S.od_beta + i] = beta;
            P.beta[gsub] = beta;
            P.beta_used[gsub] = P.beta_scale[gsub];
        }
        bool stiff = true;
        if (MIXED) {
            // stiffness test: the spread of K's diagonal bounds its condition number from
            // below; a stiff or high-mass-ratio block (spread > 1e3) is factorised in FP64
            const T bt = (T)beta;
            T dmax = (T)0, dmin = (T)3.0e38;
            for (int p = lane; p < n; p += 32) {
                T cs = (T)0;                       // rows whose span holds column p, in order
                for (int g = 0; g < e.ngrp; ++g) {
                    const int r0 = e.grp[g];
                    if (p < e.jlo[r0] || p >= e.jhi[r0]) continue;
                    for (int r = r0; r < e.grp[g + 1]; ++r) {
                        const T jr = (T)J[r * n + p];
                        cs += jr * jr;
                    }
                }
                const T dk = (T)K[p * n + p] + bt * cs;
                dmax = dk > dmax ? dk : dmax;
                dmin = dk < dmin ? dk : dmin;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const T a = __shfl_xor_sync(0xffffffffu, dmax, o);
                const T c = __shfl_xor_sync(0xffffffffu, dmin, o);
                dmax = a > dmax ? a : dmax;
                dmin = c < dmin ? c : dmin;
            }
            stiff = !(dmin > (T)0) || dmax > (T)1.0e3 * dmin;
            if (lane == 0) db[S.od_flag + i] = stiff ? 1.0 : 0.0;
        }
        bool ok;
        const bool defer = MIXED && !stiff && P.tc_factor && P.tc_phase == 1 && u.tc;
        if (stiff) {
            add_jtj<double>(K, n, J, e, beta);
            ok = env_cholesky<double, false>(K, n, e, idg);
            if (ok) {
                for (int p = 0; p < n; ++p)
                    for (int q = e.env[p] + lane; q <= p; q += 32)
                        LT[p * n + q] = (q == p) ? (T)idg[p] : (T)K[p * n + q];
            }
        } else if (defer) {
            ok = true;                            // K in FP32 by deferred_fill, below
        } else {
            for (int p = 0; p < n; ++p)
                for (int q = e.env[p] + lane; q <= p; q += 32) LT[p * n + q] = (T)K[p * n + q];
            __syncwarp();
            add_jtj<T>(LT, n, J, e, (T)beta);
            ok = env_cholesky<T, true>(LT, n, e, nullptr);
        }
        if (u.cst && lane == 0) P.subflag[gsub] = ok ? (1 | (stiff ? 2 : 0)) : 0;
        __syncwarp();
        if (lane == 0) {
            d.fence();                            // the factor before its flag
            // 3: W, then D and c, below; 4: factor, W, D and c after this launch
            *(volatile int *)&P.pending[gsub] = ok ? (defer ? 4 : 3) : 0;
            if (!ok) *s_status = ST_NOTSPD;
        }
        __syncwarp();
    }
    // W = L^-1 [J^T b] of the subsystems factorised above (flag 3); K of the deferred ones
    if (!Dist::kSpread) d.sync();
    if (P.tc_factor && P.tc_phase == 1) deferred_fill<T>(P, S, V, d);
    w_chunks<T>(P, S, V, s_status, d, 3);
    d.sync();
    // the maps D = W^T W and c = W^T g of this step (pending >= 2: D and c, 1: c only), their
    // items (rows of c, then 4 x 4 blocks of D) spread over every thread of the scene and
    // found through the scene's prefix tables; the tensor-core Gram kernel forms them for
    // the tc subsystems in the first launch of a three-launch step
    {
        const int *cpre = P.ipool + S.pre_off + (S.nsub + 1), *dpre = cpre + (S.nsub + 1);
        const int ctot = __ldg(cpre + S.nsub), total = ctot + __ldg(dpre + S.nsub);
        for (int w = d.tid; w < total; w += d.nthreads) {
            const bool cpart = w < ctot;
            const int wl = cpart ? w : w - ctot;
            const int i = pre_find(cpart ? cpre : dpre, S.nsub, wl);
            const int pend = P.pending[S.sub0 + i];
            if (pend == 0 || (!cpart && pend < 2)) continue;
            const SubDesc &u = P.subs[S.sub0 + i];
            if (P.tc_phase == 1 && u.tc) continue;
            const int nb = (u.m + 3) / 4;
            const int k = (cpart ? nb * (nb + 1) / 2 : 0) + wl - __ldg((cpart ? cpre : dpre) + i);
            const int ldw = (u.m + 1 + 3) / 4 * 4;
            map_item<T>(stb + u.ot_W, u.n, u.m, u.mpad, u.ldd, ldw, sub_env(P, u).jlo,
                        htb + u.ot_D, htb + u.ot_c, k, pend >= 2);
        }
    }
    d.sync();
    // per-step z-step constants: 1/s, soft gain k/(1 + s alpha k), alpha, mu (per row);
    // beta and 1/beta per side-row
    T *INVS = tb + S.ot_invs, *KF = tb + S.ot_kf, *AL = tb + S.ot_al, *MU = tb + S.ot_mu;
    T *INVB = tb + S.ot_invb, *BT = tb + S.ot_b;
    const double *BETA = db + S.od_beta;
    for (int j = d.tid; j < S.ncon; j += d.nthreads) {
        const ConDesc &c = P.cons[S.con0 + j];
        if (P.pj) {
            // Projected Jacobi: 1/delta per row, delta = the sum over its sides of D's diagonal
            // entry (both tangents of a contact take the larger of theirs), soft gain
            // k/(1 + k alpha delta); beta and 1/beta per side-row are zero
            double kk, al, mu;
            con_params(c, P.pool, P.h, kk, al, mu);
            double dl[3] = {0.0, 0.0, 0.0};
            for (int r = 0; r < c.rows; ++r) {
                double dr = 0.0;
                for (int q = 0; q < c.ns; ++q) {
                    const SubDesc &u = P.subs[S.sub0 + c.sub[q]];
                    const int lr = c.sr[q] + r - u.sr0;
                    dr += (double)htb[u.ot_D + (size_t)lr * u.ldd + lr];
                }
                if (c.type == TYPE_CONTACT) dl[r] = dr;
                else {
                    INVS[c.row0 + r] = (T)(1.0 / dr);
                    KF[c.row0 + r] = (T)(c.type == TYPE_SOFT ? kk / (1.0 + kk * al * dr) : 0.0);
                }
                AL[c.row0 + r] = (T)al;
                MU[c.row0 + r] = (T)mu;
            }
            if (c.type == TYPE_CONTACT) {
                const double dt = dl[1] > dl[2] ? dl[1] : dl[2];
                INVS[c.row0] = (T)(1.0 / dl[0]);
                INVS[c.row0 + 1] = (T)(1.0 / dt);
                INVS[c.row0 + 2] = (T)(1.0 / dt);
                for (int r = 0; r < 3; ++r) KF[c.row0 + r] = (T)0;
            }
            for (int q = 0; q < c.ns; ++q)
                for (int r = 0; r < c.rows; ++r) {
                    INVB[c.sr[q] + r] = (T)0;
                    BT[c.sr[q] + r] = (T)0;
                }
            continue;
        }
        double s = 0.0;
        for (int q = 0; q < c.ns; ++q) s += 1.0 / BETA[c.sub[q]];
        double kk, al, mu;
        con_params(c, P.pool, P.h, kk, al, mu);
        const double kf = (c.type == TYPE_SOFT) ? kk / (1.0 + s * al * kk) : 0.0;
        for (int r = 0; r < c.rows; ++r) {
            INVS[c.row0 + r] = (T)(1.0 / s);
            KF[c.row0 + r] = (T)kf;
            AL[c.row0 + r] = (T)al;
            MU[c.row0 + r] = (T)mu;
        }
        for (int q = 0; q < c.ns; ++q) {
            const double be = BETA[c.sub[q]];
            for (int r = 0; r < c.rows; ++r) {
                INVB[c.sr[q] + r] = (T)(1.0 / be);
                BT[c.sr[q] + r] = (T)be;
            }
        }
    }
    d.sync();
    return t_asm;
}

// out += J^T w (FP64) over the column span of each row group (lanes across the span, each
// summing over the group's rows, then one update of out per group), in row order:
// deterministic, and O(sum of spans) instead of O(m n)
template <typename W>
__device__ __forceinline__ void add_jt(double *out, const double *J, int n, const SubEnv &e,
                                       const W *w)
{
    const int lane = threadIdx.x & 31;
    for (int g = 0; g < e.ngrp; ++g) {
        const int r0 = e.grp[g], r1 = e.grp[g + 1];
        for (int p = e.jlo[r0] + lane; p < e.jhi[r0]; p += 32) {
            double acc = 0.0;
            for (int r = r0; r < r1; ++r) acc += J[(size_t)r * n + p] * (double)w[r];
            out[p] += acc;
        }
        __syncwarp();
    }
}

// Triangular solves with the T factor (1/L_pp on its diagonal), in place on s (warp),
// inside the envelope.
template <typename T>
__device__ __forceinline__ void warp_chol_solve(const T *LT, T *s, int n, const SubEnv &e)
{
    const int lane = threadIdx.x & 31;
    for (int p = 0; p < n; ++p) {              // L y = s (column-oriented)
        const T yp = s[p] * LT[p * n + p];
        __syncwarp();
        if (lane == 0) s[p] = yp;
        warp_axpy_neg(s, 1, LT + p, n, p + 1, e.lastr[p] + 1, yp);
        __syncwarp();
    }
    for (int p = n - 1; p >= 0; --p) {         // L^T v = y
        const T vp = s[p] * LT[p * n + p];
        __syncwarp();
        if (lane == 0) s[p] = vp;
        warp_axpy_neg(s, 1, LT + p * n, 1, e.env[p], p, vp);
        __syncwarp();
    }
}

// v-hat of the last v-step, v = K^-1 (b + J^T w), in FP64 (warp per subsystem) into od_v.
// With an FP64 factor (FP64 form, or a stiff block of the mixed form): two triangular
// solves.  With an FP32 factor: a solve, then one step of iterative refinement with the
// residual b + J^T w - K v formed in FP64 from A (kept in od_L) and J:
// K v = A v + beta J^T (J v).
// `fast` (may be null): per-warp shared memory of fast_len T values; the FP32 solves of a
// subsystem with n <= fast_len run on a copy there instead of on the global scratch vector.
template <typename T, typename Dist>
__device__ void recover_v(const StepParams &P, const SceneDesc &S, const View<T> &V, const T *w,
                          const Dist &d, T *fast = nullptr, int fast_len = 0)
{
    constexpr bool MIXED = sizeof(T) == 4;
    const int lane = threadIdx.x & 31;
    for (int k = d.warp; k < S.nsub; k += d.nwarps) {
        const int i = Dist::kSpread ? __ldg(P.ipool + S.ord_off + k) : k;   // largest first
        const SubDesc &u = P.subs[S.sub0 + i];
        const int n = u.n, m = u.m;
        const SubEnv e = sub_env(P, u);
        // od_L holds the FP64 factor L (FP64 form) or A itself (mixed form)
        const double *J = V.sdb + u.od_J, *Lf = V.sdb + u.od_L, *b = V.sdb + u.od_b;
        double *idg = V.sdb + u.od_id;
        double *v = V.sdb + u.od_v;
        const T *wi = w + u.sr0;
        if (!MIXED || V.db[S.od_flag + i] != 0.0) {
            for (int p = lane; p < n; p += 32) v[p] = b[p];
            __syncwarp();
            add_jt(v, J, n, e, wi);
            for (int p = 0; p < n; ++p) {          // L y = rhs (column-oriented)
                const double yp = v[p] * idg[p];
                __syncwarp();
                if (lane == 0) v[p] = yp;
                warp_axpy_neg(v, 1, Lf + p, n, p + 1, e.lastr[p] + 1, yp);
                __syncwarp();
            }
            for (int p = n - 1; p >= 0; --p) {     // L^T v = y
                const double vp = v[p] * idg[p];
                __syncwarp();
                if (lane == 0) v[p] = vp;
                warp_axpy_neg(v, 1, Lf + p * n, 1, e.env[p], p, vp);
                __syncwarp();
            }
            continue;
        }
        const T *LT = V.stb + u.ot_L;
        T *s = (fast && n <= fast_len) ? fast : V.stb + u.ot_s;
        double *rhs = idg;                          // (unused by the mixed factor)
        double *t = V.sdb + u.od_t;
        const double beta = V.db[S.od_beta + i];
        for (int p = lane; p < n; p += 32) rhs[p] = b[p];
        __syncwarp();
        add_jt(rhs, J, n, e, wi);
        for (int p = lane; p < n; p += 32) s[p] = (T)rhs[p];
        __syncwarp();
        warp_chol_solve<T>(LT, s, n, e);
        for (int p = lane; p < n; p += 32) v[p] = (double)s[p];
        __syncwarp();
        // one refinement step: r = rhs - A v - beta J^T (J v); v += K^-1 r.  Row p of A lies
        // inside the band [env[p], lastr[p]]
        for (int r = lane; r < m; r += 32) {
            double acc = 0.0;
            for (int p = e.jlo[r]; p < e.jhi[r]; ++p) acc += J[r * n + p] * v[p];
            t[r] = acc;
        }
        __syncwarp();
        for (int r = lane; r < m; r += 32) t[r] *= -beta;
        __syncwarp();
        // s = rhs - A v - beta J^T t, with J^T (-beta t) added into the FP64 rhs copy
        add_jt(rhs, J, n, e, t);
        for (int p = lane; p < n; p += 32) {
            double acc = rhs[p];
            for (int q = e.env[p]; q <= e.lastr[p]; ++q) acc -= Lf[p * n + q] * v[q];     // A v
            s[p] = (T)acc;
        }
        __syncwarp();
        warp_chol_solve<T>(LT, s, n, e);
        for (int p = lane; p < n; p += 32) v[p] += (double)s[p];
        __syncwarp();
    }
}

// The block kernel's once-per-step phases as calls (arguments by value), so that the
// register allocation of its iteration loop is not shaped by the setup code's.
template <typename T>
__device__ __noinline__ long long block_setup(StepParams P, SceneDesc S, View<T> V, int *status,
                                              int step)
{
    return scene_setup<T>(P, S, V, status, step, BlockDist());
}

template <typename T>
__device__ __noinline__ void block_recover(StepParams P, SceneDesc S, View<T> V, const T *w)
{
    recover_v<T>(P, S, V, w, BlockDist());
}

// Initial z and u = -lambda of a step (Algorithm 1, before the loop): cold (zeros), warm
// from the previous step's lambda and z, or from the learned initial lambda (z from the
// previous step); y^0 = beta z^0 + u^0 and w^0 = beta z^0 - u^0.
template <typename T, typename Dist>
__device__ void init_duals(const StepParams &P, const SceneDesc &S, const View<T> &V, T *LAM,
                           T *Z, T *ZO, T *X, T *Y, T *YO, T *W0, const T *BT, bool learned,
                           const Dist &d)
{
    const double *lam = learned ? P.lam0 : P.lam;
    const bool warm = learned || P.warm_prev;
    for (int r = d.tid; r < S.nrow; r += d.nthreads) LAM[r] = warm ? (T)lam[S.row_g0 + r] : (T)0;
    for (int t = d.tid; t < S.nsr; t += d.nthreads) {
        if (V.mlen[t] == 0) continue;                 // padding side-row
        const T beta = BT[t];
        const T z = warm ? (T)P.z[S.sr_g0 + t] : (T)0;
        const T l = warm ? (T)lam[S.row_g0 + V.row[t]] : (T)0;
        Z[t] = z;
        ZO[t] = z;
        X[t] = (T)0;
        Y[t] = beta * z - l;
        YO[t] = Y[t];
        W0[t] = beta * z + l;
    }
    d.sync();
}

// One item of a Projected Jacobi iteration (the comparison solver of Sec. IV-B): the row's
// (or contact's) constraint value from the x of its sides, the relaxed Jacobi update of its
// impulse with 1/delta from INVS (soft rows: the soft law with x linearised in the row's own
// lambda; contacts: normal clamped at 0, tangents scaled onto the friction disk), w =
// lambda on every side for the next v-step, and the natural residual |d lambda| delta /
// omega, written as x - z of the first side-row (z = x on the others) so that the step's
// residuals report it; returns its bits
template <typename T, typename U>
__device__ __forceinline__ U pj_item(const Item &it, const int *ls, const T *X, const T *E,
                                     const T *INVS, const T *KF, const T *AL, const T *MU,
                                     T *LAM, T *Z, T *ZO, T *wn, T om, U mloc)
{
    const int nr = it.type == TYPE_CONTACT ? 3 : 1;
    T xr[3] = {(T)0, (T)0, (T)0}, lo[3], ln[3], id[3];
    for (int s = 0; s < it.ns; ++s)
        for (int r = 0; r < nr; ++r) xr[r] += X[ls[s] + r];
    for (int r = 0; r < nr; ++r) { lo[r] = LAM[it.row + r]; id[r] = INVS[it.row + r]; }
    if (it.type == TYPE_CONTACT) {
        T n = lo[0] - om * (xr[0] + E[it.row]) * id[0];
        n = n > (T)0 ? n : (T)0;
        T l1 = lo[1] - om * (xr[1] + E[it.row + 1]) * id[1];
        T l2 = lo[2] - om * (xr[2] + E[it.row + 2]) * id[2];
        const T lim = MU[it.row] * n, t2 = l1 * l1 + l2 * l2;
        if (t2 > lim * lim) { const T f = lim * rsq(t2); l1 *= f; l2 *= f; }
        ln[0] = n; ln[1] = l1; ln[2] = l2;
    } else if (it.type == TYPE_SOFT) {
        const T dl = (T)1 / id[0];
        const T ls_ = -KF[it.row] * (E[it.row] + AL[it.row] * (xr[0] - dl * lo[0]));
        ln[0] = lo[0] + om * (ls_ - lo[0]);
    } else {
        ln[0] = lo[0] - om * (xr[0] + E[it.row]) * id[0];
        if (it.type == TYPE_HARD) ln[0] = ln[0] > (T)0 ? ln[0] : (T)0;
    }
    for (int r = 0; r < nr; ++r) {
        LAM[it.row + r] = ln[r];
        const T res = fabs(ln[r] - lo[r]) / (om * id[r]);
        mloc = umax(mloc, rbits(res));
        for (int s = 0; s < it.ns; ++s) {
            const int t = ls[s] + r;
            const T zv = s == 0 ? X[t] - res : X[t];
            ZO[t] = zv;
            Z[t] = zv;
            wn[t] = ln[r];
        }
    }
    return mloc;
}

// One z-step item held in a thread's registers for a whole step (items with at most two
// sides): its type, row, side-rows and the step's constants.  KEEP_Z: the z of its
// side-rows (the item is their only writer) and the previous z stay in registers until
// published; otherwise they are read and written in memory each iteration (fewer
// registers).
template <typename T, bool KEEP_Z = true>
struct RegItem {
    using U = typename VecOf<T>::U;
    static constexpr int NZ = KEEP_Z ? 6 : 1;
    bool valid = false;
    int type = 0, row = 0, t0 = 0, t1 = -1, nr = 1;
    T ib0 = (T)0, ib1 = (T)0, e0 = (T)0, e1 = (T)0, e2 = (T)0;
    T is = (T)0, kf = (T)0, al = (T)0, mu = (T)0;
    T zr[NZ] = {(T)0};
    T zq[NZ] = {(T)0};

    __device__ __forceinline__ void load(const Item *items, const int *list, int i, const T *INVB,
                                         const T *E, const T *INVS, const T *KF, const T *AL,
                                         const T *MU, const T *Z)
    {
        const Item it = items[i];
        if (it.type < 0) return;
        valid = true;
        type = it.type;
        row = it.row;
        t0 = list[it.lo];
        t1 = it.ns > 1 ? list[it.lo + 1] : -1;
        nr = type == TYPE_CONTACT ? 3 : 1;
        ib0 = INVB[t0];
        if (t1 >= 0) ib1 = INVB[t1];
        e0 = E[row];
        if (nr == 3) { e1 = E[row + 1]; e2 = E[row + 2]; }
        is = INVS[row]; kf = KF[row]; al = AL[row]; mu = MU[row];
        if constexpr (KEEP_Z) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (r < nr) {
                    zr[r] = Z[t0 + r];
                    if (t1 >= 0) zr[3 + r] = Z[t1 + r];
                }
            }
#pragma unroll
            for (int r = 0; r < 6; ++r) zq[r] = zr[r];
        }
    }

    // z of side-row t (k: its slot), replaced by zn; returns the old z
    __device__ __forceinline__ T swap_z(T *Z, T *ZO, int t, int k, T zn)
    {
        if constexpr (KEEP_Z) {
            const T zo = zr[k];
            zq[k] = zo;
            zr[k] = zn;
            return zo;
        } else {
            const T zo = Z[t];
            ZO[t] = zo;
            Z[t] = zn;
            return zo;
        }
    }

    // the item's projection (Sec. III-C): lambda, z, w of the next v-step; returns the bits
    // of max(|x - z|, |dz|) over its side-rows
    __device__ __forceinline__ U project(const T *Y, const T *X, T *LAM, T *wn, T *Z, T *ZO)
    {
        U mloc = 0;
        if (!valid) return mloc;
        if (type == TYPE_CONTACT) {
            T ya[3], yb[3] = {(T)0, (T)0, (T)0};
#pragma unroll
            for (int r = 0; r < 3; ++r) ya[r] = Y[t0 + r];
            if (t1 >= 0) {
#pragma unroll
                for (int r = 0; r < 3; ++r) yb[r] = Y[t1 + r];
            }
            const T ln = -(ya[0] * ib0 + yb[0] * ib1 + e0) * is;
            const T l1 = -(ya[1] * ib0 + yb[1] * ib1 + e1) * is;
            const T l2 = -(ya[2] * ib0 + yb[2] * ib1 + e2) * is;
            T lv[3];
            if (ln <= (T)0) {
                lv[0] = lv[1] = lv[2] = (T)0;
            } else {
                const T t2 = l1 * l1 + l2 * l2;
                const T lim = mu * ln;
                lv[0] = ln;
                if (t2 > lim * lim) { const T f = lim * rsq(t2); lv[1] = l1 * f; lv[2] = l2 * f; }
                else { lv[1] = l1; lv[2] = l2; }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                LAM[row + r] = lv[r];
                const T zn = (ya[r] + lv[r]) * ib0;
                const T zo = swap_z(Z, ZO, t0 + r, r, zn);
                mloc = umax(mloc, umax(rbits(fabs(X[t0 + r] - zn)), rbits(fabs(zn - zo))));
                wn[t0 + r] = ya[r] + (T)2 * lv[r];
            }
            if (t1 >= 0) {
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const T zn = (yb[r] + lv[r]) * ib1;
                    const T zo = swap_z(Z, ZO, t1 + r, 3 + r, zn);
                    mloc = umax(mloc, umax(rbits(fabs(X[t1 + r] - zn)), rbits(fabs(zn - zo))));
                    wn[t1 + r] = yb[r] + (T)2 * lv[r];
                }
            }
        } else {
            const T y0 = Y[t0];
            const T y1 = t1 >= 0 ? Y[t1] : (T)0;
            const T q = y0 * ib0 + y1 * ib1;
            T lv;
            if (type == TYPE_SOFT) lv = -(e0 + al * q) * kf;
            else {
                lv = -(q + e0) * is;
                if (type == TYPE_HARD) lv = lv > (T)0 ? lv : (T)0;
            }
            LAM[row] = lv;
            const T zn0 = (y0 + lv) * ib0;
            const T zo0 = swap_z(Z, ZO, t0, 0, zn0);
            mloc = umax(mloc, umax(rbits(fabs(X[t0] - zn0)), rbits(fabs(zn0 - zo0))));
            wn[t0] = y0 + (T)2 * lv;
            if (t1 >= 0) {
                const T zn1 = (y1 + lv) * ib1;
                const T zo1 = swap_z(Z, ZO, t1, 3, zn1);
                mloc = umax(mloc, umax(rbits(fabs(X[t1] - zn1)), rbits(fabs(zn1 - zo1))));
                wn[t1] = y1 + (T)2 * lv;
            }
        }
        return mloc;
    }

    // lambda of the item (Sec. III-C) from the y of its side-rows, slot s * rows + r.  In
    // FP32 one instruction stream serves every type (a warp holds items of several types):
    // the first row is -(a q + e) s with (a, s) = (alpha, k) for soft rows and
    // (1, 1 / sum 1/beta) otherwise, clamped at 0 for hard and contact rows; contact rows 1, 2
    // are then scaled into the friction cone.  In FP64, where every instruction is costly,
    // each type runs only its own formula.
    __device__ __forceinline__ void lambda_of(const T *ys, T *lv) const
    {
        const bool two = t1 >= 0, con = nr == 3;
        if constexpr (sizeof(T) == 4) {
            const T yb0 = two ? (con ? ys[3] : ys[1]) : (T)0;
            const T q0 = ys[0] * ib0 + yb0 * ib1;
            const T a0 = type == TYPE_SOFT ? al : (T)1;
            const T s0 = type == TYPE_SOFT ? kf : is;
            T l0 = -(q0 * a0 + e0) * s0;
            if (type == TYPE_HARD || con) l0 = l0 > (T)0 ? l0 : (T)0;
            const T yb1 = two ? ys[4] : (T)0, yb2 = two ? ys[5] : (T)0;
            const T l1 = -(ys[1] * ib0 + yb1 * ib1 + e1) * is;
            const T l2 = -(ys[2] * ib0 + yb2 * ib1 + e2) * is;
            const T t2 = l1 * l1 + l2 * l2;
            const T lim = mu * l0;
            const T f = t2 > lim * lim ? lim * rsq(t2) : (T)1;
            const bool on = valid && con && l0 > (T)0;
            lv[0] = valid ? l0 : (T)0;
            lv[1] = on ? l1 * f : (T)0;
            lv[2] = on ? l2 * f : (T)0;
        } else {
            lv[0] = lv[1] = lv[2] = (T)0;
            if (!valid) return;
            if (con) {
                const T yb0 = two ? ys[3] : (T)0, yb1 = two ? ys[4] : (T)0, yb2 = two ? ys[5] : (T)0;
                const T ln = -(ys[0] * ib0 + yb0 * ib1 + e0) * is;
                if (ln > (T)0) {
                    const T l1 = -(ys[1] * ib0 + yb1 * ib1 + e1) * is;
                    const T l2 = -(ys[2] * ib0 + yb2 * ib1 + e2) * is;
                    const T t2 = l1 * l1 + l2 * l2;
                    const T lim = mu * ln;
                    lv[0] = ln;
                    if (t2 > lim * lim) { const T f = lim * rsq(t2); lv[1] = l1 * f; lv[2] = l2 * f; }
                    else { lv[1] = l1; lv[2] = l2; }
                }
            } else {
                const T q = ys[0] * ib0 + (two ? ys[1] : (T)0) * ib1;
                T l;
                if (type == TYPE_SOFT) l = -(e0 + al * q) * kf;
                else {
                    l = -(q + e0) * is;
                    if (type == TYPE_HARD) l = l > (T)0 ? l : (T)0;
                }
                lv[0] = l;
            }
        }
    }

    // write the z (and the previous z) held in registers back to the scene arrays
    __device__ __forceinline__ void publish(T *Z, T *ZO) const
    {
        if constexpr (KEEP_Z) {
            if (!valid) return;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (r < nr) {
                    Z[t0 + r] = zr[r]; ZO[t0 + r] = zq[r];
                    if (t1 >= 0) { Z[t1 + r] = zr[3 + r]; ZO[t1 + r] = zq[3 + r]; }
                }
            }
        }
    }
};

// NT threads per block: SUBADMM_THREADS, or SUBADMM_WIDE for a generic variant of a class
// whose scenes take a whole SM's shared memory (one block per SM), which then uses the whole
// register file and twice the warps per scene
template <typename T, int SPLIT, bool CACHED, int NT = SUBADMM_THREADS>
__global__ void __launch_bounds__(NT, (CACHED || NT > SUBADMM_THREADS) ? 1 : 2) step_kernel(StepParams P)
{
    static_assert(!CACHED || NT == SUBADMM_THREADS, "the register-cached map is laid out for 256 threads");
    constexpr int NW = NT / 32;
    using VT = typename VecOf<T>::V;
    using U = typename VecOf<T>::U;
    constexpr int VN = VecOf<T>::N;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[4][SUBADMM_MAXWARPS];
    __shared__ U ured[2][NW];
    __shared__ T tred[2][NW];
    __shared__ int s_status;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr bool MIXED = sizeof(T) == 4;

    for (int k = blockIdx.x; k < P.nscenes; k += gridDim.x) {
        const int sc = P.scene_ids[k];
        const SceneDesc S = P.scenes[sc];
        const View<T> V = scene_view<T>(P, S, smraw);
        T *X = V.tb + S.ot_x, *Y = V.tb + S.ot_y, *Z = V.tb + S.ot_z, *LAM = V.tb + S.ot_lam;
        T *YO = V.tb + S.ot_yo, *ZO = V.tb + S.ot_zo;
        T *E = V.tb + S.ot_e, *INVB = V.tb + S.ot_invb, *BT = V.tb + S.ot_b;
        T *INVS = V.tb + S.ot_invs, *KF = V.tb + S.ot_kf, *AL = V.tb + S.ot_al;
        T *MU = V.tb + S.ot_mu;
        T *const W0 = V.tb + S.ot_w0, *const W1 = V.tb + S.ot_w1;
        // per-side-row arrays start zero (padding side-rows between subsystems stay zero)
        for (int q = tid; q < S.ot_lam - S.ot_x; q += blockDim.x) V.tb[S.ot_x + q] = (T)0;
        scene_tables<T>(P, S, V, BlockDist());
        __syncthreads();

        for (int step = 0; step < P.n_steps; ++step) {
            if (tid == 0) s_status = ST_OK;
            __syncthreads();
            PhaseClock pc(P.phase ? P.phase + 8 * sc : nullptr);
            pc.mark_at(PHASE_ASSEMBLE, block_setup<T>(P, S, V, &s_status, step));
            pc.mark(PHASE_FACTOR);
            const int status0 = s_status;
            if (status0 != ST_OK) {
                // K_i not SPD: report, leave the state untouched (the step is undefined)
                if (tid == 0) {
                    double *o = P.res + 6 * sc;
                    o[0] = o[1] = o[2] = __longlong_as_double(0x7ff8000000000000LL);
                    o[3] = 0.0; o[4] = 0.0; o[5] = (double)status0;
                }
                __syncthreads();
                continue;
            }
            // initial z, u = -lambda; a learned start (the launch's first step) is checked
            // after 10 iterations against the plain start's residual there, and replaced by
            // the plain start if worse
            const bool learned_mode = P.lam0 != nullptr && step == 0;
            const int skip0 = learned_mode ? P.learn_skip[2 * sc] : 0;
            bool learned = learned_mode && skip0 == 0;
            const unsigned long long ref10 = learned_mode ? P.ref10[sc] : 0ull;
            int wasted = 0, fallbacks = 0;
            __syncthreads();
            if (learned_mode && tid == 0 && skip0 > 0) P.learn_skip[2 * sc] = skip0 - 1;
            init_duals<T>(P, S, V, LAM, Z, ZO, X, Y, YO, W0, BT, learned, BlockDist());

            // ---- per-thread state of the register-cached iteration (CACHED).  The host's
            // thread map gives each thread a side-row (its lane group of SPLIT lanes) and puts
            // every projection item's side-rows on adjacent groups of one warp.  A thread keeps
            // its side-row's D chunks, c, beta, 1/beta, x, y, z and lambda in registers and the
            // constants of its item: the warp forms the items' y, and every lane of an item
            // projects it (Sec. III-C) from y gathered by shuffles, so an iteration needs one
            // block barrier (the new w) instead of two.
            constexpr int MAXC = CachedChunks<T>::value;   // D chunks a lane keeps in registers
            constexpr int FSI = SPLIT == 4 ? 2 : SPLIT == 2 ? 1 : 0;
            const int xg = tid / SPLIT;
            int xt = -1, xgl = tid - xg * SPLIT, flead = 0, fslot = 0, fitem = 0;
            if (CACHED) {
                const int2 fm = reinterpret_cast<const int2 *>(P.ipool + S.fmap_off[FSI])[tid];
                xt = fm.x;
                flead = fm.y & 31;
                fslot = (fm.y >> 5) & 7;
                xgl = (fm.y >> 8) & 7;
                fitem = fm.y >> 11;
            }
            VT dreg[MAXC];
            bool xv = false;
            int xwbo = 0, xnv = 0, xrow = 0, fr = 0;
            T xc = (T)0, xbt = (T)0, xib = (T)0, xx = (T)0, yreg = (T)0, yprev = (T)0;
            T zreg = (T)0, zprev = (T)0, lreg = (T)0;
            RegItem<T, false> ri;
            auto load_cache = [&]() {
                if (CACHED) {
#pragma unroll
                    for (int q = 0; q < MAXC; ++q) dreg[q] = VecZero<T>::get();
                    xv = xt >= 0 && V.mlen[xt] > 0;
                    if (xv) {
                        xwbo = V.wbase[xt];
                        xnv = (V.mlen[xt] + VN - 1) / VN;
                        xrow = V.row[xt];
                        xc = V.htb[V.coff[xt]];
                        xbt = BT[xt];
                        xib = INVB[xt];
                        xx = X[xt];
                        yreg = Y[xt];
                        yprev = yreg;
                        zreg = Z[xt];
                        zprev = zreg;
                        lreg = LAM[xrow];
                        const VT *Dr = reinterpret_cast<const VT *>(V.htb + V.drow[xt]);
#pragma unroll
                        for (int q = 0; q < MAXC; ++q)
                            if (xgl + q * SPLIT < xnv) dreg[q] = Dr[xgl + q * SPLIT];
                    }
                    ri = RegItem<T, false>();
                    if (xt >= 0) ri.load(V.item, V.list, fitem, INVB, E, INVS, KF, AL, MU, Z);
                    fr = ri.nr == 3 ? fslot % 3 : 0;
                }
            };
            load_cache();

            int par = 0, last_par = 0, iters = 0, conv = 0, status = ST_OK;
            bool restart = false;
            double th = 0.0;
            double tolc = P.tol;
            U tolb = tol_bits(T(0), tolc > 0.0 ? tolc : 0.0);
            const bool primal_stop = !P.stop_theta && P.tol > 0.0;
            // the loop holds no FP64 instruction in the mixed form, not even a predicated one
            // (an FP64 warp instruction issues for ~64 cycles on GB300 whatever its predicate)
            const T theta_thT = (T)P.theta_th;
            int l = 0;
            pc.mark(PHASE_ASSEMBLE);
            for (;;) {
                for (; l < P.max_iters; ++l) {
                    // ---- v-step through the affine map x = c + D w; y = beta x - lambda
                    const T *w = par ? W1 : W0;
                    T tpart = (T)0;
                    T *wn = par ? W0 : W1;
                    U mfused = 0;
                    if (CACHED) {
                        // x = c + D w of this side-row over its lane group
                        T acc = (T)0;
                        if (xv) {
                            const VT *wb = reinterpret_cast<const VT *>(w + xwbo);
                            T a1 = (T)0;
#pragma unroll
                            for (int q = 0; q < MAXC; ++q) {
                                if (xgl + q * SPLIT < xnv) {
                                    const VT wq = wb[xgl + q * SPLIT];
                                    if (q & 1) a1 = vdot(dreg[q], wq, a1);
                                    else acc = vdot(dreg[q], wq, acc);
                                }
                            }
                            acc += a1;
                        }
#pragma unroll
                        for (int o = SPLIT / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        const T xn = acc + xc;
                        const T yn = xbt * xn - lreg;
                        // the item's y (slot k on the group at lane flead + k SPLIT), its lambda,
                        // then z, w and the residual of this side-row
                        T ys[6], lv[3];
#pragma unroll
                        for (int k = 0; k < 6; ++k) ys[k] = __shfl_sync(0xffffffffu, yn, (flead + k * SPLIT) & 31);
                        ri.lambda_of(ys, lv);
                        const T ln = fr == 0 ? lv[0] : fr == 1 ? lv[1] : lv[2];
                        if (xv) {
                            const T zn = (yn + ln) * xib;
                            if (xgl == 0) {
                                mfused = umax(rbits(fabs(xn - zn)), rbits(fabs(zn - zreg)));
                                wn[xt] = yn + (T)2 * ln;
                            }
                            zprev = zreg;
                            zreg = zn;
                            yprev = yreg;
                            yreg = yn;
                            xx = xn;
                            lreg = ln;
                        }
                    } else {
                        // two side-rows per trip, two accumulators per row: independent
                        // load and FMA chains overlap
                        constexpr int groups = NT / SPLIT;
                        const int trips = (S.nsr + groups - 1) / groups;
                        for (int k = 0; k < trips; k += 2) {
                            int tt[2], mm[2];
                            T acc[2];
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                tt[h] = xg + (k + h) * groups;
                                mm[h] = (k + h < trips && tt[h] < S.nsr) ? V.mlen[tt[h]] : 0;
                                T a0 = (T)0, a1 = (T)0;
                                if (mm[h] > 0) {
                                    const VT *Dr = reinterpret_cast<const VT *>(V.htb + V.drow[tt[h]]);
                                    const VT *wb = reinterpret_cast<const VT *>(w + V.wbase[tt[h]]);
                                    const int nv = (mm[h] + VN - 1) / VN;
                                    int c = xgl;
                                    for (; c + SPLIT < nv; c += 2 * SPLIT) {
                                        a0 = vdot(Dr[c], wb[c], a0);
                                        a1 = vdot(Dr[c + SPLIT], wb[c + SPLIT], a1);
                                    }
                                    if (c < nv) a0 = vdot(Dr[c], wb[c], a0);
                                }
                                acc[h] = a0 + a1;
                            }
#pragma unroll
                            for (int o = SPLIT / 2; o; o >>= 1) {
                                acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
                                acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
                            }
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int t = tt[h];
                                if (mm[h] > 0 && xgl == 0) {
                                    const T a = acc[h] + V.htb[V.coff[t]];
                                    const T ynew = BT[t] * a - LAM[V.row[t]];
                                    if (P.stop_theta) {
                                        const T d = ynew - Y[t];
                                        tpart += d * d;
                                    }
                                    YO[t] = Y[t];
                                    Y[t] = ynew;
                                    X[t] = a;
                                }
                            }
                        }
                    }
                    if (!CACHED) {
                        if (P.stop_theta) {
#pragma unroll
                            for (int o = 16; o; o >>= 1) tpart += __shfl_xor_sync(0xffffffffu, tpart, o);
                            if (lane == 0) tred[l & 1][warp] = tpart;
                        }
                        __syncthreads();
                    }
                    pc.mark(PHASE_VSTEP);
                    last_par = par;
                    iters = l + 1;
                    if (!CACHED && P.stop_theta) {
                        T ths = (T)0;
                        for (int q = 0; q < NW; ++q) ths += tred[l & 1][q];
                        if (l >= 1 && ths < theta_thT) { th = (double)ths; conv = 1; break; }
                    }
                    // ---- z-step (Sec. III-C); u = -lambda; max(|x - z|, |dz|) as bits
                    U mloc = 0;
                    if (CACHED) {
                        mloc = mfused;
                    } else {
                        for (int i = tid; i < S.nitem; i += NT) {
                            const Item it = V.item[i];
                            if (it.type < 0) continue;
                            const int *ls = V.list + it.lo;
                            if (P.pj) {
                                mloc = pj_item<T, U>(it, ls, X, E, INVS, KF, AL, MU, LAM, Z, ZO,
                                                     wn, (T)P.pj_omega, mloc);
                                continue;
                            }
                            if (it.type == TYPE_CONTACT) {
                                T q0 = (T)0, q1 = (T)0, q2 = (T)0;
                                for (int s = 0; s < it.ns; ++s) {
                                    const int t = ls[s];
                                    const T ib = INVB[t];
                                    q0 += Y[t] * ib; q1 += Y[t + 1] * ib; q2 += Y[t + 2] * ib;
                                }
                                const T is = INVS[it.row];
                                const T ln = -(q0 + E[it.row]) * is;
                                const T l1 = -(q1 + E[it.row + 1]) * is;
                                const T l2 = -(q2 + E[it.row + 2]) * is;
                                T lv[3];
                                if (ln <= (T)0) {
                                    lv[0] = lv[1] = lv[2] = (T)0;
                                } else {
                                    const T t2 = l1 * l1 + l2 * l2;
                                    const T lim = MU[it.row] * ln;
                                    lv[0] = ln;
                                    if (t2 > lim * lim) { const T f = lim * rsq(t2); lv[1] = l1 * f; lv[2] = l2 * f; }
                                    else { lv[1] = l1; lv[2] = l2; }
                                }
                                LAM[it.row] = lv[0]; LAM[it.row + 1] = lv[1]; LAM[it.row + 2] = lv[2];
                                for (int s = 0; s < it.ns; ++s) {
#pragma unroll
                                    for (int r = 0; r < 3; ++r) {
                                        const int t = ls[s] + r;
                                        const T yv = Y[t], zo = Z[t];
                                        const T zn = (yv + lv[r]) * INVB[t];
                                        mloc = umax(mloc, umax(rbits(fabs(X[t] - zn)), rbits(fabs(zn - zo))));
                                        ZO[t] = zo;
                                        Z[t] = zn;
                                        wn[t] = yv + (T)2 * lv[r];
                                    }
                                }
                            } else {
                                T q = (T)0;
                                for (int s = 0; s < it.ns; ++s) q += Y[ls[s]] * INVB[ls[s]];
                                const T e = E[it.row];
                                T lv;
                                if (it.type == TYPE_EQUALITY) lv = -(q + e) * INVS[it.row];
                                else if (it.type == TYPE_HARD) { lv = -(q + e) * INVS[it.row]; lv = lv > (T)0 ? lv : (T)0; }
                                else lv = -(e + AL[it.row] * q) * KF[it.row];
                                LAM[it.row] = lv;
                                for (int s = 0; s < it.ns; ++s) {
                                    const int t = ls[s];
                                    const T yv = Y[t], zo = Z[t];
                                    const T zn = (yv + lv) * INVB[t];
                                    mloc = umax(mloc, umax(rbits(fabs(X[t] - zn)), rbits(fabs(zn - zo))));
                                    ZO[t] = zo;
                                    Z[t] = zn;
                                    wn[t] = yv + (T)2 * lv;
                                }
                            }
                        }
                    }
                    if (!(learned_mode && l == 9)) {
                        // the stop test rides on the barrier: the number of threads whose
                        // residual is finite and above the tolerance.  A non-finite iterate
                        // stays non-finite (c is fixed for the step and w carries it to every
                        // coupled side-row), so the count drops to 0 or the limit ends the
                        // loop, and the step's FP64 residuals below report it
                        const int over = __syncthreads_count(primal_stop && mloc > tolb &&
                                                             mloc < inf_bits(T(0)));
                        par ^= 1;
                        pc.mark(PHASE_ZSTEP);
                        if (primal_stop && over == 0) { conv = 1; break; }
                        continue;
                    }
                    mloc = warp_umax(mloc);
                    if (lane == 0) ured[l & 1][warp] = mloc;
                    __syncthreads();
                    U mx = 0;
#pragma unroll
                    for (int q = 0; q < NW; ++q) mx = umax(mx, ured[l & 1][q]);
                    par ^= 1;
                    pc.mark(PHASE_ZSTEP);
                    {
                        if (learned && (unsigned long long)mx > ref10) { restart = true; break; }
                        if (!learned && tid == 0) P.ref10[sc] = (unsigned long long)mx;
                        if (learned && tid == 0) P.learn_skip[2 * sc + 1] = 0;   // kept: streak ends
                    }
                    if (mx >= inf_bits(T(0))) { status = ST_NAN; break; }
                    if (primal_stop && mx <= tolb) { conv = 1; break; }
                }
                if (restart) {
                    // the learned start trails the plain one after 10 iterations: restart the
                    // step from the plain start, and start plain for the next 2^streak - 1 steps
                    if (tid == 0) {
                        const int streak = min(P.learn_skip[2 * sc + 1] + 1, 5);
                        P.learn_skip[2 * sc + 1] = streak;
                        P.learn_skip[2 * sc] = (1 << streak) - 1;
                    }
                    restart = false;
                    learned = false;
                    ++fallbacks;
                    wasted += l + 1;
                    init_duals<T>(P, S, V, LAM, Z, ZO, X, Y, YO, W0, BT, false, BlockDist());
                    load_cache();
                    par = 0;
                    l = 0;
                    continue;
                }
                // the register-cached iterate: publish x, y, z, lambda (and the previous y, z)
                if (CACHED && xv && xgl == 0) {
                    X[xt] = xx;
                    Y[xt] = yreg;
                    YO[xt] = yprev;
                    Z[xt] = zreg;
                    ZO[xt] = zprev;
                    LAM[xrow] = lreg;
                }
                __syncthreads();
                // v-hat from the last v-step's w (ADMM), or from the last z-step's lambda
                // (Projected Jacobi: v-hat = A^-1 (b + J^T lambda) with the reported impulses)
                block_recover<T>(P, S, V, (P.pj ? par : last_par) ? W1 : W0);
                __syncthreads();
                if (MIXED && conv && primal_stop && status == ST_OK) {
                    // FP64 primal residual max |J v - z|; on a miss, refine c by the FP64 - FP32
                    // difference of x at this iterate and resume
                    double part = 0.0;
                    for (int t = tid; t < S.nsr; t += blockDim.x) {
                        if (V.mlen[t] == 0) continue;
                        const SubDesc &u = P.subs[S.sub0 + V.sub[t]];
                        const int lr = t - u.sr0, n = u.n;
                        const double *Jr = V.sdb + u.od_J + lr * n;
                        const double *v = V.sdb + u.od_v;
                        const int *jl = P.ipool + u.env_off + 2 * n;
                        double x = 0.0;
                        for (int p = jl[lr]; p < jl[u.m + lr]; ++p) x += Jr[p] * v[p];
                        part = nanmax(part, fabs(x - (double)Z[t]));
                        V.htb[V.coff[t]] += (T)(x - (double)X[t]);
                    }
                    double d0 = 0.0, d2 = 0.0;
                    block_reduce3(red, d0, part, d2);
                    if (part > P.tol && l + 1 < P.max_iters) {
                        tolc *= 0.5;
                        tolb = tol_bits(T(0), tolc);
                        if (CACHED && xv) xc = V.htb[V.coff[xt]];
                        conv = 0;
                        ++l;
                        continue;
                    }
                    if (part > P.tol) conv = 0;
                }
                break;
            }
            // reported residuals of the last iteration: theta, r_p = max|x - z|,
            // r_d = max beta |z^{l+1} - z^l|
            double rp, rd;
            {
                double tp = 0.0, pp = 0.0, dd = 0.0;
                for (int t = tid; t < S.nsr; t += blockDim.x) {
                    if (V.mlen[t] == 0) continue;
                    const double dy = (double)Y[t] - (double)YO[t];
                    tp += dy * dy;
                    pp = nanmax(pp, fabs((double)X[t] - (double)Z[t]));
                    dd = nanmax(dd, (double)BT[t] * fabs((double)Z[t] - (double)ZO[t]));
                }
                block_reduce3(red, tp, pp, dd);
                if (!P.stop_theta) th = tp;
                rp = pp;
                rd = dd;
            }
            // a non-finite iterate (the loop itself does not stop on one)
            if (status == ST_OK && !(isfinite(rp) && isfinite(rd))) { status = ST_NAN; conv = 0; }
            pc.mark(PHASE_EXIT);
            // v-hat out and state update of rigid bodies (Algorithm 1, after the loop)
            for (int i = warp; i < S.nsub; i += NW) {
                const SubDesc &u = P.subs[S.sub0 + i];
                const double *v = V.sdb + u.od_v;
                for (int p = lane; p < u.n; p += 32) P.vhat[u.v_off + p] = v[p];
                if (u.kind == KIND_LINEAR) {
                    double *nd = P.nodes + (size_t)u.body0 * SUBADMM_NODE;
                    for (int p = lane; p < u.n; p += 32) {
                        nd[(p / 3) * SUBADMM_NODE + p % 3] += P.h * v[p];
                        double &vel = nd[(p / 3) * SUBADMM_NODE + 3 + p % 3];
                        vel = 2.0 * v[p] - vel;
                    }
                    continue;
                }
                if (u.kind != KIND_RIGID) continue;
                for (int k = lane; k < u.nb; k += 32)
                    body_update(P.bodies + (size_t)(u.body0 + k) * SUBADMM_BODY, v + 6 * k, P.h);
            }
            __syncthreads();
            pc.mark(PHASE_RECOVER);
            pc.flush(iters);
            // warm-start state and reports
            for (int r = tid; r < S.nrow; r += blockDim.x) P.lam[S.row_g0 + r] = (double)LAM[r];
            for (int t = tid; t < S.nsr; t += blockDim.x) P.z[S.sr_g0 + t] = (double)Z[t];
            if (tid == 0) {
                double *o = P.res + 6 * sc;
                o[0] = rp; o[1] = rd; o[2] = th; o[3] = (double)iters; o[4] = (double)conv;
                o[5] = (double)status;
                long long *st = P.stats + 5 * sc;
                st[0] += iters + wasted;
                if (iters + wasted > st[1]) st[1] = iters + wasted;
                st[2] += conv ? 0 : 1;
                st[3] += 1;
                st[4] += fallbacks;
            }
            __syncthreads();
        }
    }
}

}  // namespace subadmm
