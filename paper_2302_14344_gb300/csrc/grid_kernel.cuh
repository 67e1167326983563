// One scene over the whole GPU: the inner ADMM loop of Algorithm 1 for a scene too large
// for one block (a cooperative launch, all blocks resident).  The scene's per-row arrays
// and tables live in global memory, laid out as the block kernel lays them out in shared
// memory; every loop of the step is spread over all threads (side-rows, rows, items) or
// warps (subsystems) of the grid.  Two grid barriers per iteration: after the v-step (the
// z-step reads y of any subsystem) and after the z-step (the next v-step reads w of any
// constraint, and the iteration's residual maximum, gathered by atomics, decides the stop).
#pragma once

#include "step_kernel.cuh"

namespace subadmm {

// bit pattern of a non-negative double: orders like the value (NaN above infinity)
__device__ __forceinline__ unsigned long long dbits(double x)
{
    return (unsigned long long)__double_as_longlong(x);
}

template <typename F>
__device__ __forceinline__ F vload(const F *p)
{
    return *reinterpret_cast<const volatile F *>(p);
}

// ---- bulk asynchronous copies global -> shared with an mbarrier transaction count
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// generic-proxy writes (D of this step) made visible to later bulk copies of this thread
__device__ __forceinline__ void proxy_fence_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// one arrival that also expects `bytes`, then the copy of `bytes` (a multiple of 16, both
// addresses 16-byte aligned) that completes them
__device__ __forceinline__ void bulk_row_load(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// wait for the phase `parity` of the barrier to complete; false after limit_ns
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// After a stage's copy missed its wait: wait once more, bounded, for every copy the warp
// still has in flight (bit s of *pend: stage s's copy was issued and not yet waited for), so
// that no bulk copy lands in the block's shared memory after the block stops expecting it.
// Stages whose copy completes are cleared from *pend (their parity advances); a copy that
// never completes stays in *pend, and the caller no longer uses the stage buffers at all.
__device__ __forceinline__ void drain_stages(unsigned long long *bars, unsigned *pend,
                                             unsigned *ph, int nst)
{
    for (int s = 0; s < nst; ++s) {
        if (!((*pend >> s) & 1u)) continue;
        const bool got = __all_sync(0xffffffffu, mbar_wait(&bars[s], (*ph >> s) & 1u, 2000000000ull));
        if (got) {
            *ph ^= 1u << s;
            *pend &= ~(1u << s);
        }
    }
}

template <typename T, int SPLIT>
__global__ void __launch_bounds__(SUBADMM_THREADS, 2) grid_step_kernel(StepParams P)
{
    using VT = typename VecOf<T>::V;
    using U = typename VecOf<T>::U;
    constexpr int VN = VecOf<T>::N;
    constexpr bool MIXED = sizeof(T) == 4;
    GridScratch *G = P.grid;
    const GridDist d(&G->count, &G->gen, &G->err);
    const int lane = threadIdx.x & 31;
    const bool lead = d.tid == 0;
    const int sc = P.scene_ids[0];
    const SceneDesc S = P.scenes[sc];
    unsigned char *raw = reinterpret_cast<unsigned char *>(P.work) + S.g_scene;
    const View<T> V = scene_view<T>(P, S, raw);
    T *X = V.tb + S.ot_x, *Y = V.tb + S.ot_y, *Z = V.tb + S.ot_z, *LAM = V.tb + S.ot_lam;
    T *YO = V.tb + S.ot_yo, *ZO = V.tb + S.ot_zo;
    T *E = V.tb + S.ot_e, *INVB = V.tb + S.ot_invb, *BT = V.tb + S.ot_b;
    T *INVS = V.tb + S.ot_invs, *KF = V.tb + S.ot_kf, *AL = V.tb + S.ot_al;
    T *MU = V.tb + S.ot_mu;
    T *const W0 = V.tb + S.ot_w0, *const W1 = V.tb + S.ot_w1;
    // staged D rows: grid_nstage row buffers per warp (dynamic shared memory), each with an
    // mbarrier that completes when its bulk copy has landed
    extern __shared__ __align__(128) unsigned char stage_raw[];
    __shared__ __align__(8) unsigned long long stage_bar[SUBADMM_WARPS][4];
    // per-warp partials of the iteration's reductions: a block combines its warps' values
    // and adds one atomic to the grid-wide slot (one per block rather than one per warp:
    // atomics on one address serialise at its L2 slice)
    __shared__ unsigned long long s_umax[SUBADMM_WARPS];
    __shared__ double s_theta[SUBADMM_WARPS];
    const int wl = threadIdx.x >> 5;
    const int nst = P.grid_nstage;
    if (P.grid_stage > 0 && lane == 0) {
        for (int k = 0; k < nst; ++k) mbar_init(&stage_bar[wl][k], 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned ph = 0;            // parity of the next completion of each stage's barrier
    unsigned pend = 0;          // stages whose issued copy has not been waited for yet
    bool stage_ok = true;       // false after a copy that did not complete in time
    // tc_phase 2 continues the step that a tc_phase 1 launch set up (its per-side-row
    // constants and status are kept; the Gram kernel formed D and c in between); tc_phase 3,
    // between the two, solves W for the subsystems that the blocked tensor-core
    // factorisation factorised after tc_phase 1
    const int tc_phase = P.tc_phase;
    const bool fresh = tc_phase == 0 || tc_phase == 1;     // a launch that starts the step
    if (fresh)
        for (int q = d.tid; q < S.ot_lam - S.ot_x; q += d.nthreads) V.tb[S.ot_x + q] = (T)0;
    scene_tables<T>(P, S, V, d);
    d.sync();

    for (int step = 0; step < P.n_steps; ++step) {
        if (lead) {
            if (fresh) G->status = ST_OK;
            G->tsum = 0.0;
            G->pmax = 0ull;
            G->dmax = 0ull;
            for (int k = 0; k < 3; ++k) { G->umax[k] = 0ull; G->theta[k] = 0.0; }
        }
        d.sync();
        PhaseClock pc((P.phase && blockIdx.x == 0) ? P.phase + 8 * sc : nullptr);
        if (fresh) pc.mark_at(PHASE_ASSEMBLE, scene_setup<T>(P, S, V, &G->status, step, d));
        if (tc_phase == 3) {
            w_chunks<T>(P, S, V, &G->status, d, 4);
            d.sync();
        }
        pc.mark(PHASE_FACTOR);
        const int status0 = vload(&G->status);
        if (status0 != ST_OK) {
            if (lead && tc_phase != 2) {
                double *o = P.res + 6 * sc;
                o[0] = o[1] = o[2] = __longlong_as_double(0x7ff8000000000000LL);
                o[3] = 0.0; o[4] = 0.0; o[5] = (double)status0;
            }
            d.sync();
            continue;
        }
        if (tc_phase == 1 || tc_phase == 3) {
            d.sync();
            pc.flush(0, 0);         // the setup's cycles; the iteration launch counts the step
            continue;
        }
        // z-step items in registers for the whole step when the scene has at most one item
        // per thread (an item's tables are constant within a step): each iteration then loads
        // only its y, x and z, in one round trip, instead of a chain of table loads; items of
        // more than two sides stay on the generic path
        // Items go by the block-interleaved warp numbering (item group g of 32, one type each,
        // to warp g, i.e. warp g / blocks of block g % blocks), so that a scene with few
        // items spreads them over the SMs rather than filling the first blocks.
        const int ix = 32 * d.warp + lane;
        const bool icache = S.nitem <= d.nthreads && !P.pj;
        RegItem<T, false> ri;
        bool igeneric = false;
        if (icache && ix < S.nitem) {
            const Item it = V.item[ix];
            if (it.ns <= 2) ri.load(V.item, V.list, ix, INVB, E, INVS, KF, AL, MU, Z);
            else igeneric = it.type >= 0;
        }
        // initial z, u = -lambda; a learned start is checked after 10 iterations against the
        // plain start's residual there, and replaced by the plain start if worse
        const bool learned_mode = P.lam0 != nullptr && step == 0;    // the launch's first step
        const int skip0 = learned_mode ? vload(&P.learn_skip[2 * sc]) : 0;
        bool learned = learned_mode && skip0 == 0;
        const unsigned long long ref10 = learned_mode ? vload(&P.ref10[sc]) : 0ull;
        int wasted = 0, fallbacks = 0;
        d.sync();
        if (learned_mode && lead && skip0 > 0) P.learn_skip[2 * sc] = skip0 - 1;
        init_duals<T>(P, S, V, LAM, Z, ZO, X, Y, YO, W0, BT, learned, d);
        pc.mark(PHASE_ASSEMBLE);

        constexpr int groups_per_block = SUBADMM_THREADS / SPLIT;
        const int groups = gridDim.x * groups_per_block;
        const int xg = d.tid / SPLIT, xgl = d.tid - xg * SPLIT;
        const int trips = (S.nsr + groups - 1) / groups;
        // warp per side-row (SPLIT 32) with at most 32 rows per warp: lane k keeps the tables
        // of the warp's k-th row for the whole step (no dependent table loads per iteration)
        const bool rowcache = SPLIT == 32 && trips <= 32;
        int r_len = 0, r_drow = 0, r_wb = 0, r_coff = 0, r_row = 0;
        T r_bt = (T)0;
        if (rowcache && lane < trips) {
            const int t = xg + lane * groups;
            if (t < S.nsr) {
                r_len = V.mlen[t]; r_drow = V.drow[t]; r_wb = V.wbase[t]; r_coff = V.coff[t];
                r_row = V.row[t]; r_bt = BT[t];
            }
        }
        // staged rows: every row of the warp starts 16-byte aligned and fits a stage
        unsigned char *const stg = stage_raw + (size_t)wl * nst * (size_t)P.grid_stage;
        bool staged = false;
        if (P.grid_stage > 0 && rowcache && stage_ok) {
            const bool fits = r_len == 0 ||
                              (((size_t)(V.htb + r_drow) & 15) == 0 &&
                               (r_len + VN - 1) / VN * 16 <= P.grid_stage);
            staged = __all_sync(0xffffffffu, fits);
            if (staged && lane == 0) proxy_fence_global();   // D of this step's setup
        }
        int par = 0, last_par = 0, iters = 0, conv = 0, status = ST_OK;
        bool restart = false;
        double th = 0.0;
        double tolc = P.tol;
        U tolb = tol_bits(T(0), tolc > 0.0 ? tolc : 0.0);
        const bool primal_stop = !P.stop_theta && P.tol > 0.0;
        const T theta_thT = (T)P.theta_th;
        int l = 0;
        for (;;) {
            for (; l < P.max_iters; ++l) {
                // ---- v-step through the affine map x = c + D w; y = beta x - lambda
                const T *w = par ? W1 : W0;
                T tpart = (T)0;
                constexpr int CH = VN == 4 ? 6 : 8;     // chunks per lane per pass
                if (staged) {
                    // warp per row, the warp's rows in order through nst shared-memory stages:
                    // row k + nst is copied into row k's stage once the warp has read it, so
                    // nst - 1 copies are in flight while a row is used
                    T own_c = (T)0, own_lam = (T)0, own_y = (T)0;
                    if (r_len > 0) {
                        own_c = V.htb[r_coff];
                        own_lam = LAM[r_row];
                        own_y = Y[xg + lane * groups];
                    }
                    for (int k = 0; k < nst && k < trips; ++k) {
                        const int len = __shfl_sync(0xffffffffu, r_len, k);
                        const int drow = __shfl_sync(0xffffffffu, r_drow, k);
                        if (lane == 0 && len > 0)
                            bulk_row_load(stg + (size_t)k * P.grid_stage, V.htb + drow,
                                          (unsigned)((len + VN - 1) / VN * 16), &stage_bar[wl][k]);
                        if (len > 0) pend |= 1u << k;
                    }
                    for (int k = 0; k < trips; ++k) {
                        const int s = k % nst;
                        const int len = __shfl_sync(0xffffffffu, r_len, k);
                        const int wbk = __shfl_sync(0xffffffffu, r_wb, k);
                        T acc = (T)0;
                        if (len > 0 && staged) {
                            const bool got = __all_sync(0xffffffffu,
                                                        mbar_wait(&stage_bar[wl][s], (ph >> s) & 1u, 2000000000ull));
                            if (got) {
                                ph ^= 1u << s;
                                pend &= ~(1u << s);
                            } else {
                                // the copy did not complete: flag the launch (as a barrier
                                // time-out does, so the grid runs to its end and the step
                                // reports it), stop staging rows and wait, bounded, for the
                                // copies still in flight
                                if (lane == 0) atomicExch(&G->err, 1);
                                staged = false;
                                stage_ok = false;
                                drain_stages(stage_bar[wl], &pend, &ph, nst);
                            }
                            const VT *Ds = reinterpret_cast<const VT *>(stg + (size_t)s * P.grid_stage);
                            const VT *wv = reinterpret_cast<const VT *>(w + wbk);
                            // the products and sums of the direct path below, in its order
                            const int nv = got ? (len + VN - 1) / VN : 0;
                            for (int base = 0; base < nv; base += CH * 32) {
                                T a0 = (T)0;
#pragma unroll
                                for (int q = 0; q < CH; ++q) {
                                    const int c = base + lane + 32 * q;
                                    if (c < nv) a0 = vdot(Ds[c], wv[c], a0);
                                }
                                acc += a0;
                            }
                        }
                        __syncwarp();
                        if (k + nst < trips) {
                            const int len2 = __shfl_sync(0xffffffffu, r_len, k + nst);
                            const int drow2 = __shfl_sync(0xffffffffu, r_drow, k + nst);
                            if (staged && lane == 0 && len2 > 0)
                                bulk_row_load(stg + (size_t)s * P.grid_stage, V.htb + drow2,
                                              (unsigned)((len2 + VN - 1) / VN * 16), &stage_bar[wl][s]);
                            if (staged && len2 > 0) pend |= 1u << s;
                        }
#pragma unroll
                        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        if (lane == k && r_len > 0) {
                            const int t = xg + lane * groups;
                            const T a = acc + own_c;
                            const T ynew = r_bt * a - own_lam;
                            if (P.stop_theta) {
                                const T dy = ynew - own_y;
                                tpart += dy * dy;
                            }
                            YO[t] = own_y;
                            Y[t] = ynew;
                            X[t] = a;
                        }
                    }
                } else if (rowcache) {
                    // each lane's own row: c, lambda and the old y, fetched before the sweep
                    T own_c = (T)0, own_lam = (T)0, own_y = (T)0;
                    if (r_len > 0) {
                        own_c = V.htb[r_coff];
                        own_lam = LAM[r_row];
                        own_y = Y[xg + lane * groups];
                    }
                    // two rows at a time, every D chunk of a pass loaded before any FMA
                    for (int k = 0; k < trips; k += 2) {
                        int len[2], drow[2], wb[2];
                        T acc[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int kk = k + h < trips ? k + h : 0;
                            len[h] = __shfl_sync(0xffffffffu, r_len, kk);
                            drow[h] = __shfl_sync(0xffffffffu, r_drow, kk);
                            wb[h] = __shfl_sync(0xffffffffu, r_wb, kk);
                            if (k + h >= trips) len[h] = 0;
                            acc[h] = (T)0;
                        }
                        const int nv0 = (len[0] + VN - 1) / VN, nv1 = (len[1] + VN - 1) / VN;
                        const int nvm = nv0 > nv1 ? nv0 : nv1;
                        for (int base = 0; base < nvm; base += CH * 32) {
                            VT dv0[CH], dv1[CH];
                            const VT *D0 = reinterpret_cast<const VT *>(V.htb + drow[0]);
                            const VT *D1 = reinterpret_cast<const VT *>(V.htb + drow[1]);
#pragma unroll
                            for (int q = 0; q < CH; ++q) {
                                const int c = base + lane + 32 * q;
                                dv0[q] = c < nv0 ? D0[c] : VecZero<T>::get();
                                dv1[q] = c < nv1 ? D1[c] : VecZero<T>::get();
                            }
                            const VT *w0 = reinterpret_cast<const VT *>(w + wb[0]);
                            const VT *w1 = reinterpret_cast<const VT *>(w + wb[1]);
                            T a0 = (T)0, a1 = (T)0;
#pragma unroll
                            for (int q = 0; q < CH; ++q) {
                                const int c = base + lane + 32 * q;
                                if (c < nv0) a0 = vdot(dv0[q], w0[c], a0);
                                if (c < nv1) a1 = vdot(dv1[q], w1[c], a1);
                            }
                            acc[0] += a0;
                            acc[1] += a1;
                        }
#pragma unroll
                        for (int o = 16; o; o >>= 1) {
                            acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
                            acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
                        }
                        // lane k + h owns row k + h's tables: it writes the row's outputs
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (lane == k + h && r_len > 0) {
                                const int t = xg + lane * groups;
                                const T a = acc[h] + own_c;
                                const T ynew = r_bt * a - own_lam;
                                if (P.stop_theta) {
                                    const T dy = ynew - own_y;
                                    tpart += dy * dy;
                                }
                                YO[t] = own_y;
                                Y[t] = ynew;
                                X[t] = a;
                            }
                        }
                    }
                }
                for (int k = 0; k < (rowcache || staged ? 0 : trips); k += 2) {
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
                                const T dy = ynew - Y[t];
                                tpart += dy * dy;
                            }
                            YO[t] = Y[t];
                            Y[t] = ynew;
                            X[t] = a;
                        }
                    }
                }
                if (P.stop_theta) {
#pragma unroll
                    for (int o = 16; o; o >>= 1) tpart += __shfl_xor_sync(0xffffffffu, tpart, o);
                    if (lane == 0) s_theta[wl] = (double)tpart;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        double tb = 0.0;
                        for (int k = 0; k < SUBADMM_WARPS; ++k) tb += s_theta[k];
                        if (tb != 0.0) atomicAdd(&G->theta[(l + wasted) % 3], tb);
                    }
                }
                d.sync();
                pc.mark(PHASE_VSTEP);
                // slots rotate with the iterations run in this step, restarts included: the
                // next iteration's slot was last read two barriers ago
                if (lead) {
                    G->umax[(l + wasted + 1) % 3] = 0ull;
                    G->theta[(l + wasted + 1) % 3] = 0.0;
                }
                last_par = par;
                iters = l + 1;
                if (P.stop_theta) {
                    const double ths = vload(&G->theta[(l + wasted) % 3]);
                    if (l >= 1 && (T)ths < theta_thT) { th = ths; conv = 1; break; }
                }
                // ---- z-step (Sec. III-C); u = -lambda; max(|x - z|, |dz|) as bits
                T *wn = par ? W0 : W1;
                U mloc = icache ? ri.project(Y, X, LAM, wn, Z, ZO) : (U)0;
                for (int i = icache && !igeneric ? S.nitem : ix; i < S.nitem; i += d.nthreads) {
                    const Item it = V.item[i];
                    if (it.type < 0) continue;
                    const int *ls = V.list + it.lo;
                    if (P.pj) {
                        mloc = pj_item<T, U>(it, ls, X, E, INVS, KF, AL, MU, LAM, Z, ZO, wn,
                                             (T)P.pj_omega, mloc);
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
                    if (icache) break;                  // this thread's one item
                }
                mloc = warp_umax(mloc);
                if (lane == 0) s_umax[wl] = (unsigned long long)mloc;
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned long long mb = 0ull;
                    for (int k = 0; k < SUBADMM_WARPS; ++k) mb = umax(mb, s_umax[k]);
                    if (mb) atomicMax(&G->umax[(l + wasted) % 3], mb);
                }
                d.sync();
                const U mx = (U)vload(&G->umax[(l + wasted) % 3]);
                par ^= 1;
                pc.mark(PHASE_ZSTEP);
                if (learned_mode && l == 9) {
                    if (learned && (unsigned long long)mx > ref10) { restart = true; break; }
                    if (!learned && lead) P.ref10[sc] = (unsigned long long)mx;
                    if (learned && lead) P.learn_skip[2 * sc + 1] = 0;
                }
                if (mx >= inf_bits(T(0))) { status = ST_NAN; break; }
                if (primal_stop && mx <= tolb) { conv = 1; break; }
            }
            if (restart) {
                // the learned start trails the plain one after 10 iterations: restart the step
                // from the plain start, and start plain for the next 2^streak - 1 steps
                if (lead) {
                    const int streak = min(P.learn_skip[2 * sc + 1] + 1, 5);
                    P.learn_skip[2 * sc + 1] = streak;
                    P.learn_skip[2 * sc] = (1 << streak) - 1;
                }
                restart = false;
                learned = false;
                ++fallbacks;
                wasted += l + 1;
                init_duals<T>(P, S, V, LAM, Z, ZO, X, Y, YO, W0, BT, false, d);
                par = 0;
                l = 0;
                continue;
            }
            if (lead) G->chk = 0ull;
            // the warp's stage buffers (idle outside the v-step) hold the solves' vector,
            // unless a copy into them may still be in flight (after a missed wait)
            const bool stg_free = P.grid_stage > 0 && __all_sync(0xffffffffu, pend == 0u);
            // v-hat from the last v-step's w (ADMM), or from the last z-step's lambda
            // (Projected Jacobi: v-hat = A^-1 (b + J^T lambda) with the impulses it reports)
            const int wpar = P.pj ? par : last_par;
            recover_v<T>(P, S, V, wpar ? W1 : W0, d,
                         stg_free ? reinterpret_cast<T *>(stg) : nullptr,
                         stg_free ? nst * P.grid_stage / (int)sizeof(T) : 0);
            d.sync();
            if (MIXED && conv && primal_stop && status == ST_OK) {
                // FP64 primal residual max |J v - z|; on a miss, refine c by the FP64 - FP32
                // difference of x at this iterate and resume
                double part = 0.0;
                for (int t = d.tid; t < S.nsr; t += d.nthreads) {
                    if (V.mlen[t] == 0) continue;
                    const SubDesc &u = P.subs[S.sub0 + V.sub[t]];
                    const int lr = t - u.sr0, n = u.n;
                    const double *Jr = V.sdb + u.od_J + (size_t)lr * n;
                    const double *v = V.sdb + u.od_v;
                    const int *jl = P.ipool + u.env_off + 2 * n;
                    double x = 0.0;
                    for (int p = jl[lr]; p < jl[u.m + lr]; ++p) x += Jr[p] * v[p];
                    part = nanmax(part, fabs(x - (double)Z[t]));
                    V.htb[V.coff[t]] += (T)(x - (double)X[t]);
                }
                part = warp_max(part);
                if (lane == 0 && part > 0.0) atomicMax(&G->chk, dbits(part));
                d.sync();
                part = __longlong_as_double((long long)vload(&G->chk));
                if (part > P.tol && l + 1 < P.max_iters) {
                    tolc *= 0.5;
                    tolb = tol_bits(T(0), tolc);
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
        {
            double tp = 0.0, pp = 0.0, dd = 0.0;
            for (int t = d.tid; t < S.nsr; t += d.nthreads) {
                if (V.mlen[t] == 0) continue;
                const double dy = (double)Y[t] - (double)YO[t];
                tp += dy * dy;
                pp = nanmax(pp, fabs((double)X[t] - (double)Z[t]));
                dd = nanmax(dd, (double)BT[t] * fabs((double)Z[t] - (double)ZO[t]));
            }
            tp = warp_sum(tp);
            pp = warp_max(pp);
            dd = warp_max(dd);
            if (lane == 0) {
                if (tp != 0.0) atomicAdd(&G->tsum, tp);
                if (pp > 0.0) atomicMax(&G->pmax, dbits(pp));
                if (dd > 0.0) atomicMax(&G->dmax, dbits(dd));
            }
        }
        d.sync();
        const double rp = __longlong_as_double((long long)vload(&G->pmax));
        const double rd = __longlong_as_double((long long)vload(&G->dmax));
        if (!P.stop_theta) th = vload(&G->tsum);
        pc.mark(PHASE_EXIT);
        // v-hat out and state update (Algorithm 1, after the loop)
        for (int i = d.warp; i < S.nsub; i += d.nwarps) {
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
        pc.mark(PHASE_RECOVER);
        pc.flush(iters);
        // warm-start state and reports
        for (int r = d.tid; r < S.nrow; r += d.nthreads) P.lam[S.row_g0 + r] = (double)LAM[r];
        for (int t = d.tid; t < S.nsr; t += d.nthreads) P.z[S.sr_g0 + t] = (double)Z[t];
        d.sync();
        if (lead) {
            if (vload(&G->err)) status = ST_TIMEOUT;
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
    }
    // a copy still in flight after a missed wait: wait for it (bounded) before the block exits
    if (pend) drain_stages(stage_bar[wl], &pend, &ph, nst);
}

// Self-test of the barrier's time limit: every block waits once for `expected` arrivals and
// counts itself in `passed` when the wait ends (expected > blocks: nothing completes the
// barrier, so every wait runs out and raises the error flag).
__global__ void barrier_probe_kernel(unsigned *count, unsigned *gen, int *err, unsigned expected,
                                     unsigned long long limit_ns, int *passed)
{
    grid_barrier(count, gen, err, expected, limit_ns);
    if (threadIdx.x == 0) atomicAdd(passed, 1);
}

}  // namespace subadmm
