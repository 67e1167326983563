// libsubadmm: host runtime and C ABI (include/subadmm.h) of the sm_103a subsystem-based
// ADMM solver.  The runtime lays the scenes out for the step kernel once, when the topology
// is fixed, and then only enqueues launches and copies on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "subadmm.h"
#include "layout.h"
#include "step_kernel.cuh"
#include "grid_kernel.cuh"
#include "features.cuh"
#include "warmstart.h"
#include "device_guard.h"
#include "gram.h"
#include "chol.h"

namespace {

std::string g_create_error;
constexpr int kGridSideRows = 8192;   // default: scenes with at least this many side-rows use
                                      // the grid kernel

struct HostSub {
    int scene = 0, kind = 0, n = 0, nb = 0;
    std::vector<double> Ab;      // generic: A (n*n) then b (n)
    std::vector<double> bodies;  // rigid: nb records of 17
    std::vector<double> lin;     // linear: mass (nb), f (n), X0 (n), K values (CSR)
    std::vector<int> csr;        // linear: K row pointers (n+1), then column indices
    std::vector<double> nodes;   // linear: nb records of 6 (x[3], v[3])
    int ne = 0;                  // co-rotational linear block: elements
    std::vector<int> tets;       // 4 node indices per element
    std::vector<double> Ke;      // 12 x 12 rest stiffness per element
};

struct LaunchClass {
    bool cached = false;           // register-cached iteration
    int split = 1;                 // lanes per side-row in the v-step mat-vec
    bool half = false;             // placed within half an SM's shared memory (two blocks/SM)
    bool grid = false;             // one scene at a time over the whole GPU (cooperative launch)
    int nt = SUBADMM_THREADS;      // threads per block (SUBADMM_WIDE: a generic class whose
                                   // scenes take a whole SM, one block per SM)
    int blocks = 0;                // grid class: blocks of the cooperative launch
    int block_div = 1;             // grid class: the launch takes the resident blocks / this
                                   // (autotuned: fewer blocks make cheaper grid barriers)
    std::vector<int> scenes;
    int ids_off = 0;               // offset of the scene list in d_scene_ids
    int max_smem = 0;
    cudaStream_t stream = nullptr; // class 0 runs on the simulation's stream
    cudaEvent_t done = nullptr;
};

struct HostCon {
    int scene = 0, src = 0, type = 0, rows = 0, ns = 0;
    int side_sub[SUBADMM_MAXS] = {0};   // global subsystem ids
    int sa = -1, ba = 0, sb = -1, bb = 0;
    std::vector<double> data;    // explicit: k, alpha, mu, e[rows], J blocks ; model: 23 params
};

}  // namespace

struct sim_s {
    sim_options opt{};
    std::string err;
    cudaStream_t stream = nullptr;
    std::vector<HostSub> subs;
    std::vector<HostCon> cons;
    bool finalized = false;
    // layout (device order) and maps from public ids
    std::vector<SceneDesc> scenes;
    std::vector<SubDesc> sdesc;
    std::vector<ConDesc> cdesc;
    std::vector<int> sub_dev;      // public subsystem id -> device index
    std::vector<int> con_dev;      // public interface id -> device index
    std::vector<int> con_rowg;     // device constraint -> global row of row 0
    std::vector<int> con_srg;      // device constraint -> global side-row of side 0 row 0 (per side below)
    std::vector<std::vector<int>> con_sr_global;  // per device constraint, global side-row per side
    int nscenes = 0;
    long long dof = 0, nrows = 0, nsr = 0, nbodies = 0;
    int max_smem = 0;
    std::vector<int> pool_gen_off; // device subsystem -> pool offset of A,b (generic)
    // device buffers
    SceneDesc *d_scenes = nullptr;
    SubDesc *d_subs = nullptr;
    ConDesc *d_cons = nullptr;
    Item *d_items = nullptr;
    int *d_lists = nullptr;
    int *d_asm = nullptr;
    // launch classes: scenes that share a kernel variant (register-cached or generic, lanes
    // per side-row) and a shared-memory budget; each class is one launch, the classes run
    // concurrently on forked streams
    std::vector<LaunchClass> classes;
    int *d_scene_ids = nullptr;    // every class's scene list, concatenated
    GridScratch *d_grid = nullptr; // grid kernel scratch
    // learned warm start: interface maps, the residual reference per scene, buffers
    int *d_pub2dev = nullptr;      // public interface id -> device constraint
    int *d_con_scene = nullptr;    // device constraint -> scene
    unsigned long long *d_ref10 = nullptr;
    int *d_learn_skip = nullptr;   // per scene: plain steps left, fallback streak
    double *d_lam0 = nullptr;      // learned initial lambda per row
    float *d_feat = nullptr, *d_netout = nullptr;
    cudaEvent_t ev_fork = nullptr;
    int split_override = 0;        // tuning: force the split of every class (0: heuristic)
    std::vector<int> sc_nsr, sc_items, sc_sides, sc_mpad;   // per scene: register-cache limits
    std::vector<int> sc_fmap_ok;   // per scene: bit si set if the thread map for 2^si lanes exists
    int smem_full = 0;             // dynamic shared memory a block may use
    int grid_side_rows = kGridSideRows;
    int grid_staging = 1;          // grid kernel: stage D rows in shared memory by bulk copies
    int grid_blocks = 0;           // grid kernel: blocks of the cooperative launch (0: all resident)
    int keep_factors = 1;          // keep the factors of constant blocks across steps
    int pj = 0;                    // Projected Jacobi instead of ADMM (sim_set_solver)
    double pj_omega = 1.0;
    int tensor_cores = 1;          // grid scenes, mixed form: D, c by the tcgen05 Gram kernel
    std::vector<subadmm::GramPlan> gram;   // per scene: Gram jobs of its tc subsystems
    int tc_factor = 1;             // refactorised tc subsystems' FP32 factors by the blocked
                                   // Cholesky with tensor-core Schur updates
    std::vector<subadmm::CholPlan> chol;   // per scene: the blocked factorisation's panels
    std::vector<int> h_ipool;      // host copy of the integer pool (envelopes)
    std::vector<char> grid_factored;       // per scene: its tc subsystems hold kept factors
    // graph replay of sim_step
    bool use_graph = false;
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t graph_learned = nullptr;   // one learned step, captured for one network
    void *graph_learned_net = nullptr;
    long long graph_learned_ws = -1;           // the network workspace it was captured with
    int graph_learned_steps = 0;               // and its step count
    cudaStream_t graph_stream = nullptr;   // capture and replay stream when the simulation's
                                           // stream is the legacy default stream
    double *d_pool = nullptr, *d_bodies = nullptr, *d_vhat = nullptr, *d_lam = nullptr;
    double *d_z = nullptr, *d_beta = nullptr, *d_res = nullptr, *d_stage = nullptr;
    long long *d_stats = nullptr;
    long long *d_phase = nullptr;  // phase tracer counters (8 per scene) when enabled
    double *d_work = nullptr;      // per-subsystem arrays of scenes too large for shared memory
    double *d_nodes = nullptr;     // node states of linear blocks
    int *d_ipool = nullptr;        // integer constant data
    int *d_subflag = nullptr;      // per subsystem: kept-factor flags
    int *d_pending = nullptr;      // per subsystem: map formation of the current step
    double *d_beta_scale = nullptr;   // per subsystem: beta = scale x (trace rule or rho)
    double *d_beta_used = nullptr;    // per subsystem: the scale of the kept factor
    float *d_bacc = nullptr;          // learned beta: per-scene sums and counts
    long long nnodes = 0;
    long long work_bytes = 0;
    size_t pool_size = 0;
};

namespace {

int fail(sim_t s, int code, const std::string &msg)
{
    if (s) s->err = msg; else g_create_error = msg;
    return code;
}

int cuda_fail(sim_t s, cudaError_t e, const char *what)
{
    return fail(s, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, what); \
    } while (0)

int model_rows_of(int src)
{
    switch (src) {
    case SRC_BALL: return 3;
    case SRC_REVOLUTE: return 5;
    case SRC_ANGLE_PD: return 1;
    case SRC_PLANE: return 3;
    case SRC_SPHERE: return 3;
    default: return 0;
    }
}

int model_type_of(int src)
{
    switch (src) {
    case SRC_ANGLE_PD: return TYPE_SOFT;
    case SRC_PLANE: return TYPE_CONTACT;
    case SRC_SPHERE: return TYPE_CONTACT;
    default: return TYPE_EQUALITY;
    }
}

// pack / unpack of the 13 state doubles (p, q, v, w) of every body record
// Packed state: 13 doubles per rigid body (p, q, v, w), then 6 per node of the linear blocks
// (x, v; the node records are stored in exactly that layout).
__global__ void pack_state(const double *bodies, const double *nodes, double *out, long long nb,
                           long long nn)
{
    const long long nbd = nb * 13, total = nbd + nn * SUBADMM_NODE;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < nbd) {
            const long long b = i / 13, k = i - b * 13;
            out[i] = bodies[b * SUBADMM_BODY + 4 + k];
        } else {
            out[i] = nodes[i - nbd];
        }
    }
}

__global__ void unpack_state(double *bodies, double *nodes, const double *in, long long nb,
                             long long nn)
{
    const long long nbd = nb * 13, total = nbd + nn * SUBADMM_NODE;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < nbd) {
            const long long b = i / 13, k = i - b * 13;
            bodies[b * SUBADMM_BODY + 4 + k] = in[i];
        } else {
            nodes[i - nbd] = in[i];
        }
    }
}

#define ON_DEVICE(dev)                                                  \
    subadmm::DeviceGuard device_guard_(dev);                                     \
    if (device_guard_.err != cudaSuccess) return cuda_fail(s, device_guard_.err, "cudaSetDevice")

// Drops the captured graphs of sim_step and sim_step_learned: their launches hold the kernel
// arguments (variants, flags, tracer pointer) of their capture, so they are captured again.
void drop_graphs(sim_t s)
{
    if (s->graph) cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
    s->graph_steps = 0;
    if (s->graph_learned) cudaGraphExecDestroy(s->graph_learned);
    s->graph_learned = nullptr;
    s->graph_learned_net = nullptr;
}

long long state_doubles(const sim_t s) { return 13 * s->nbodies + SUBADMM_NODE * s->nnodes; }

void free_device(sim_t s)
{
    cudaFree(s->d_scenes); cudaFree(s->d_subs); cudaFree(s->d_cons); cudaFree(s->d_pool);
    cudaFree(s->d_items); cudaFree(s->d_lists); cudaFree(s->d_asm);
    s->d_items = nullptr; s->d_lists = nullptr; s->d_asm = nullptr;
    cudaFree(s->d_bodies); cudaFree(s->d_vhat); cudaFree(s->d_lam); cudaFree(s->d_z);
    cudaFree(s->d_beta); cudaFree(s->d_res); cudaFree(s->d_stats); cudaFree(s->d_stage);
    cudaFree(s->d_phase);
    s->d_phase = nullptr;
    cudaFree(s->d_work);
    s->d_work = nullptr;
    cudaFree(s->d_nodes); cudaFree(s->d_ipool); cudaFree(s->d_subflag);
    cudaFree(s->d_beta_scale); cudaFree(s->d_beta_used); cudaFree(s->d_bacc);
    cudaFree(s->d_pending);
    s->d_pending = nullptr;
    s->d_beta_scale = nullptr; s->d_beta_used = nullptr; s->d_bacc = nullptr;
    cudaFree(s->d_scene_ids);
    s->d_scene_ids = nullptr;
    cudaFree(s->d_grid);
    s->d_grid = nullptr;
    cudaFree(s->d_pub2dev); cudaFree(s->d_con_scene); cudaFree(s->d_ref10); cudaFree(s->d_learn_skip);
    s->d_learn_skip = nullptr;
    cudaFree(s->d_lam0); cudaFree(s->d_feat); cudaFree(s->d_netout);
    s->d_pub2dev = nullptr; s->d_con_scene = nullptr; s->d_ref10 = nullptr;
    s->d_lam0 = nullptr; s->d_feat = nullptr; s->d_netout = nullptr;
    for (auto &c : s->classes) {
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    s->classes.clear();
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    s->ev_fork = nullptr;
    drop_graphs(s);
    for (auto &g : s->gram) subadmm::gram_plan_free(g);
    s->gram.clear();
    for (auto &c : s->chol) subadmm::chol_plan_free(c);
    s->chol.clear();
    s->grid_factored.clear();
    if (s->graph_stream) cudaStreamDestroy(s->graph_stream);
    s->graph_stream = nullptr;
    s->d_nodes = nullptr; s->d_ipool = nullptr; s->d_subflag = nullptr;
    s->d_scenes = nullptr; s->d_subs = nullptr; s->d_cons = nullptr; s->d_pool = nullptr;
    s->d_bodies = nullptr; s->d_vhat = nullptr; s->d_lam = nullptr; s->d_z = nullptr;
    s->d_beta = nullptr; s->d_res = nullptr; s->d_stats = nullptr; s->d_stage = nullptr;
}

template <typename T>
int upload(sim_t s, T **dst, const std::vector<T> &src, const char *what)
{
    const size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) return fail(s, SIM_ENOMEM, std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
    if (!src.empty()) {
        e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, what);
    }
    return SIM_OK;
}

int zeros(sim_t s, double **dst, size_t count, const char *what)
{
    cudaError_t e = cudaMalloc((void **)dst, std::max<size_t>(count, 1) * sizeof(double));
    if (e != cudaSuccess) return fail(s, SIM_ENOMEM, std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
    e = cudaMemsetAsync(*dst, 0, std::max<size_t>(count, 1) * sizeof(double), s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, what);
    return SIM_OK;
}

// Lays out every scene for the step kernel and uploads it.
int finalize(sim_t s)
{
    if (s->finalized) return SIM_OK;
    ON_DEVICE(s->opt.device);
    const int nsubs = (int)s->subs.size(), ncons = (int)s->cons.size();
    int nscenes = 0;
    for (auto &u : s->subs) nscenes = std::max(nscenes, u.scene + 1);
    for (auto &c : s->cons) nscenes = std::max(nscenes, c.scene + 1);
    s->nscenes = nscenes;
    // device order: by scene, stable in call order
    std::vector<int> sub_order(nsubs), con_order(ncons);
    for (int i = 0; i < nsubs; ++i) sub_order[i] = i;
    for (int j = 0; j < ncons; ++j) con_order[j] = j;
    std::stable_sort(sub_order.begin(), sub_order.end(), [&](int a, int b) { return s->subs[a].scene < s->subs[b].scene; });
    std::stable_sort(con_order.begin(), con_order.end(), [&](int a, int b) { return s->cons[a].scene < s->cons[b].scene; });
    s->sub_dev.assign(nsubs, 0);
    s->con_dev.assign(ncons, 0);
    for (int k = 0; k < nsubs; ++k) s->sub_dev[sub_order[k]] = k;
    for (int k = 0; k < ncons; ++k) s->con_dev[con_order[k]] = k;

    std::vector<double> pool;
    std::vector<double> bodies;
    std::vector<double> nodes;
    std::vector<int> ipool;
    std::vector<Item> items;
    std::vector<int> lists;
    std::vector<int> asm_order;
    int dev_max_smem = 0;
    CK(cudaDeviceGetAttribute(&dev_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->opt.device),
       "attribute");
    // the kernels' static shared memory (the wide FP64 variant's reduction arrays: ~1 KB)
    const int smem_budget = dev_max_smem - 2048;
    s->smem_full = smem_budget;
    int sm_smem = 0;
    CK(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->opt.device),
       "attribute");
    long long work_bytes = 0;
    int max_nsr = 0, max_items = 0, max_sides = 0, max_mpad = 0;
    struct Place { long long sd, st, sh, scd, scene_t, ints; };
    std::vector<Place> place(nscenes);
    std::vector<int> sc_mpad(nscenes, 0), sc_sides(nscenes, 0), sc_fmap_ok(nscenes, 0);
    s->sdesc.assign(nsubs, SubDesc{});
    s->cdesc.assign(ncons, ConDesc{});
    s->scenes.assign(nscenes, SceneDesc{});
    s->con_sr_global.assign(ncons, std::vector<int>());
    s->con_rowg.assign(ncons, 0);
    long long dof = 0, rows_g = 0, sr_g = 0;
    int max_smem = 0;
    int si = 0, cj = 0;
    for (int sc = 0; sc < nscenes; ++sc) {
        SceneDesc &S = s->scenes[sc];
        S.sub0 = si;
        while (si < nsubs && s->subs[sub_order[si]].scene == sc) ++si;
        S.nsub = si - S.sub0;
        S.con0 = cj;
        while (cj < ncons && s->cons[con_order[cj]].scene == sc) ++cj;
        S.ncon = cj - S.con0;
        S.sr_g0 = (int)sr_g;
        S.row_g0 = (int)rows_g;
        // subsystems of the scene
        for (int i = 0; i < S.nsub; ++i) {
            const HostSub &h = s->subs[sub_order[S.sub0 + i]];
            SubDesc &u = s->sdesc[S.sub0 + i];
            u.kind = h.kind; u.n = h.n; u.m = 0; u.local = i;
            u.nb = h.nb;
            u.body0 = (int)(bodies.size() / SUBADMM_BODY);
            if (h.kind == KIND_RIGID) bodies.insert(bodies.end(), h.bodies.begin(), h.bodies.end());
            if (h.kind == KIND_LINEAR) {
                u.body0 = (int)(nodes.size() / SUBADMM_NODE);
                nodes.insert(nodes.end(), h.nodes.begin(), h.nodes.end());
                u.csr_off = (int)ipool.size();
                ipool.insert(ipool.end(), h.csr.begin(), h.csr.end());
            }
            u.gen_off = (int)pool.size();
            if (h.kind == KIND_GENERIC) pool.insert(pool.end(), h.Ab.begin(), h.Ab.end());
            if (h.kind == KIND_LINEAR) pool.insert(pool.end(), h.lin.begin(), h.lin.end());
            u.ne = h.ne;
            if (h.ne > 0) {
                u.tet_off = (int)ipool.size();
                ipool.insert(ipool.end(), h.tets.begin(), h.tets.end());
                u.ke_off = (int)pool.size();
                pool.insert(pool.end(), h.Ke.begin(), h.Ke.end());
            }
            u.v_off = (int)dof;
            dof += h.n;
        }
        // constraints: rows, local sides
        int row = 0;
        for (int j = 0; j < S.ncon; ++j) {
            const HostCon &h = s->cons[con_order[S.con0 + j]];
            ConDesc &c = s->cdesc[S.con0 + j];
            c.src = h.src; c.type = h.type; c.rows = h.rows; c.ns = h.ns;
            c.row0 = row;
            s->con_rowg[S.con0 + j] = (int)rows_g + row;
            row += h.rows;
            c.par_off = (int)pool.size();
            pool.insert(pool.end(), h.data.begin(), h.data.end());
            for (int q = 0; q < h.ns; ++q) {
                const int d = s->sub_dev[h.side_sub[q]];
                if (d < S.sub0 || d >= S.sub0 + S.nsub)
                    return fail(s, SIM_EINVAL, "an interface side is a subsystem of another scene");
                c.sub[q] = d - S.sub0;
            }
            c.ba = h.ba; c.bb = h.bb; c.gb_a = -1; c.gb_b = -1; c.side_b = -1;
            c.node_a = 0; c.node_b = 0;
        }
        S.nrow = row;
        // side-rows, subsystem by subsystem so each subsystem's rows are contiguous; each
        // subsystem's block starts on a 16-byte boundary of the iteration type (padding
        // side-rows between blocks belong to no constraint and stay zero)
        const int vn = s->opt.precision == SIM_MIXED ? 4 : 2;
        int sr = 0;
        for (int i = 0; i < S.nsub; ++i) {
            SubDesc &u = s->sdesc[S.sub0 + i];
            sr = (sr + vn - 1) / vn * vn;
            u.sr0 = sr;
            for (int j = 0; j < S.ncon; ++j) {
                ConDesc &c = s->cdesc[S.con0 + j];
                for (int q = 0; q < c.ns; ++q)
                    if (c.sub[q] == i) { c.sr[q] = sr; sr += c.rows; }
            }
            u.m = sr - u.sr0;
            u.mpad = (u.m + vn - 1) / vn * vn;
            max_mpad = std::max(max_mpad, u.mpad);
            sc_mpad[sc] = std::max(sc_mpad[sc], u.mpad);
        }
        sr = (sr + vn - 1) / vn * vn;
        S.nsr = sr;
        for (int j = 0; j < S.ncon; ++j) {
            const ConDesc &c = s->cdesc[S.con0 + j];
            std::vector<int> g(c.ns);
            for (int q = 0; q < c.ns; ++q) g[q] = (int)sr_g + c.sr[q];
            s->con_sr_global[S.con0 + j] = g;
        }
        // model constraints: global bodies
        for (int j = 0; j < S.ncon; ++j) {
            const HostCon &h = s->cons[con_order[S.con0 + j]];
            ConDesc &c = s->cdesc[S.con0 + j];
            if (h.src <= SRC_CONTACT) continue;
            const SubDesc &ua = s->sdesc[s->sub_dev[h.sa]];
            c.gb_a = ua.body0 + h.ba;
            c.node_a = ua.kind == KIND_LINEAR ? 1 : 0;
            c.node_b = 0;
            if (h.sb >= 0) {
                const SubDesc &ub = s->sdesc[s->sub_dev[h.sb]];
                c.gb_b = ub.body0 + h.bb;
                c.node_b = ub.kind == KIND_LINEAR ? 1 : 0;
                c.side_b = (h.sb == h.sa) ? 0 : 1;
            }
        }
        // profile of every K_i = A_i + beta_i J_i^T J_i: env[p] = first column of row p inside
        // the envelope, lastr[k] = last row whose envelope reaches column k; and the column
        // span [jlo, jhi) of every J row (empty rows: jlo = jhi = n).  Cholesky fill stays
        // inside the envelope, so the factorisation and the solves skip everything outside.
        std::vector<long long> setup_cost(S.nsub, 0);
        for (int i = 0; i < S.nsub; ++i) {
            SubDesc &u = s->sdesc[S.sub0 + i];
            const HostSub &hs = s->subs[sub_order[S.sub0 + i]];
            const int n = u.n, m = u.m;
            std::vector<int> env(n), lastr(n), jlo(m, n), jhi(m, n);
            for (int p = 0; p < n; ++p) env[p] = u.kind == KIND_GENERIC ? 0 : p;
            if (u.kind == KIND_LINEAR) {
                const int *rowp = hs.csr.data(), *col = rowp + n + 1;
                for (int p = 0; p < n; ++p)
                    for (int q = rowp[p]; q < rowp[p + 1]; ++q) {
                        const int hi = std::max(p, col[q]), lo = std::min(p, col[q]);
                        env[hi] = std::min(env[hi], lo);
                    }
            }
            // A of a linear block is constant, and every row on it is a constant selector or
            // an explicit row, so its K_i (and factor) is the same at every step; a
            // co-rotational block's A changes with its elements' rotations, and a sphere
            // contact on one of its nodes turns its rows with the contact normal (K_i stays,
            // as the frame is orthonormal, but the map D = J K^-1 J^T does not)
            bool turning_rows = false;
            for (int j = 0; j < S.ncon; ++j) {
                const ConDesc &c = s->cdesc[S.con0 + j];
                if (c.src != SRC_SPHERE) continue;
                if ((c.node_a && c.sub[0] == i) ||
                    (c.node_b && c.side_b >= 0 && c.sub[c.side_b] == i))
                    turning_rows = true;
            }
            u.cst = (u.kind == KIND_LINEAR && u.ne == 0 && !turning_rows) ? 1 : 0;
            // every element's node pairs must lie inside the envelope of K's pattern (they are
            // scattered there each step)
            for (int el = 0; el < u.ne; ++el)
                for (int a = 0; a < 4; ++a)
                    for (int b2 = 0; b2 < 4; ++b2) {
                        const int na = hs.tets[4 * el + a], nb2 = hs.tets[4 * el + b2];
                        const int hi = 3 * std::max(na, nb2), lo = 3 * std::min(na, nb2);
                        for (int r = 0; r < 3; ++r)
                            if (env[hi + r] > lo)
                                return fail(s, SIM_EINVAL, "an element couples nodes outside the "
                                                           "stiffness pattern of its linear block");
                    }
            auto span = [&](int lr, int a, int b) {
                if (b <= a) return;
                if (jlo[lr] == n) { jlo[lr] = a; jhi[lr] = b; }
                else { jlo[lr] = std::min(jlo[lr], a); jhi[lr] = std::max(jhi[lr], b); }
            };
            for (int j = 0; j < S.ncon; ++j) {
                const HostCon &h = s->cons[con_order[S.con0 + j]];
                const ConDesc &c = s->cdesc[S.con0 + j];
                if (h.src <= SRC_CONTACT) {
                    size_t off = 3 + (size_t)c.rows;
                    for (int q = 0; q < c.ns; ++q) {
                        const int nq = s->sdesc[S.sub0 + c.sub[q]].n;
                        if (c.sub[q] == i) {
                            for (int r = 0; r < c.rows; ++r) {
                                int a = n, b = 0;
                                for (int p = 0; p < n; ++p)
                                    if (h.data[off + (size_t)r * n + p] != 0.0) { a = std::min(a, p); b = p + 1; }
                                span(c.sr[q] + r - u.sr0, a, b);
                            }
                        }
                        off += (size_t)c.rows * nq;
                    }
                    continue;
                }
                const int wa = c.node_a ? 3 : 6, wb = c.node_b ? 3 : 6;
                for (int r = 0; r < c.rows; ++r) {
                    if (c.sub[0] == i) span(c.sr[0] + r - u.sr0, wa * c.ba, wa * c.ba + wa);
                    if (c.side_b >= 0 && c.sub[c.side_b] == i)
                        span(c.sr[c.side_b] + r - u.sr0, wb * c.bb, wb * c.bb + wb);
                }
            }
            for (int t = 0; t < m; ++t)
                for (int p = jlo[t]; p < jhi[t]; ++p) env[p] = std::min(env[p], jlo[t]);
            // make the envelope monotone (suffix minimum), so that every row a column reaches,
            // (k, lastr[k]], holds its column-k entry inside its own band (assembled and
            // zeroed there; entries outside any band are never read)
            for (int p = n - 2; p >= 0; --p) env[p] = std::min(env[p], env[p + 1]);
            for (int k = 0; k < n; ++k) lastr[k] = k;
            for (int r = 0; r < n; ++r)
                for (int k = env[r]; k < r; ++k) lastr[k] = std::max(lastr[k], r);
            u.env_off = (int)ipool.size();
            ipool.insert(ipool.end(), env.begin(), env.end());
            ipool.insert(ipool.end(), lastr.begin(), lastr.end());
            ipool.insert(ipool.end(), jlo.begin(), jlo.end());
            ipool.insert(ipool.end(), jhi.begin(), jhi.end());
            // row groups: J^T J and J^T w sum a group's rows before touching K or the vector
            u.grp_off = (int)ipool.size();
            u.ngrp = 0;
            for (int t = 0; t < m; ++t)
                if (t == 0 || jlo[t] != jlo[t - 1] || jhi[t] != jhi[t - 1]) {
                    ipool.push_back(t);
                    ++u.ngrp;
                }
            ipool.push_back(m);
            // the subsystem's per-warp work in the setup and the recovery: the envelope
            // Cholesky and solves (band width squared per column) and J^T J (span squared
            // per row)
            long long c = 0;
            for (int p = 0; p < n; ++p) c += (long long)(p - env[p] + 1) * (p - env[p] + 1);
            for (int t = 0; t < m; ++t) c += (long long)(jhi[t] - jlo[t]) * (jhi[t] - jlo[t]);
            setup_cost[i] = c;
        }
        // the order in which warps take the subsystems in the per-warp loops (largest first,
        // so that the largest ones go to different warps)
        S.ord_off = (int)ipool.size();
        {
            std::vector<int> ord(S.nsub);
            for (int i = 0; i < S.nsub; ++i) ord[i] = i;
            std::stable_sort(ord.begin(), ord.end(),
                             [&](int a, int b) { return setup_cost[a] > setup_cost[b]; });
            ipool.insert(ipool.end(), ord.begin(), ord.end());
        }
        // work of the setup's scene-wide passes, as prefix sums over the scene's subsystems:
        // chunks of 32 columns of W = L^-1 [J^T b] (m + 1 columns), then the map's items of
        // c (one per 4 rows) and of D (4 x 4 blocks of its lower triangle)
        // (the chunks of W are listed smallest subsystem first: position k is subsystem
        // ord[nsub - 1 - k])
        S.pre_off = (int)ipool.size();
        for (int tab = 0; tab < 3; ++tab) {
            int acc = 0;
            ipool.push_back(0);
            for (int k = 0; k < S.nsub; ++k) {
                const int i = tab == 0 ? ipool[S.ord_off + S.nsub - 1 - k] : k;
                const int m = s->sdesc[S.sub0 + i].m, nb = (m + 3) / 4;
                acc += tab == 0 ? (m + 1 + 31) / 32 : tab == 1 ? nb : nb * (nb + 1) / 2;
                ipool.push_back(acc);
            }
        }
        // z-step items: one per row of an equality / hard / soft constraint, one per contact;
        // ordered by type so that neighbouring threads run the same projection
        S.item_g0 = (int)items.size();
        S.list_g0 = (int)lists.size();
        for (int type = 0; type < 4; ++type) {
            // each type starts on a warp boundary (idle items, type -1, fill the gap) so a
            // warp runs a single projection's code path
            while ((items.size() - S.item_g0) % 32) items.push_back(Item{-1, 0, 0, 0});
            for (int j = 0; j < S.ncon; ++j) {
                const ConDesc &c = s->cdesc[S.con0 + j];
                if (c.type != type) continue;
                max_sides = std::max(max_sides, c.ns);
                sc_sides[sc] = std::max(sc_sides[sc], c.ns);
                if (c.type == TYPE_CONTACT) {
                    items.push_back(Item{c.type, c.ns, c.row0, (int)lists.size() - S.list_g0});
                    for (int q = 0; q < c.ns; ++q) lists.push_back(c.sr[q]);
                } else {
                    for (int r = 0; r < c.rows; ++r) {
                        items.push_back(Item{c.type, c.ns, c.row0 + r, (int)lists.size() - S.list_g0});
                        for (int q = 0; q < c.ns; ++q) lists.push_back(c.sr[q] + r);
                    }
                }
            }
        }
        // assembly slots: constraints grouped by how their rows are built (explicit rows, or
        // one model kind), each group padded to whole warps
        S.asm_g0 = (int)asm_order.size();
        for (int grp = 0; grp <= SRC_SPHERE - SRC_CONTACT; ++grp) {
            int cnt = 0;
            for (int j = 0; j < S.ncon; ++j) {
                const int src = s->cdesc[S.con0 + j].src;
                const int g = src <= SRC_CONTACT ? 0 : src - SRC_CONTACT;
                if (g != grp) continue;
                asm_order.push_back(j);
                ++cnt;
            }
            while (cnt % 32) { asm_order.push_back(-1); ++cnt; }
        }
        S.nasm = (int)asm_order.size() - S.asm_g0;
        S.nitem = (int)items.size() - S.item_g0;
        S.nlist = (int)lists.size() - S.list_g0;
        max_items = std::max(max_items, S.nitem);
        // thread maps of the register-cached iteration: every item's side-rows on adjacent
        // lane groups of one warp (SPLIT lanes per side-row, groups aligned to SPLIT), so a
        // warp both forms the items' y and projects them; slot s * rows + r is side s, row r
        for (int si = 0; si < 3; ++si) {
            const int split = 1 << si;
            S.fmap_off[si] = -1;
            std::vector<int> map(2 * SUBADMM_THREADS, 0);
            for (int k = 0; k < SUBADMM_THREADS; ++k) map[2 * k] = -1;
            int cursor = 0;
            bool ok = true;
            for (int it = 0; it < S.nitem && ok; ++it) {
                const Item &I = items[S.item_g0 + it];
                if (I.type < 0) continue;
                const int nr = I.type == TYPE_CONTACT ? 3 : 1;
                const int lanes = I.ns * nr * split;
                if (I.ns > 2 || lanes > 32) { ok = false; break; }
                if (cursor % 32 + lanes > 32) cursor = (cursor + 31) / 32 * 32;
                if (cursor + lanes > SUBADMM_THREADS) { ok = false; break; }
                const int leader = cursor % 32;
                for (int sd = 0; sd < I.ns; ++sd)
                    for (int r = 0; r < nr; ++r)
                        for (int g = 0; g < split; ++g) {
                            const int slot = sd * nr + r;
                            const int th = cursor + slot * split + g;
                            map[2 * th] = lists[S.list_g0 + I.lo + sd] + r;
                            map[2 * th + 1] = leader | (slot << 5) | (g << 8) | (it << 11);
                        }
                cursor += lanes;
            }
            // every real side-row on exactly one lane group
            std::vector<int> seen(S.nsr, 0);
            for (int k = 0; ok && k < SUBADMM_THREADS; ++k) {
                const int t = map[2 * k];
                if (t < 0) continue;
                if (t >= S.nsr) ok = false;
                else if ((map[2 * k + 1] >> 8 & 7) == 0) ++seen[t];
            }
            for (int i = 0; ok && i < S.nsub; ++i) {
                const SubDesc &u = s->sdesc[S.sub0 + i];
                for (int r = 0; r < u.m; ++r)
                    if (seen[u.sr0 + r] != 1) { ok = false; break; }
            }
            if (!ok) continue;
            if (ipool.size() & 1) ipool.push_back(0);       // read as int2: 8-byte aligned
            S.fmap_off[si] = (int)ipool.size();
            ipool.insert(ipool.end(), map.begin(), map.end());
        }
        sc_fmap_ok[sc] = (S.fmap_off[0] >= 0 ? 1 : 0) | (S.fmap_off[1] >= 0 ? 2 : 0) | (S.fmap_off[2] >= 0 ? 4 : 0);
        // per-subsystem arrays (doubles: J, K or A, b, v, 1/L_pp or rhs, J v; T: L, W, s;
        // iteration T arrays: D, c).  T offsets are whole 16-byte vectors so D rows load as
        // vectors.
        auto tal = [&](long long v) { return (v + vn - 1) / vn * vn; };
        long long sd = 0, st = 0, sh = 0;
        S.row_bytes = 0;
        for (int i = 0; i < S.nsub; ++i) {
            SubDesc &u = s->sdesc[S.sub0 + i];
            if (u.m > SUBADMM_MAXM)
                return fail(s, SIM_EINVAL, "a subsystem has more constraint rows than supported (2048)");
            u.od_J = (int)sd; sd += (long long)u.m * u.n;
            u.od_L = (int)sd; sd += (long long)u.n * u.n;
            u.od_b = (int)sd; sd += u.n;
            u.od_v = (int)sd; sd += u.n;
            u.od_id = (int)sd; sd += u.n;
            u.od_t = (int)sd; sd += u.m;
            u.ot_L = (int)st; st += (long long)u.n * u.n;
            u.ot_W = (int)st; st = tal(st + (long long)((u.m + 4) / 4 * 4) * u.n);   // W: n rows
                                                                     // of m + 1 rounded up to 4
            u.ot_s = (int)st; st = tal(st + u.n);
            // D rows are ldd apart: an odd number of 16-byte vectors, so the rows that the
            // lanes of a warp read at once fall in different shared-memory banks
            u.ldd = ((u.mpad / vn) % 2 == 0) ? u.mpad + vn : u.mpad;
            u.ot_D = (int)sh; sh = tal(sh + (long long)u.m * u.ldd);
            S.row_bytes = std::max(S.row_bytes, (u.m + vn - 1) / vn * 16);
            u.ot_c = (int)sh; sh = tal(sh + u.m);
            if (sd > (1LL << 30) || st + sh > (1LL << 30)) return fail(s, SIM_EINVAL, "scene too large");
        }
        // scene arrays (shared memory): per side-row arrays contiguous from ot_x to ot_lam
        place[sc] = Place{sd, st, sh, 2LL * S.nsub, tal((long long)S.nsr) * 9 + 6LL * S.nrow,
                          6LL * S.nsr + 4LL * S.nitem + S.nlist};
        max_nsr = std::max(max_nsr, S.nsr);
        sr_g += S.nsr;
        rows_g += S.nrow;
    }
    s->dof = dof; s->nrows = rows_g; s->nsr = sr_g;
    s->nbodies = (long long)(bodies.size() / SUBADMM_BODY);
    // launch classes.  Per scene: lanes per side-row of the v-step mat-vec (the largest of
    // 1, 2, 4 whose groups still cover the side-rows twice), and whether it fits the
    // register-cached iteration (one side-row group and one item per thread, at most 4
    // float4 / 6 double2 chunks of a D row per lane).  The register-cached kernel runs one
    // block per SM and may take all of its shared memory; the generic kernel runs two blocks
    // per SM, so a generic scene whose per-row and iteration arrays fit within half an SM is
    // placed there, and the others get the whole budget in a class of their own.
    const int tsize = s->opt.precision == SIM_MIXED ? 4 : 8;
    const int vn = s->opt.precision == SIM_MIXED ? 4 : 2;
    const int chunks = s->opt.precision == SIM_MIXED ? 4 : 6;
    auto tal = [&](long long v) { return (v + vn - 1) / vn * vn; };
    const int half_budget = std::min(smem_budget, sm_smem / 2 - 2048);
    auto bytes_with = [&](const Place &q, long long d, long long tt) {
        const long long tb = (d * 8 + 15) / 16 * 16;
        const long long ib = (tb + tt * tsize + 15) / 16 * 16;
        return ib + 4 * q.ints;
    };
    std::vector<int> sc_budget(nscenes, smem_budget), sc_class(nscenes, 0);
    s->sc_nsr.assign(nscenes, 0);
    s->sc_items.assign(nscenes, 0);
    for (int sc = 0; sc < nscenes; ++sc) {
        s->sc_nsr[sc] = s->scenes[sc].nsr;
        s->sc_items[sc] = s->scenes[sc].nitem;
    }
    s->sc_sides = sc_sides;
    s->sc_mpad = sc_mpad;
    s->sc_fmap_ok = sc_fmap_ok;
    for (int sc = 0; sc < nscenes; ++sc) s->scenes[sc].max_sides = sc_sides[sc];
    s->classes.clear();
    for (int sc = 0; sc < nscenes; ++sc) {
        const SceneDesc &S = s->scenes[sc];
        const Place &q = place[sc];
        // a scene with many side-rows runs alone over the whole GPU (grid kernel, lanes per
        // side-row 8 / 16 / 32 by the mean row length of D)
        const bool grid = S.nsr >= s->grid_side_rows;
        int split = 1;
        if (grid) {
            const double mean_m = (double)S.nsr / std::max(S.nsub, 1);
            split = mean_m >= 256 ? 32 : mean_m >= 64 ? 16 : 8;
        } else {
            while (split < 4 && 2 * split * std::max(S.nsr, 1) <= SUBADMM_THREADS) split *= 2;
        }
        if (s->split_override > 0) split = s->split_override;
        const int si = split == 4 ? 2 : split == 2 ? 1 : 0;
        const bool cached = !grid && !s->pj && s->opt.stop != SIM_STOP_THETA && (sc_fmap_ok[sc] >> si & 1) &&
                            sc_sides[sc] <= 2 && (sc_mpad[sc] + vn - 1) / vn <= chunks * split;
        const bool half = !grid && !cached && bytes_with(q, q.scd, q.sh + q.scene_t) <= half_budget;
        sc_budget[sc] = half ? half_budget : smem_budget;
        int k = 0;
        while (k < (int)s->classes.size() && !(s->classes[k].cached == cached &&
               s->classes[k].split == split && s->classes[k].half == half &&
               s->classes[k].grid == grid)) ++k;
        if (k == (int)s->classes.size()) {
            LaunchClass c;
            c.cached = cached; c.split = split; c.half = half; c.grid = grid;
            c.nt = (!cached && !half && !grid) ? SUBADMM_WIDE : SUBADMM_THREADS;
            s->classes.push_back(c);
        }
        s->classes[k].scenes.push_back(sc);
        sc_class[sc] = k;
    }
    for (int sc = 0; sc < nscenes; ++sc) {
        SceneDesc &S = s->scenes[sc];
        const Place &q = place[sc];
        const int budget = sc_budget[sc];
        auto bytes_of = [&](long long d, long long tt) { return bytes_with(q, d, tt); };
        // everything on chip if it fits; else the setup arrays (J, K, L, W: O(n^2)) in the
        // workspace and the iteration arrays (D, c: O(m^2)) on chip; else all in the workspace
        long long od = 0, ot = 0;
        S.g_scene = -1;
        const bool grid_scene = s->classes[sc_class[sc]].grid;
        if (grid_scene) {
            // large blocks of the mixed form have their map formed on the tensor cores
            // whenever they are refactorised
            for (int i = 0; i < S.nsub; ++i) {
                SubDesc &u = s->sdesc[S.sub0 + i];
                u.tc = (s->tensor_cores && !s->pj && s->opt.precision == SIM_MIXED && u.n >= 128 &&
                        u.m >= 16) ? 1 : 0;
            }
            // everything in the workspace: the per-subsystem arrays, then the scene arrays
            S.sub_global = 1; S.hot_global = 1;
            S.g_base = work_bytes;
            S.g_tbase = (q.sd * 8 + 255) / 256 * 256;
            work_bytes += (S.g_tbase + (q.st + q.sh) * tsize + 255) / 256 * 256;
            for (int i = 0; i < S.nsub; ++i) {
                s->sdesc[S.sub0 + i].ot_D += (int)q.st;
                s->sdesc[S.sub0 + i].ot_c += (int)q.st;
            }
            S.g_scene = work_bytes;
        } else if (bytes_of(q.sd + q.scd, q.st + q.sh + q.scene_t) <= (long long)budget) {
            S.sub_global = 0; S.hot_global = 0; S.g_base = 0; S.g_tbase = 0;
            od = q.sd; ot = q.st + q.sh;
            for (int i = 0; i < S.nsub; ++i) {
                s->sdesc[S.sub0 + i].ot_D += (int)q.st;
                s->sdesc[S.sub0 + i].ot_c += (int)q.st;
            }
        } else if (bytes_of(q.scd, q.sh + q.scene_t) <= (long long)budget) {
            S.sub_global = 1; S.hot_global = 0;
            S.g_base = work_bytes;
            S.g_tbase = (q.sd * 8 + 255) / 256 * 256;
            work_bytes += (S.g_tbase + q.st * tsize + 255) / 256 * 256;
            ot = q.sh;
        } else {
            S.sub_global = 1; S.hot_global = 1;
            S.g_base = work_bytes;
            S.g_tbase = (q.sd * 8 + 255) / 256 * 256;
            work_bytes += (S.g_tbase + (q.st + q.sh) * tsize + 255) / 256 * 256;
            for (int i = 0; i < S.nsub; ++i) {
                s->sdesc[S.sub0 + i].ot_D += (int)q.st;
                s->sdesc[S.sub0 + i].ot_c += (int)q.st;
            }
        }
        S.od_beta = (int)od; od += S.nsub;
        S.od_flag = (int)od; od += S.nsub;
        S.ot_x = (int)ot; ot = tal(ot + S.nsr);
        S.ot_y = (int)ot; ot = tal(ot + S.nsr);
        S.ot_z = (int)ot; ot = tal(ot + S.nsr);
        S.ot_yo = (int)ot; ot = tal(ot + S.nsr);
        S.ot_zo = (int)ot; ot = tal(ot + S.nsr);
        S.ot_w0 = (int)ot; ot = tal(ot + S.nsr);
        S.ot_w1 = (int)ot; ot = tal(ot + S.nsr);
        S.ot_invb = (int)ot; ot = tal(ot + S.nsr);
        S.ot_b = (int)ot; ot = tal(ot + S.nsr);
        S.ot_lam = (int)ot; ot += S.nrow;
        S.ot_e = (int)ot; ot += S.nrow;
        S.ot_invs = (int)ot; ot += S.nrow;
        S.ot_kf = (int)ot; ot += S.nrow;
        S.ot_al = (int)ot; ot += S.nrow;
        S.ot_mu = (int)ot; ot += S.nrow;
        const long long t_base = (od * 8 + 15) / 16 * 16;
        const long long i_base = (t_base + ot * tsize + 15) / 16 * 16;
        const long long bytes = i_base + 4 * q.ints;
        if (grid_scene) {
            work_bytes += (bytes + 255) / 256 * 256;
            S.t_base = (int)t_base;
            S.i_base = (int)i_base;
            S.smem_bytes = 0;
            continue;
        }
        if (bytes > (long long)budget) {
            char buf[256];
            snprintf(buf, sizeof buf, "scene %d needs %lld bytes of shared memory for its per-row "
                     "arrays alone; at most %d are available", sc, bytes, budget);
            return fail(s, SIM_EINVAL, buf);
        }
        S.t_base = (int)t_base;
        S.i_base = (int)i_base;
        S.smem_bytes = (int)bytes;
        max_smem = std::max(max_smem, S.smem_bytes);
        LaunchClass &cl = s->classes[sc_class[sc]];
        cl.max_smem = std::max(cl.max_smem, S.smem_bytes);
    }
    s->max_smem = max_smem;
    {
        // scene lists, streams and events of the classes (class 0 uses the simulation's stream)
        std::vector<int> ids;
        for (auto &c : s->classes) {
            c.ids_off = (int)ids.size();
            ids.insert(ids.end(), c.scenes.begin(), c.scenes.end());
        }
        int rc2 = upload(s, &s->d_scene_ids, ids, "scene lists");
        if (rc2) return rc2;
        cudaError_t e = cudaMalloc((void **)&s->d_grid, sizeof(GridScratch));
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc grid scratch");
        std::vector<int> con_scene(std::max(ncons, 1), 0);
        for (int sc = 0; sc < nscenes; ++sc)
            for (int j = 0; j < s->scenes[sc].ncon; ++j) con_scene[s->scenes[sc].con0 + j] = sc;
        std::vector<int> pub2dev(s->con_dev.begin(), s->con_dev.end());
        if (pub2dev.empty()) pub2dev.push_back(0);
        if ((rc2 = upload(s, &s->d_con_scene, con_scene, "interface scenes"))) return rc2;
        if ((rc2 = upload(s, &s->d_pub2dev, pub2dev, "interface map"))) return rc2;
        e = cudaMalloc((void **)&s->d_ref10, sizeof(unsigned long long) * std::max(1, nscenes));
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc residual references");
        CK(cudaMemsetAsync(s->d_ref10, 0, sizeof(unsigned long long) * std::max(1, nscenes), s->stream),
           "memset references");
        e = cudaMalloc((void **)&s->d_learn_skip, sizeof(int) * 2 * std::max(1, nscenes));
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc learned-start state");
        CK(cudaMemsetAsync(s->d_learn_skip, 0, sizeof(int) * 2 * std::max(1, nscenes), s->stream),
           "memset learned-start state");
        CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming), "event");
        for (size_t k = 0; k < s->classes.size(); ++k) {
            LaunchClass &c = s->classes[k];
            if (k > 0) CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "class stream");
            CK(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming), "event");
        }
    }
    if (work_bytes > 0) {
        cudaError_t e = cudaMalloc((void **)&s->d_work, (size_t)work_bytes);
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
    }
    s->work_bytes = work_bytes;
    s->pool_gen_off.assign(nsubs, 0);
    for (int k = 0; k < nsubs; ++k) s->pool_gen_off[k] = s->sdesc[k].gen_off;
    int rc;
    if ((rc = upload(s, &s->d_scenes, s->scenes, "scenes"))) return rc;
    if ((rc = upload(s, &s->d_subs, s->sdesc, "subsystems"))) return rc;
    if ((rc = upload(s, &s->d_cons, s->cdesc, "interfaces"))) return rc;
    if ((rc = upload(s, &s->d_pool, pool, "pool"))) return rc;
    if ((rc = upload(s, &s->d_items, items, "items"))) return rc;
    if ((rc = upload(s, &s->d_lists, lists, "lists"))) return rc;
    if ((rc = upload(s, &s->d_asm, asm_order, "assembly order"))) return rc;
    if ((rc = upload(s, &s->d_bodies, bodies, "bodies"))) return rc;
    if ((rc = upload(s, &s->d_nodes, nodes, "nodes"))) return rc;
    if ((rc = upload(s, &s->d_ipool, ipool, "integer pool"))) return rc;
    s->h_ipool = ipool;
    {
        {
            const std::vector<double> ones(std::max(1, nsubs), 1.0);
            if (cudaMalloc((void **)&s->d_beta_scale, ones.size() * sizeof(double)) != cudaSuccess ||
                cudaMalloc((void **)&s->d_beta_used, ones.size() * sizeof(double)) != cudaSuccess ||
                cudaMalloc((void **)&s->d_bacc, 2 * std::max<size_t>(1, s->nscenes) * sizeof(float)) != cudaSuccess)
                return fail(s, SIM_ENOMEM, "cudaMalloc beta scale");
            CK(cudaMemcpy(s->d_beta_scale, ones.data(), ones.size() * sizeof(double),
                          cudaMemcpyHostToDevice), "beta scale");
            CK(cudaMemcpy(s->d_beta_used, ones.data(), ones.size() * sizeof(double),
                          cudaMemcpyHostToDevice), "beta scale");
        }
        if (cudaMalloc((void **)&s->d_pending, std::max(1, nsubs) * sizeof(int)) != cudaSuccess)
            return fail(s, SIM_ENOMEM, "cudaMalloc map flags");
        CK(cudaMemset(s->d_pending, 0, std::max(1, nsubs) * sizeof(int)), "map flags");
        cudaError_t e = cudaMalloc((void **)&s->d_subflag, std::max(1, nsubs) * sizeof(int));
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc subsystem flags");
        CK(cudaMemsetAsync(s->d_subflag, 0, std::max(1, nsubs) * sizeof(int), s->stream), "memset flags");
    }
    s->nnodes = (long long)(nodes.size() / SUBADMM_NODE);
    s->pool_size = pool.size();
    if ((rc = zeros(s, &s->d_vhat, (size_t)dof, "vhat"))) return rc;
    if ((rc = zeros(s, &s->d_lam, (size_t)rows_g, "lambda"))) return rc;
    if ((rc = zeros(s, &s->d_z, (size_t)sr_g, "z"))) return rc;
    if ((rc = zeros(s, &s->d_beta, (size_t)nsubs, "beta"))) return rc;
    if ((rc = zeros(s, &s->d_res, (size_t)6 * nscenes, "residuals"))) return rc;
    if ((rc = zeros(s, &s->d_stage, (size_t)state_doubles(s), "state staging"))) return rc;
    {
        cudaError_t e = cudaMalloc((void **)&s->d_stats, std::max(1, 5 * nscenes) * sizeof(long long));
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc stats");
        CK(cudaMemsetAsync(s->d_stats, 0, std::max(1, 5 * nscenes) * sizeof(long long), s->stream), "memset stats");
    }
    s->finalized = true;
    return SIM_OK;
}

int check_rows_data(sim_t s, int kind, int rows, int n_sides, const int *sides, const double *J,
                    const double *e, const double *params, HostCon &c)
{
    if (rows < 1 || rows > 8) return fail(s, SIM_EINVAL, "rows must be in 1..8");
    if (kind == SRC_CONTACT && rows != 3) return fail(s, SIM_EINVAL, "a contact has 3 rows");
    if (n_sides < 1 || n_sides > SUBADMM_MAXS) return fail(s, SIM_EINVAL, "n_sides must be in 1..8");
    if (!sides || !J || !e) return fail(s, SIM_EINVAL, "sides, J and e are required");
    if (kind == SRC_SOFT && (!params || !(params[0] > 0.0) || !(params[1] > 0.0)))
        return fail(s, SIM_EINVAL, "a soft interface needs k > 0 and alpha > 0");
    if (kind == SRC_CONTACT && (!params || !(params[2] >= 0.0)))
        return fail(s, SIM_EINVAL, "a contact needs mu >= 0");
    c.src = kind; c.type = kind; c.rows = rows; c.ns = n_sides;
    c.data.clear();
    c.data.push_back(params ? params[0] : 0.0);
    c.data.push_back(params ? params[1] : 0.0);
    c.data.push_back(params ? params[2] : 0.0);
    for (int r = 0; r < rows; ++r) c.data.push_back(e[r]);
    const double *Jp = J;
    for (int q = 0; q < n_sides; ++q) {
        const int id = sides[q];
        if (id < 0 || id >= (int)s->subs.size()) return fail(s, SIM_EINVAL, "unknown subsystem id");
        for (int t = 0; t < q; ++t)
            if (sides[t] == id) return fail(s, SIM_EINVAL, "sides must be distinct subsystems");
        c.side_sub[q] = id;
        const int n = s->subs[id].n;
        c.data.insert(c.data.end(), Jp, Jp + (size_t)rows * n);
        Jp += (size_t)rows * n;
    }
    for (double v : c.data)
        if (!std::isfinite(v)) return fail(s, SIM_EINVAL, "non-finite value in J, e or params");
    return SIM_OK;
}

}  // namespace

extern "C" {

void sim_default_options(sim_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->h = 1e-3;
    o->gravity[0] = 0.0; o->gravity[1] = 0.0; o->gravity[2] = -9.81;
    o->baumgarte = 0.2;
    o->beta_mode = SIM_BETA_TRACE;
    o->rho = 1e3;
    o->warm = SIM_WARM_PREV;
    o->stop = SIM_STOP_PRIMAL;
    o->tol_primal = 1e-6;
    o->theta_th = 1e-12;
    o->max_iters = 1000;
    o->precision = SIM_FP64;
    o->device = 0;
    o->stream = nullptr;
}

int sim_create(const sim_options *opt, sim_t *out)
{
    if (!out) return fail(nullptr, SIM_EINVAL, "out is NULL");
    *out = nullptr;
    sim_options o;
    if (opt) o = *opt; else sim_default_options(&o);
    if (!(o.h > 0.0) || o.max_iters < 1 || (o.precision != SIM_FP64 && o.precision != SIM_MIXED) ||
        (o.beta_mode != SIM_BETA_TRACE && o.beta_mode != SIM_BETA_FIXED) ||
        (o.beta_mode == SIM_BETA_FIXED && !(o.rho > 0.0)) ||
        (o.warm != SIM_WARM_COLD && o.warm != SIM_WARM_PREV) ||
        (o.stop != SIM_STOP_PRIMAL && o.stop != SIM_STOP_THETA))
        return fail(nullptr, SIM_EINVAL, "invalid options");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, SIM_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    if (o.device < 0 || o.device >= ndev) return fail(nullptr, SIM_EINVAL, "device ordinal out of range");
    {
        subadmm::DeviceGuard on_device(o.device);
        if (on_device.err != cudaSuccess)
            return fail(nullptr, SIM_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(on_device.err));
    }
    sim_t s = new (std::nothrow) sim_s();
    if (!s) return fail(nullptr, SIM_ENOMEM, "host allocation failed");
    s->opt = o;
    s->stream = (cudaStream_t)o.stream;
    *out = s;
    return SIM_OK;
}

void sim_destroy(sim_t s)
{
    if (!s) return;
    {
        subadmm::DeviceGuard on_device(s->opt.device);
        cudaStreamSynchronize(s->stream);
        free_device(s);
    }
    delete s;
}

int sim_add_subsystem(sim_t s, int scene, int kind, int count, const double *data, int *out_id)
{
    if (!s) return SIM_EINVAL;
    if (s->finalized) return fail(s, SIM_EINVAL, "topology is fixed after the first sim_step");
    if (scene < 0) return fail(s, SIM_EINVAL, "scene must be >= 0");
    if (count < 1 || !data) return fail(s, SIM_EINVAL, "count >= 1 and data are required");
    HostSub u;
    u.scene = scene;
    if (kind == SIM_SUB_GENERIC) {
        if (count > SUBADMM_MAXN) return fail(s, SIM_EINVAL, "generic subsystem larger than 2048 DOF");
        u.kind = KIND_GENERIC; u.n = count;
        u.Ab.assign(data, data + (size_t)count * count + count);
    } else if (kind == SIM_SUB_RIGID) {
        if (6 * count > SUBADMM_MAXN) return fail(s, SIM_EINVAL, "rigid subsystem larger than 2048 DOF");
        u.kind = KIND_RIGID; u.nb = count; u.n = 6 * count;
        u.bodies.assign(data, data + (size_t)count * SUBADMM_BODY);
        for (int b = 0; b < count; ++b) {
            const double *r = data + (size_t)b * SUBADMM_BODY;
            if (!(r[0] > 0.0) || !(r[1] > 0.0) || !(r[2] > 0.0) || !(r[3] > 0.0))
                return fail(s, SIM_EINVAL, "body mass and inertia must be positive");
        }
    } else if (kind == SIM_SUB_LINEAR) {
        // data: mass (nn), f (n), X0 (n), x (n), v (n), nnz, then nnz triplets (row, col,
        // value) of the symmetric stiffness K, indices stored exactly as doubles
        const int nn = count, n = 3 * count;
        if (n > SUBADMM_MAXN) return fail(s, SIM_EINVAL, "linear subsystem larger than 2048 DOF");
        u.kind = KIND_LINEAR; u.nb = nn; u.n = n;
        const double *mass = data, *f = data + nn, *X0 = f + n, *x = X0 + n, *v = x + n;
        const double nnzd = v[n];
        if (!(nnzd >= 0.0) || nnzd > (double)n * n || nnzd != (double)(long long)nnzd)
            return fail(s, SIM_EINVAL, "bad non-zero count of K");
        const long long nnz = (long long)nnzd;
        const double *trip = v + n + 1;
        for (int q = 0; q < nn; ++q)
            if (!(mass[q] > 0.0)) return fail(s, SIM_EINVAL, "node masses must be positive");
        for (long long q = 0; q < (long long)nn + 4LL * n + 3 * nnz; ++q)
            if (!std::isfinite(data[q])) return fail(s, SIM_EINVAL, "non-finite linear block data");
        std::vector<std::vector<std::pair<int, double>>> rows(n);
        for (long long t = 0; t < nnz; ++t) {
            const double rd = trip[3 * t], cd = trip[3 * t + 1];
            if (rd < 0 || rd >= n || cd < 0 || cd >= n || rd != (double)(int)rd || cd != (double)(int)cd)
                return fail(s, SIM_EINVAL, "K index out of range");
            rows[(int)rd].push_back({(int)cd, trip[3 * t + 2]});
        }
        u.lin.assign(mass, mass + nn);
        u.lin.insert(u.lin.end(), f, f + n);
        u.lin.insert(u.lin.end(), X0, X0 + n);
        u.csr.assign(1, 0);
        std::vector<int> cols;
        for (int p = 0; p < n; ++p) {
            std::sort(rows[p].begin(), rows[p].end());
            for (size_t q = 0; q < rows[p].size(); ++q) {
                if (q + 1 < rows[p].size() && rows[p][q + 1].first == rows[p][q].first)
                    return fail(s, SIM_EINVAL, "duplicate K entry");
                cols.push_back(rows[p][q].first);
                u.lin.push_back(rows[p][q].second);
            }
            u.csr.push_back((int)cols.size());
        }
        u.csr.insert(u.csr.end(), cols.begin(), cols.end());
        for (int q = 0; q < nn; ++q) {
            for (int d = 0; d < 3; ++d) u.nodes.push_back(x[3 * q + d]);
            for (int d = 0; d < 3; ++d) u.nodes.push_back(v[3 * q + d]);
        }
    } else {
        return fail(s, SIM_EINVAL, "unknown subsystem kind");
    }
    for (double v : u.Ab) if (!std::isfinite(v)) return fail(s, SIM_EINVAL, "non-finite A or b");
    for (double v : u.bodies) if (!std::isfinite(v)) return fail(s, SIM_EINVAL, "non-finite body record");
    s->subs.push_back(std::move(u));
    if (out_id) *out_id = (int)s->subs.size() - 1;
    return SIM_OK;
}

int sim_add_interface(sim_t s, int scene, int kind, int rows, int n_sides, const int *sides,
                      const double *J, const double *e, const double *params, int *out_id)
{
    if (!s) return SIM_EINVAL;
    if (s->finalized) return fail(s, SIM_EINVAL, "topology is fixed after the first sim_step");
    if (scene < 0) return fail(s, SIM_EINVAL, "scene must be >= 0");
    HostCon c;
    c.scene = scene;
    if (kind >= SIM_IF_EQUALITY && kind <= SIM_IF_CONTACT) {
        int rc = check_rows_data(s, kind, rows, n_sides, sides, J, e, params, c);
        if (rc) return rc;
        for (int q = 0; q < n_sides; ++q)
            if (s->subs[sides[q]].scene != scene) return fail(s, SIM_EINVAL, "a side belongs to another scene");
    } else if (kind >= SIM_IF_BALL && kind <= SIM_IF_SPHERE_CONTACT) {
        if (!sides || !params) return fail(s, SIM_EINVAL, "sides and params are required");
        if (J || e) return fail(s, SIM_EINVAL, "model interfaces take no J or e");
        const int sa = sides[0], ba = sides[1];
        int sb = sides[2], bb = sides[3];
        if (kind == SIM_IF_PLANE_CONTACT) { sb = -1; bb = 0; }
        // a node of a linear block may be a side of a ball joint or a contact
        const bool node_ok = kind == SIM_IF_BALL || kind == SIM_IF_PLANE_CONTACT ||
                             kind == SIM_IF_SPHERE_CONTACT;
        auto side_kind_ok = [&](int sub) {
            const int kd = s->subs[sub].kind;
            return kd == KIND_RIGID || (kd == KIND_LINEAR && node_ok);
        };
        if (sa < 0 || sa >= (int)s->subs.size() || !side_kind_ok(sa))
            return fail(s, SIM_EINVAL, "side a must be a rigid subsystem (or a linear one for BALL and the contacts)");
        if (ba < 0 || ba >= s->subs[sa].nb) return fail(s, SIM_EINVAL, "body a out of range");
        if (s->subs[sa].scene != scene) return fail(s, SIM_EINVAL, "body a belongs to another scene");
        if (sb >= 0) {
            if (sb >= (int)s->subs.size() || !side_kind_ok(sb))
                return fail(s, SIM_EINVAL, "side b must be a rigid subsystem (or a linear one for BALL and the contacts), or -1");
            if (bb < 0 || bb >= s->subs[sb].nb) return fail(s, SIM_EINVAL, "body b out of range");
            if (sb == sa && bb == ba) return fail(s, SIM_EINVAL, "a body cannot be joined to itself");
            if (s->subs[sb].scene != scene) return fail(s, SIM_EINVAL, "body b belongs to another scene");
        }
        for (int q = 0; q < SUBADMM_PARAMS; ++q)
            if (!std::isfinite(params[q])) return fail(s, SIM_EINVAL, "non-finite parameter");
        if (kind == SIM_IF_ANGLE_PD && !(params[18] > 0.0))
            return fail(s, SIM_EINVAL, "ANGLE_PD needs kp > 0");
        const bool contact = kind == SIM_IF_PLANE_CONTACT || kind == SIM_IF_SPHERE_CONTACT;
        if (contact && !(params[22] >= 0.0)) return fail(s, SIM_EINVAL, "a contact needs mu >= 0");
        if (contact && !(params[12] >= 0.0)) return fail(s, SIM_EINVAL, "a contact radius is negative");
        if (kind == SIM_IF_SPHERE_CONTACT && !(params[15] >= 0.0))
            return fail(s, SIM_EINVAL, "a contact radius is negative");
        double nrm = 0.0;
        if (kind == SIM_IF_PLANE_CONTACT) {
            nrm = std::sqrt(params[9] * params[9] + params[10] * params[10] + params[11] * params[11]);
            if (!(nrm > 0.0) || !std::isfinite(nrm))
                return fail(s, SIM_EINVAL, "PLANE_CONTACT needs a nonzero normal (axis_b)");
        }
        c.src = kind; c.type = model_type_of(kind); c.rows = model_rows_of(kind);
        c.sa = sa; c.ba = ba; c.sb = sb; c.bb = bb;
        c.side_sub[0] = sa;
        c.ns = 1;
        if (sb >= 0 && sb != sa) { c.ns = 2; c.side_sub[1] = sb; }
        c.data.assign(params, params + SUBADMM_PARAMS);
        if (kind == SIM_IF_PLANE_CONTACT)
            for (int d = 0; d < 3; ++d) c.data[9 + d] = params[9 + d] / nrm;
    } else {
        return fail(s, SIM_EINVAL, "unknown interface kind");
    }
    s->cons.push_back(std::move(c));
    if (out_id) *out_id = (int)s->cons.size() - 1;
    return SIM_OK;
}

int sim_set_generic(sim_t s, int sub, const double *A, const double *b)
{
    if (!s) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    if (sub < 0 || sub >= (int)s->subs.size() || s->subs[sub].kind != KIND_GENERIC)
        return fail(s, SIM_EINVAL, "not a generic subsystem");
    HostSub &u = s->subs[sub];
    const int n = u.n;
    if (A) for (int q = 0; q < n * n; ++q) if (!std::isfinite(A[q])) return fail(s, SIM_EINVAL, "non-finite A");
    if (b) for (int q = 0; q < n; ++q) if (!std::isfinite(b[q])) return fail(s, SIM_EINVAL, "non-finite b");
    if (A) std::memcpy(u.Ab.data(), A, sizeof(double) * n * n);
    if (b) std::memcpy(u.Ab.data() + (size_t)n * n, b, sizeof(double) * n);
    if (s->finalized) {
        const int off = s->pool_gen_off[s->sub_dev[sub]];
        CK(cudaMemcpyAsync(s->d_pool + off, u.Ab.data(), sizeof(double) * ((size_t)n * n + n),
                           cudaMemcpyHostToDevice, s->stream), "set_generic");
        // the host copy must outlive the async copy: wait for it
        CK(cudaStreamSynchronize(s->stream), "set_generic sync");
    }
    return SIM_OK;
}

}  // extern "C"

namespace {

using KernFn = void (*)(StepParams);

// `iters` rounds of the block barrier that ends every iteration of the block kernel
// (__syncthreads_count), with nothing else between them: the floor of one iteration
__global__ void barrier_floor_kernel(int iters, long long *cycles)
{
    const long long t0 = clock64();
    int acc = 0;
    for (int k = 0; k < iters; ++k) acc += __syncthreads_count((int)threadIdx.x == (k & 255));
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = (t1 - t0) + (acc < 0 ? 1 : 0);
}

// kernel parameters of a step launch (scene list filled in per class)
StepParams step_params(const sim_t s, int n_steps)
{
    StepParams P;
    P.scenes = s->d_scenes; P.subs = s->d_subs; P.cons = s->d_cons; P.pool = s->d_pool;
    P.bodies = s->d_bodies; P.vhat = s->d_vhat; P.lam = s->d_lam; P.z = s->d_z;
    P.work = s->d_work;
    P.nodes = s->d_nodes;
    P.ipool = s->d_ipool;
    P.subflag = s->d_subflag;
    P.pending = s->d_pending;
    P.beta_scale = s->d_beta_scale;
    P.beta_used = s->d_beta_used;
    P.keep_factors = s->keep_factors;
    P.beta = s->d_beta; P.res = s->d_res; P.stats = s->d_stats; P.phase = s->d_phase;
    P.nscenes = s->nscenes;
    P.n_steps = n_steps;
    P.h = s->opt.h; P.g0 = s->opt.gravity[0]; P.g1 = s->opt.gravity[1]; P.g2 = s->opt.gravity[2];
    P.gamma = s->opt.baumgarte; P.rho = s->opt.rho; P.tol = s->opt.tol_primal;
    P.theta_th = s->opt.theta_th;
    P.beta_fixed = s->opt.beta_mode == SIM_BETA_FIXED;
    P.warm_prev = s->opt.warm == SIM_WARM_PREV;
    P.stop_theta = s->opt.stop == SIM_STOP_THETA;
    // Projected Jacobi: always exactly max_iters iterations
    P.pj = s->pj;
    P.pj_omega = s->pj_omega;
    if (s->pj) { P.tol = -1.0; P.stop_theta = 0; }
    P.max_iters = s->opt.max_iters;
    P.items = s->d_items;
    P.lists = s->d_lists;
    P.asm_order = s->d_asm;
    P.scene_ids = s->d_scene_ids;
    P.grid = s->d_grid;
    P.lam0 = nullptr;
    P.tc_phase = 0;
    P.tc_factor = 0;
    P.ref10 = s->d_ref10;
    P.learn_skip = s->d_learn_skip;
    return P;
}

KernFn kernel_for(bool mixed, bool cached, int split, int nt = SUBADMM_THREADS)
{
    using namespace subadmm;
    if (!cached && nt == SUBADMM_WIDE) {
        if (mixed)
            return split == 4 ? step_kernel<float, 4, false, SUBADMM_WIDE>
                 : split == 2 ? step_kernel<float, 2, false, SUBADMM_WIDE>
                              : step_kernel<float, 1, false, SUBADMM_WIDE>;
        return split == 4 ? step_kernel<double, 4, false, SUBADMM_WIDE>
             : split == 2 ? step_kernel<double, 2, false, SUBADMM_WIDE>
                          : step_kernel<double, 1, false, SUBADMM_WIDE>;
    }
    if (mixed) {
        if (cached) return split == 4 ? step_kernel<float, 4, true> : split == 2 ? step_kernel<float, 2, true> : step_kernel<float, 1, true>;
        return split == 4 ? step_kernel<float, 4, false> : split == 2 ? step_kernel<float, 2, false> : step_kernel<float, 1, false>;
    }
    if (cached) return split == 4 ? step_kernel<double, 4, true> : split == 2 ? step_kernel<double, 2, true> : step_kernel<double, 1, true>;
    return split == 4 ? step_kernel<double, 4, false> : split == 2 ? step_kernel<double, 2, false> : step_kernel<double, 1, false>;
}

KernFn grid_kernel_for(bool mixed, int split)
{
    using namespace subadmm;
    if (mixed) return split == 32 ? grid_step_kernel<float, 32> : split == 16 ? grid_step_kernel<float, 16> : grid_step_kernel<float, 8>;
    return split == 32 ? grid_step_kernel<double, 32> : split == 16 ? grid_step_kernel<double, 16> : grid_step_kernel<double, 8>;
}

// One cooperative launch per scene of a grid class, in turn on `st`, each after zeroing the
// grid scratch; as many blocks as fit on the GPU at once.
// The Gram plan of grid scene sc (its tc subsystems' W -> D, c), built on first use.
int gram_plan_of(sim_t s, int sc)
{
    if ((int)s->gram.size() < s->nscenes) {
        s->gram.resize(s->nscenes);
        s->grid_factored.assign(s->nscenes, 0);
    }
    subadmm::GramPlan &G = s->gram[sc];
    if (G.device >= 0) return SIM_OK;
    const SceneDesc &S = s->scenes[sc];
    std::vector<subadmm::GramJob> jobs;
    unsigned char *tbase = reinterpret_cast<unsigned char *>(s->d_work) + S.g_base + S.g_tbase;
    float *stb = reinterpret_cast<float *>(tbase);
    for (int i = 0; i < S.nsub; ++i) {
        const SubDesc &u = s->sdesc[S.sub0 + i];
        if (!u.tc) continue;
        subadmm::GramJob J{};
        J.W = stb + u.ot_W;
        J.ldw = (u.m + 1 + 3) / 4 * 4;
        J.rows = u.m + 1;
        J.k = u.n;
        J.D = stb + u.ot_D;
        J.ldd = u.ldd;
        J.mpad = u.mpad;
        J.c = stb + u.ot_c;
        jobs.push_back(J);
    }
    cudaError_t e = subadmm::gram_plan_build(G, jobs);
    if (e == cudaSuccess && jobs.empty()) e = cudaGetDevice(&G.device);
    if (e == cudaErrorMemoryAllocation) return fail(s, SIM_ENOMEM, "Gram plan allocation");
    CK(e, "Gram plan");
    return SIM_OK;
}

// The blocked factorisation plan of grid scene sc (its tc subsystems' K_i), built on first use.
int chol_plan_of(sim_t s, int sc)
{
    if ((int)s->chol.size() < s->nscenes) s->chol.resize(s->nscenes);
    subadmm::CholPlan &C = s->chol[sc];
    if (C.device >= 0) return SIM_OK;
    const SceneDesc &S = s->scenes[sc];
    std::vector<subadmm::CholMatrix> mats;
    unsigned char *tbase = reinterpret_cast<unsigned char *>(s->d_work) + S.g_base + S.g_tbase;
    float *stb = reinterpret_cast<float *>(tbase);
    for (int i = 0; i < S.nsub; ++i) {
        const SubDesc &u = s->sdesc[S.sub0 + i];
        if (!u.tc) continue;
        subadmm::CholMatrix M;
        M.L = stb + u.ot_L;
        M.n = u.n;
        M.env.assign(s->h_ipool.begin() + u.env_off, s->h_ipool.begin() + u.env_off + u.n);
        M.pending = s->d_pending + S.sub0 + i;
        M.subflag = u.cst ? s->d_subflag + S.sub0 + i : nullptr;
        mats.push_back(std::move(M));
    }
    int *status = reinterpret_cast<int *>(reinterpret_cast<char *>(s->d_grid) +
                                          offsetof(GridScratch, status));
    cudaError_t e = subadmm::chol_plan_build(C, mats, status, ST_NOTSPD);
    if (e == cudaErrorMemoryAllocation) return fail(s, SIM_ENOMEM, "blocked factorisation plan");
    CK(e, "blocked factorisation plan");
    return SIM_OK;
}

int launch_grid_class(sim_t s, LaunchClass &c, StepParams P, cudaStream_t st, int split)
{
    KernFn kf = grid_kernel_for(s->opt.precision == SIM_MIXED, split);
    int per_sm = 0, sms = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, SUBADMM_THREADS, 0), "occupancy");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->opt.device), "attribute");
    const int resident = std::max(1, per_sm * sms);
    const int blocks = s->grid_blocks > 0 ? std::min(s->grid_blocks, resident)
                                          : std::max(1, resident / std::max(1, c.block_div));
    c.max_smem = 0;                 // reported: the largest stage buffers of the class's launches
    for (size_t i = 0; i < c.scenes.size(); ++i) {
        // D rows staged in shared memory by bulk copies (the warp-per-row v-step only), two
        // stages per warp if that keeps the blocks per SM of the launch without them.  (The
        // kernel takes up to 4; on the FEM beam 3 and 4 measured slower than 2: the larger
        // shared memory leaves less L1 for the w that each row is multiplied with.)
        const SceneDesc &S = s->scenes[c.scenes[i]];
        int stage = (s->grid_staging && split == 32) ? S.row_bytes : 0;
        int nst = 0;
        size_t dyn = 0;
        for (int k = 2; k >= 2 && stage > 0 && nst == 0; --k) {
            const size_t want = (size_t)stage * k * SUBADMM_WARPS;
            int per_sm_dyn = 0;
            if (cudaFuncSetAttribute((const void *)kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)want) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_dyn, kf, SUBADMM_THREADS, want) ==
                    cudaSuccess &&
                per_sm_dyn >= per_sm) {
                nst = k;
                dyn = want;
            }
            cudaGetLastError();
        }
        if (nst == 0) stage = 0;
        P.scene_ids = s->d_scene_ids + c.ids_off + (int)i;
        P.nscenes = 1;
        P.grid_stage = stage;
        P.grid_nstage = nst;
        c.max_smem = std::max(c.max_smem, (int)dyn);
        const int sc = c.scenes[i];
        int rc = gram_plan_of(s, sc);
        if (rc) return rc;
        const bool blocked = s->tc_factor && s->gram[sc].njobs > 0;
        if (blocked && (rc = chol_plan_of(s, sc))) return rc;
        // steps that refactorise tc subsystems: setup launch, (the blocked factorisation's
        // panels and the W launch,) Gram kernel, iteration launch
        int left = P.n_steps;
        // (blocks whose K changes every step, co-rotational ones, refactorise every step)
        bool changing = false;
        for (int q = 0; q < S.nsub; ++q) {
            const SubDesc &u = s->sdesc[S.sub0 + q];
            changing = changing || (u.tc && !u.cst);
        }
        while (left > 0 && s->gram[sc].njobs > 0 &&
               (changing || !s->keep_factors || !s->grid_factored[sc])) {
            StepParams Q = P;
            Q.n_steps = 1;
            Q.tc_phase = 1;
            Q.tc_factor = blocked ? 1 : 0;
            void *a1[] = {&Q};
            CK(cudaMemsetAsync(s->d_grid, 0, sizeof(GridScratch), st), "grid scratch");
            CK(cudaLaunchCooperativeKernel((const void *)kf, dim3(blocks), dim3(SUBADMM_THREADS), a1, dyn, st),
               "grid kernel launch (setup)");
            if (blocked) {
                // the deferred FP32 factors: panel kernels and tensor-core Schur updates, then
                // W of those subsystems
                CK(subadmm::chol_plan_run(s->chol[sc], st, &s->d_grid->err),
                   "blocked factorisation launch");
                Q.tc_phase = 3;
                CK(cudaMemsetAsync(s->d_grid, 0, 2 * sizeof(unsigned), st), "grid barrier");
                CK(cudaLaunchCooperativeKernel((const void *)kf, dim3(blocks), dim3(SUBADMM_THREADS), a1, dyn, st),
                   "grid kernel launch (W of the blocked factors)");
            }
            CK(subadmm::gram_plan_run(s->gram[sc], st, &s->d_grid->err), "Gram kernel launch");
            Q.tc_phase = 2;
            // the barrier counter restarts; the step's status and error word carry over
            CK(cudaMemsetAsync(s->d_grid, 0, 2 * sizeof(unsigned), st), "grid barrier");
            CK(cudaLaunchCooperativeKernel((const void *)kf, dim3(blocks), dim3(SUBADMM_THREADS), a1, dyn, st),
               "grid kernel launch (iterations)");
            if (s->keep_factors) s->grid_factored[sc] = 1;
            --left;
        }
        if (left == 0) continue;
        StepParams R = P;
        R.n_steps = left;
        CK(cudaMemsetAsync(s->d_grid, 0, sizeof(GridScratch), st), "grid scratch");
        void *args[] = {&R};
        CK(cudaLaunchCooperativeKernel((const void *)kf, dim3(blocks), dim3(SUBADMM_THREADS), args, dyn, st),
           "grid kernel launch");
    }
    return SIM_OK;
}

// Enqueue one launch per class: class 0 on the simulation's stream, the others on their
// own streams forked from it and joined back, so the classes run concurrently.
int launch_classes(sim_t s, StepParams P, cudaStream_t base)
{
    const bool mixed = s->opt.precision == SIM_MIXED;
    // grid classes first, alone on the GPU (their blocks must all be resident at once)
    std::vector<int> block_classes;
    for (int k = 0; k < (int)s->classes.size(); ++k) {
        LaunchClass &c = s->classes[k];
        if (c.grid) {
            const int rc = launch_grid_class(s, c, P, base, c.split);
            if (rc) return rc;
        } else {
            block_classes.push_back(k);
        }
    }
    const int nc = (int)block_classes.size();
    if (nc > 1) CK(cudaEventRecord(s->ev_fork, base), "fork");
    for (int j = 0; j < nc; ++j) {
        const LaunchClass &c = s->classes[block_classes[j]];
        cudaStream_t st = j == 0 ? base : c.stream;
        if (j > 0) CK(cudaStreamWaitEvent(st, s->ev_fork, 0), "fork wait");
        P.scene_ids = s->d_scene_ids + c.ids_off;
        P.nscenes = (int)c.scenes.size();
        kernel_for(mixed, c.cached, c.split, c.nt)<<<P.nscenes, c.nt, c.max_smem, st>>>(P);
        CK(cudaGetLastError(), "step kernel launch");
        if (j > 0) {
            CK(cudaEventRecord(c.done, st), "join");
            CK(cudaStreamWaitEvent(base, c.done, 0), "join wait");
        }
    }
    return SIM_OK;
}

}  // namespace

extern "C" {

int sim_step(sim_t s, int n_steps)
{
    if (!s) return SIM_EINVAL;
    if (n_steps < 1) return fail(s, SIM_EINVAL, "n_steps must be >= 1");
    int rc = finalize(s);
    if (rc) return rc;
    if (s->nscenes == 0) return SIM_OK;
    ON_DEVICE(s->opt.device);
    StepParams P = step_params(s, n_steps);
    // the attribute is per function (shared by every simulation of the process): allow the
    // full budget; each launch requests its class's own size, which sets its occupancy
    for (const LaunchClass &c : s->classes)
        CK(cudaFuncSetAttribute(kernel_for(s->opt.precision == SIM_MIXED, c.cached, c.split, c.nt),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_full),
           "shared memory attribute");
    bool has_grid = false;
    for (const LaunchClass &c : s->classes) has_grid = has_grid || c.grid;
    // (cooperative launches of the grid kernel are issued directly, not captured)
    if (s->use_graph && !has_grid) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(s->stream, &cs), "capture status");
        if (cs == cudaStreamCaptureStatusNone) {
            // the legacy default stream cannot be captured: capture on and replay from a
            // private blocking stream, which the legacy stream orders implicitly
            cudaStream_t gs = s->stream;
            if (!gs) {
                if (!s->graph_stream) CK(cudaStreamCreate(&s->graph_stream), "graph stream");
                gs = s->graph_stream;
            }
            // replay the captured launches of this step count (captured on first use)
            if (!s->graph || s->graph_steps != n_steps) {
                if (s->graph) cudaGraphExecDestroy(s->graph);
                s->graph = nullptr;
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal), "begin capture");
                const int lrc = launch_classes(s, P, gs);
                cudaError_t ec = cudaStreamEndCapture(gs, &g);
                if (lrc) { if (g) cudaGraphDestroy(g); return lrc; }
                CK(ec, "end capture");
                cudaError_t ei = cudaGraphInstantiate(&s->graph, g, 0);
                cudaGraphDestroy(g);
                CK(ei, "graph instantiate");
                s->graph_steps = n_steps;
            }
            CK(cudaGraphLaunch(s->graph, gs), "graph launch");
            if (gs != s->stream) {
                // an explicit join, so that waits on the simulation's stream cover the replay
                CK(cudaEventRecord(s->ev_fork, gs), "graph join");
                CK(cudaStreamWaitEvent(s->stream, s->ev_fork, 0), "graph join wait");
            }
            return SIM_OK;
        }
    }
    return launch_classes(s, P, s->stream);
}

int sim_use_graph(sim_t s, int enable)
{
    if (!s) return SIM_EINVAL;
    s->use_graph = enable != 0;
    if (!s->use_graph) drop_graphs(s);
    return SIM_OK;
}

namespace {

// a scene fits the register-cached iteration with `split` lanes per side-row
bool cache_fits(const sim_t s, int sc, int split)
{
    const int vn = s->opt.precision == SIM_MIXED ? 4 : 2;
    const int chunks = s->opt.precision == SIM_MIXED ? 4 : 6;
    const int si = split == 4 ? 2 : split == 2 ? 1 : 0;
    return s->opt.stop != SIM_STOP_THETA && (s->sc_fmap_ok[sc] >> si & 1) &&
           s->sc_sides[sc] <= 2 && (s->sc_mpad[sc] + vn - 1) / vn <= chunks * split;
}

void class_rows(const sim_t s, int max_classes, long long *out, const std::vector<double> *ns)
{
    for (int k = 0; k < (int)s->classes.size() && k < max_classes; ++k) {
        const LaunchClass &c = s->classes[k];
        out[5 * k + 0] = (long long)c.scenes.size();
        out[5 * k + 1] = c.grid ? 2 : c.cached ? 1 : c.nt == SUBADMM_WIDE ? 3 : 0;
        out[5 * k + 2] = c.split;
        out[5 * k + 3] = c.max_smem;
        out[5 * k + 4] = ns ? (long long)(*ns)[k] : 0;
    }
}

}  // namespace

int sim_launch_classes(sim_t s, int max_classes, long long *out)
{
    if (!s || (max_classes > 0 && !out)) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    class_rows(s, max_classes, out, nullptr);
    return (int)s->classes.size();
}

int sim_autotune(sim_t s, int steps, int max_classes, long long *out)
{
    if (!s || steps < 1 || (max_classes > 0 && !out)) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    if (s->nscenes == 0) return 0;
    CK(cudaStreamSynchronize(s->stream), "stream synchronize");
    // snapshot of everything a step writes
    struct Arr { void *p; size_t bytes; };
    const size_t nsub = s->sdesc.size();
    std::vector<Arr> arrs = {
        {s->d_bodies, sizeof(double) * SUBADMM_BODY * (size_t)s->nbodies},
        {s->d_nodes, sizeof(double) * SUBADMM_NODE * (size_t)s->nnodes},
        {s->d_vhat, sizeof(double) * (size_t)s->dof},
        {s->d_lam, sizeof(double) * (size_t)s->nrows},
        {s->d_z, sizeof(double) * (size_t)s->nsr},
        {s->d_beta, sizeof(double) * nsub},
        {s->d_res, sizeof(double) * 6 * (size_t)s->nscenes},
        {s->d_stats, sizeof(long long) * 5 * (size_t)s->nscenes},
        {s->d_ref10, sizeof(unsigned long long) * (size_t)s->nscenes},
        {s->d_learn_skip, sizeof(int) * 2 * (size_t)s->nscenes},
        {s->d_subflag, sizeof(int) * nsub},
        {s->d_beta_used, sizeof(double) * nsub},
        {s->d_phase, s->d_phase ? sizeof(long long) * 8 * (size_t)s->nscenes : 0}};
    size_t total = 0;
    for (auto &a : arrs) total += (a.p ? (a.bytes + 255) / 256 * 256 : 0);
    unsigned char *snap = nullptr;
    if (total) {
        cudaError_t e = cudaMalloc((void **)&snap, total);
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc autotune snapshot");
    }
    auto copy_all = [&](bool save) -> cudaError_t {
        size_t off = 0;
        for (auto &a : arrs) {
            if (!a.p || !a.bytes) continue;
            cudaError_t e = save ? cudaMemcpyAsync(snap + off, a.p, a.bytes, cudaMemcpyDeviceToDevice, s->stream)
                                 : cudaMemcpyAsync(a.p, snap + off, a.bytes, cudaMemcpyDeviceToDevice, s->stream);
            if (e != cudaSuccess) return e;
            off += (a.bytes + 255) / 256 * 256;
        }
        return cudaSuccess;
    };
    StepParams P = step_params(s, steps);
    for (int variant = 0; variant < 3; ++variant)
        for (int split = 1; split <= 4; split *= 2)
            CK(cudaFuncSetAttribute(kernel_for(s->opt.precision == SIM_MIXED, variant == 1, split,
                                               variant == 2 ? SUBADMM_WIDE : SUBADMM_THREADS),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_full),
               "shared memory attribute");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<double> best_ns(s->classes.size(), 0.0);
    cudaError_t err = copy_all(true);
    const std::vector<char> grid_factored = s->grid_factored;   // restored with the snapshot
    for (size_t k = 0; k < s->classes.size() && err == cudaSuccess; ++k) {
        LaunchClass &c = s->classes[k];
        P.scene_ids = s->d_scene_ids + c.ids_off;
        P.nscenes = (int)c.scenes.size();
        double best = 1e300;
        bool bc = c.cached;
        int bs = c.split, bt = c.nt;
        if (c.grid) {
            // lanes per side-row, and all resident blocks or half of them (unless the caller
            // fixed the block count); half the blocks must win by 3% over all of them, as the
            // short timing is noisy
            double best_div[3] = {1e300, 1e300, 1e300};
            int split_div[3] = {c.split, c.split, c.split};
            for (int div = 1; div <= (s->grid_blocks > 0 ? 1 : 2) && err == cudaSuccess; ++div)
            for (int split = 8; split <= 32 && err == cudaSuccess; split *= 2) {
                c.block_div = div;
                float ms = 0.0f;
                for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {   // warm, then timed
                    err = copy_all(false);
                    if (err != cudaSuccess) break;
                    cudaEventRecord(e0, s->stream);
                    const int lrc = launch_grid_class(s, c, P, s->stream, split);
                    cudaEventRecord(e1, s->stream);
                    if (lrc) { err = cudaErrorLaunchFailure; break; }
                    err = cudaEventSynchronize(e1);
                    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                }
                if (err == cudaSuccess && ms < best_div[div]) { best_div[div] = ms; split_div[div] = split; }
            }
            const int bd = best_div[2] < 0.97 * best_div[1] ? 2 : 1;
            best = best_div[bd];
            bs = split_div[bd];
            c.split = bs;
            c.block_div = bd;
            best_ns[k] = best * 1e6 / steps;
            continue;
        }
        // variants: generic (256 threads), register-cached (256), generic wide (512 threads)
        for (int variant = 0; variant < 3 && err == cudaSuccess; ++variant) {
            const bool cached = variant == 1;
            const int nt = variant == 2 ? SUBADMM_WIDE : SUBADMM_THREADS;
            for (int split = 1; split <= 4 && err == cudaSuccess; split *= 2) {
                if (cached) {
                    bool ok = !s->pj && s->opt.stop != SIM_STOP_THETA;
                    for (int sc : c.scenes) ok = ok && cache_fits(s, sc, split);
                    if (!ok) continue;
                }
                KernFn kf = kernel_for(s->opt.precision == SIM_MIXED, cached, split, nt);
                float ms = 0.0f;
                for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {   // warm, then timed
                    err = copy_all(false);
                    if (err != cudaSuccess) break;
                    cudaEventRecord(e0, s->stream);
                    kf<<<P.nscenes, nt, c.max_smem, s->stream>>>(P);
                    err = cudaGetLastError();
                    cudaEventRecord(e1, s->stream);
                    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                }
                if (err == cudaSuccess && ms < best) { best = ms; bc = cached; bs = split; bt = nt; }
            }
        }
        c.cached = bc;
        c.split = bs;
        c.nt = bt;
        best_ns[k] = best * 1e6 / steps;
    }
    if (err == cudaSuccess) err = copy_all(false);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
    s->grid_factored = grid_factored;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    if (err != cudaSuccess) return cuda_fail(s, err, "autotune");
    drop_graphs(s);            // the captured launches used the old variants
    class_rows(s, max_classes, out, &best_ns);
    return (int)s->classes.size();
}

namespace {

int interface_buffers(sim_t s)
{
    const size_t nif = std::max<size_t>(1, s->cons.size());
    if (!s->d_feat) {
        cudaError_t e = cudaMalloc((void **)&s->d_feat, sizeof(float) * nif * subadmm::kFeatures);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_netout, sizeof(float) * nif * subadmm::kDualOut);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_lam0, sizeof(double) * std::max<long long>(1, s->nrows));
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc warm-start buffers");
    }
    return SIM_OK;
}

int grid_of(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 127) / 128, 4096)); }

}  // namespace

int sim_interface_features(sim_t s, float *x_dev)
{
    if (!s || !x_dev) return SIM_EINVAL;
    int rc = finalize(s);
    if (rc) return rc;
    const int nif = (int)s->cons.size();
    if (nif == 0) return SIM_OK;
    ON_DEVICE(s->opt.device);
    subadmm::interface_features_kernel<<<grid_of(nif), 128, 0, s->stream>>>(
        step_params(s, 1), s->d_pub2dev, s->d_con_scene, nif, x_dev);
    CK(cudaGetLastError(), "features launch");
    return SIM_OK;
}

int sim_interface_targets(sim_t s, const float *x_dev, float *t_dev, float *mask_dev)
{
    if (!s || !x_dev || !t_dev || !mask_dev) return SIM_EINVAL;
    if (!s->finalized) return fail(s, SIM_EINVAL, "no step has run");
    const int nif = (int)s->cons.size();
    if (nif == 0) return SIM_OK;
    ON_DEVICE(s->opt.device);
    subadmm::interface_targets_kernel<<<grid_of(nif), 128, 0, s->stream>>>(
        step_params(s, 1), s->d_pub2dev, s->d_con_scene, nif, x_dev, t_dev, mask_dev);
    CK(cudaGetLastError(), "targets launch");
    return SIM_OK;
}

int sim_step_learned(sim_t s, wsn_t net, int n_steps)
{
    if (!s || !net) return SIM_EINVAL;
    if (n_steps < 1) return fail(s, SIM_EINVAL, "n_steps must be >= 1");
    if (s->pj) return fail(s, SIM_EINVAL, "the learned warm start serves the ADMM solver only");
    int shape[2] = {0, 0};
    if (wsn_shape(net, shape) || shape[0] != subadmm::kFeatures || shape[1] != subadmm::kDualOut)
        return fail(s, SIM_EINVAL, "the network must map 32 features to 7 outputs");
    int rc = finalize(s);
    if (rc) return rc;
    if (s->nscenes == 0) return SIM_OK;
    if ((rc = interface_buffers(s))) return rc;
    ON_DEVICE(s->opt.device);
    const int nif = (int)s->cons.size();
    StepParams P = step_params(s, n_steps);
    for (const LaunchClass &c : s->classes)
        CK(cudaFuncSetAttribute(kernel_for(s->opt.precision == SIM_MIXED, c.cached, c.split, c.nt),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_full),
           "shared memory attribute");
    // one network evaluation: features, the network, lambda^0 and the beta scales, then the
    // launches of n_steps steps, the first started from lambda^0
    auto enqueue = [&](cudaStream_t st) -> int {
        if (nif > 0) {
            subadmm::interface_features_kernel<<<grid_of(nif), 128, 0, st>>>(
                P, s->d_pub2dev, s->d_con_scene, nif, s->d_feat);
            CK(cudaGetLastError(), "features launch");
            const int r = wsn_forward(net, s->d_feat, subadmm::kFeatures, nif, s->d_netout, st);
            if (r) return fail(s, r, std::string("network: ") + wsn_last_error(net));
            subadmm::learned_duals_kernel<<<grid_of(nif), 128, 0, st>>>(
                P, s->d_pub2dev, s->d_con_scene, nif, s->d_netout, s->d_lam0);
            CK(cudaGetLastError(), "learned duals launch");
            const int nsc = s->nscenes;
            CK(cudaMemsetAsync(s->d_bacc, 0, 2 * sizeof(float) * nsc, st), "learned beta clear");
            subadmm::learned_beta_accumulate_kernel<<<grid_of(nif), 128, 0, st>>>(
                s->d_con_scene, nif, s->d_pub2dev, s->d_netout, s->d_bacc, nsc);
            CK(cudaGetLastError(), "learned beta launch");
            subadmm::learned_beta_scale_kernel<<<grid_of(nsc), 128, 0, st>>>(
                s->d_scenes, s->d_bacc, nsc, s->d_beta_scale);
            CK(cudaGetLastError(), "learned beta scale launch");
        }
        StepParams Q = P;
        Q.lam0 = nif > 0 ? s->d_lam0 : nullptr;
        return launch_classes(s, Q, st);
    };
    bool has_grid = false;
    for (const LaunchClass &c : s->classes) has_grid = has_grid || c.grid;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s->stream, &cs), "capture status");
    if (!s->use_graph || has_grid || cs != cudaStreamCaptureStatusNone) return enqueue(s->stream);
    // graph replay: capture one learned step once per network (the network's workspace is
    // reserved by a first direct step, so the capture allocates nothing)
    cudaStream_t gs = s->stream;
    if (!gs) {
        if (!s->graph_stream) CK(cudaStreamCreate(&s->graph_stream), "graph stream");
        gs = s->graph_stream;
    }
    // the first call runs directly (it reserves the network's workspace for this batch) and
    // then captures; later calls with the same network and step count replay
    if (!s->graph_learned || s->graph_learned_net != (void *)net ||
        s->graph_learned_ws != wsn_workspace_generation(net) || s->graph_learned_steps != n_steps) {
        if (s->graph_learned) cudaGraphExecDestroy(s->graph_learned);
        s->graph_learned = nullptr;
        if ((rc = enqueue(s->stream))) return rc;
        if (gs != s->stream) {
            CK(cudaEventRecord(s->ev_fork, s->stream), "graph fork");
            CK(cudaStreamWaitEvent(gs, s->ev_fork, 0), "graph fork wait");
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int lrc = enqueue(gs);
        cudaError_t ec = cudaStreamEndCapture(gs, &g);
        if (lrc) { if (g) cudaGraphDestroy(g); return lrc; }
        CK(ec, "end capture");
        cudaError_t ei = cudaGraphInstantiate(&s->graph_learned, g, 0);
        cudaGraphDestroy(g);
        CK(ei, "graph instantiate");
        s->graph_learned_net = (void *)net;
        s->graph_learned_ws = wsn_workspace_generation(net);
        s->graph_learned_steps = n_steps;
        return SIM_OK;                 // this call's steps ran directly
    }
    if (gs != s->stream) {
        CK(cudaEventRecord(s->ev_fork, s->stream), "graph fork");
        CK(cudaStreamWaitEvent(gs, s->ev_fork, 0), "graph fork wait");
    }
    CK(cudaGraphLaunch(s->graph_learned, gs), "graph launch");
    if (gs != s->stream) {
        CK(cudaEventRecord(s->ev_fork, gs), "graph join");
        CK(cudaStreamWaitEvent(s->stream, s->ev_fork, 0), "graph join wait");
    }
    return SIM_OK;
}

int sim_grid_threshold(sim_t s, int side_rows)
{
    if (!s) return SIM_EINVAL;
    if (s->finalized) return fail(s, SIM_EINVAL, "the layout is fixed after the first sim_step");
    if (side_rows < 1) return fail(s, SIM_EINVAL, "side_rows must be >= 1");
    s->grid_side_rows = side_rows;
    return SIM_OK;
}

int sim_grid_staging(sim_t s, int enable)
{
    if (!s) return SIM_EINVAL;
    s->grid_staging = enable ? 1 : 0;
    return SIM_OK;
}

int sim_set_corotational(sim_t s, int subsystem, int ne, const int *tets, const double *Ke)
{
    if (!s || !tets || !Ke) return SIM_EINVAL;
    if (s->finalized) return fail(s, SIM_EINVAL, "the layout is fixed after the first sim_step");
    if (subsystem < 0 || subsystem >= (int)s->subs.size())
        return fail(s, SIM_EINVAL, "no such subsystem");
    HostSub &h = s->subs[subsystem];
    if (h.kind != KIND_LINEAR) return fail(s, SIM_EINVAL, "not a linear subsystem");
    if (ne < 1) return fail(s, SIM_EINVAL, "ne must be >= 1");
    for (long long q = 0; q < 4LL * ne; ++q)
        if (tets[q] < 0 || tets[q] >= h.nb) return fail(s, SIM_EINVAL, "element node out of range");
    for (long long q = 0; q < 144LL * ne; ++q)
        if (!std::isfinite(Ke[q])) return fail(s, SIM_EINVAL, "non-finite element stiffness");
    h.ne = ne;
    h.tets.assign(tets, tets + 4LL * ne);
    h.Ke.assign(Ke, Ke + 144LL * ne);
    return SIM_OK;
}

int sim_set_beta_scale(sim_t s, const double *scale)
{
    if (!s || !scale) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    const int nsub = (int)s->subs.size();
    std::vector<double> dev(std::max(1, nsub), 1.0);
    for (int i = 0; i < nsub; ++i) {
        if (!(scale[i] > 0.0) || !std::isfinite(scale[i]))
            return fail(s, SIM_EINVAL, "beta scales must be positive and finite");
        dev[s->sub_dev[i]] = scale[i];
    }
    CK(cudaMemcpyAsync(s->d_beta_scale, dev.data(), sizeof(double) * dev.size(),
                       cudaMemcpyHostToDevice, s->stream), "beta scale");
    CK(cudaStreamSynchronize(s->stream), "beta scale");
    return SIM_OK;
}

int sim_grid_blocks(sim_t s, int blocks)
{
    if (!s) return SIM_EINVAL;
    if (blocks < 0) return fail(s, SIM_EINVAL, "blocks must be >= 0");
    s->grid_blocks = blocks;
    return SIM_OK;
}

int sim_set_solver(sim_t s, int solver, double omega)
{
    if (!s) return SIM_EINVAL;
    if (s->finalized) return fail(s, SIM_EINVAL, "the solver is fixed after the first sim_step");
    if (solver != SIM_SOLVER_ADMM && solver != SIM_SOLVER_PJ)
        return fail(s, SIM_EINVAL, "unknown solver");
    if (solver == SIM_SOLVER_PJ && !(omega > 0.0 && std::isfinite(omega)))
        return fail(s, SIM_EINVAL, "Projected Jacobi needs a finite omega > 0");
    s->pj = solver == SIM_SOLVER_PJ ? 1 : 0;
    s->pj_omega = s->pj ? omega : 1.0;
    return SIM_OK;
}

int sim_tensor_cores(sim_t s, int enable)
{
    if (!s) return SIM_EINVAL;
    if (s->finalized) return fail(s, SIM_EINVAL, "the layout is fixed after the first sim_step");
    s->tensor_cores = enable ? 1 : 0;
    return SIM_OK;
}

int sim_tc_factor(sim_t s, int enable)
{
    if (!s) return SIM_EINVAL;
    s->tc_factor = enable ? 1 : 0;
    return SIM_OK;
}

int sim_keep_factors(sim_t s, int enable)
{
    if (!s) return SIM_EINVAL;
    const int k = enable ? 1 : 0;
    // the flag is a kernel argument: a graph captured with the old value must not replay
    if (k != s->keep_factors) drop_graphs(s);
    s->keep_factors = k;
    return SIM_OK;
}

int sim_probe_barrier(int device, int blocks, int expected, double limit_s, int out[2])
{
    if (!out || blocks < 1 || expected < 1 || !(limit_s > 0.0) || limit_s > 10.0) return SIM_EINVAL;
    subadmm::DeviceGuard on_device(device);
    if (on_device.err != cudaSuccess) return SIM_ECUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, subadmm::barrier_probe_kernel, 32, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return SIM_ECUDA;
    if (blocks > per_sm * sms) return SIM_EINVAL;          // must all be resident
    unsigned *w = nullptr;
    if (cudaMalloc((void **)&w, 4 * sizeof(unsigned)) != cudaSuccess) return SIM_ENOMEM;
    cudaMemset(w, 0, 4 * sizeof(unsigned));
    unsigned *count = w, *gen = w + 1;
    int *err = reinterpret_cast<int *>(w + 2), *passed = reinterpret_cast<int *>(w + 3);
    unsigned ex = (unsigned)expected;
    unsigned long long lim = (unsigned long long)(limit_s * 1e9);
    void *args[] = {&count, &gen, &err, &ex, &lim, &passed};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)subadmm::barrier_probe_kernel,
                                                dim3(blocks), dim3(32), args, 0, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int host[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(host, w + 2, sizeof host, cudaMemcpyDeviceToHost);
    cudaFree(w);
    if (e != cudaSuccess) return SIM_ECUDA;
    out[0] = host[0];
    out[1] = host[1];
    return SIM_OK;
}

int sim_barrier_floor(int device, int iters, double out[2])
{
    if (!out || iters < 1 || iters > 10000000) return SIM_EINVAL;
    subadmm::DeviceGuard on_device(device);
    if (on_device.err != cudaSuccess) return SIM_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return SIM_ECUDA;
    long long *cyc = nullptr;
    if (cudaMalloc((void **)&cyc, sizeof(long long) * sms) != cudaSuccess) return SIM_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    barrier_floor_kernel<<<sms, SUBADMM_THREADS>>>(iters, cyc);     // warm-up
    cudaEventRecord(e0, 0);
    barrier_floor_kernel<<<sms, SUBADMM_THREADS>>>(iters, cyc);
    cudaEventRecord(e1, 0);
    cudaError_t e = cudaEventSynchronize(e1);
    std::vector<long long> host(sms, 0);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(host.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(cyc);
    if (e != cudaSuccess) return SIM_ECUDA;
    double sum = 0.0;
    for (long long c : host) sum += (double)c;
    out[0] = sum / sms / iters;
    out[1] = (double)ms * 1e6 / iters;
    return SIM_OK;
}

int sim_sync(sim_t s)
{
    if (!s) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    CK(cudaStreamSynchronize(s->stream), "stream synchronize");
    return SIM_OK;
}

int sim_residuals(sim_t s, int scene, double out[6])
{
    if (!s || !out) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    if (!s->finalized) return fail(s, SIM_EINVAL, "no step has run");
    if (scene < 0 || scene >= s->nscenes) return fail(s, SIM_EINVAL, "scene out of range");
    CK(cudaStreamSynchronize(s->stream), "stream synchronize");
    CK(cudaMemcpy(out, s->d_res + 6 * scene, 6 * sizeof(double), cudaMemcpyDeviceToHost), "residuals");
    const int st = (int)out[5];
    if (st != 0) {
        s->err = st == SIM_ENOTSPD ? "K_i is not positive definite" : "a residual is not finite";
        return st;
    }
    return out[4] != 0.0 ? SIM_OK : SIM_NOT_CONVERGED;
}

int sim_get(sim_t s, int what, int id, double *dst)
{
    if (!s || !dst) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    if (!s->finalized) return fail(s, SIM_EINVAL, "no step has run");
    CK(cudaStreamSynchronize(s->stream), "stream synchronize");
    if (what == SIM_GET_VHAT || what == SIM_GET_BODIES || what == SIM_GET_BETA) {
        if (id < 0 || id >= (int)s->subs.size()) return fail(s, SIM_EINVAL, "subsystem id out of range");
        const SubDesc &u = s->sdesc[s->sub_dev[id]];
        if (what == SIM_GET_VHAT)
            CK(cudaMemcpy(dst, s->d_vhat + u.v_off, sizeof(double) * u.n, cudaMemcpyDeviceToHost), "get");
        else if (what == SIM_GET_BETA)
            CK(cudaMemcpy(dst, s->d_beta + s->sub_dev[id], sizeof(double), cudaMemcpyDeviceToHost), "get");
        else {
            if (u.kind != KIND_RIGID) return fail(s, SIM_EINVAL, "not a rigid subsystem");
            CK(cudaMemcpy(dst, s->d_bodies + (size_t)u.body0 * SUBADMM_BODY,
                          sizeof(double) * SUBADMM_BODY * u.nb, cudaMemcpyDeviceToHost), "get");
        }
        return SIM_OK;
    }
    if (what == SIM_GET_NODES) {
        if (id < 0 || id >= (int)s->subs.size()) return fail(s, SIM_EINVAL, "subsystem id out of range");
        const SubDesc &u = s->sdesc[s->sub_dev[id]];
        if (u.kind != KIND_LINEAR) return fail(s, SIM_EINVAL, "not a linear subsystem");
        CK(cudaMemcpy(dst, s->d_nodes + (size_t)u.body0 * SUBADMM_NODE,
                      sizeof(double) * SUBADMM_NODE * u.nb, cudaMemcpyDeviceToHost), "get");
        return SIM_OK;
    }
    if (what == SIM_GET_LAMBDA || what == SIM_GET_Z) {
        if (id < 0 || id >= (int)s->cons.size()) return fail(s, SIM_EINVAL, "interface id out of range");
        const int d = s->con_dev[id];
        const ConDesc &c = s->cdesc[d];
        if (what == SIM_GET_LAMBDA) {
            CK(cudaMemcpy(dst, s->d_lam + s->con_rowg[d], sizeof(double) * c.rows, cudaMemcpyDeviceToHost), "get");
        } else {
            for (int q = 0; q < c.ns; ++q)
                CK(cudaMemcpy(dst + q * c.rows, s->d_z + s->con_sr_global[d][q], sizeof(double) * c.rows,
                              cudaMemcpyDeviceToHost), "get");
        }
        return SIM_OK;
    }
    return fail(s, SIM_EINVAL, "unknown quantity");
}

int sim_read_state(sim_t s, double *dst)
{
    if (!s || !dst) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    const long long nd = state_doubles(s);
    if (nd == 0) return SIM_OK;
    const int grid = (int)std::min<long long>((nd + 255) / 256, 1024);
    pack_state<<<grid, 256, 0, s->stream>>>(s->d_bodies, s->d_nodes, s->d_stage, s->nbodies, s->nnodes);
    CK(cudaGetLastError(), "pack state");
    CK(cudaMemcpyAsync(dst, s->d_stage, sizeof(double) * nd, cudaMemcpyDeviceToHost, s->stream), "read state");
    CK(cudaStreamSynchronize(s->stream), "read state sync");
    return SIM_OK;
}

}  // extern "C"

namespace {

// Staging area of sim_read_state_noalloc: a fixed 1 MiB array in device memory, one copy on
// every GPU that loads the library, held until the process exits.  Host code cannot use the
// symbol as a device address; its address is looked up once per device.
constexpr long long kNoallocStageDoubles = 131072;     // 1 MiB
__device__ __align__(256) double g_noalloc_stage[kNoallocStageDoubles];
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_addr[kNoallocMaxDevices] = {nullptr};

}  // namespace

extern "C" {

int sim_read_state_noalloc(sim_t s, double *dst)
{
    if (!s || !dst) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    if (!s->finalized)
        return fail(s, SIM_EINVAL, "sim_read_state_noalloc needs a simulation whose device memory "
                                   "is laid out (after its first sim_step)");
    const long long nd = state_doubles(s);
    if (nd == 0) return SIM_OK;
    if (nd > kNoallocStageDoubles)
        return fail(s, SIM_EINVAL, "sim_read_state_noalloc holds at most 131072 state doubles "
                                   "(1 MiB staging)");
    const int dev = s->opt.device;
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(s, SIM_EINVAL, "device ordinal too large");
    double *stage = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
            if (e != cudaSuccess) return cuda_fail(s, e, "cudaGetSymbolAddress of the staging area");
            g_noalloc_addr[dev] = static_cast<double *>(p);
        }
        stage = g_noalloc_addr[dev];
    }
    const int grid = (int)std::min<long long>((nd + 255) / 256, 1024);
    pack_state<<<grid, 256, 0, s->stream>>>(s->d_bodies, s->d_nodes, stage, s->nbodies, s->nnodes);
    CK(cudaGetLastError(), "pack state");
    CK(cudaMemcpyAsync(dst, stage, sizeof(double) * nd, cudaMemcpyDeviceToHost, s->stream), "read state");
    CK(cudaStreamSynchronize(s->stream), "read state sync");
    return SIM_OK;
}

int sim_write_state(sim_t s, const double *src)
{
    if (!s || !src) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    const long long nd = state_doubles(s);
    if (nd == 0) return SIM_OK;
    CK(cudaMemcpyAsync(s->d_stage, src, sizeof(double) * nd, cudaMemcpyHostToDevice, s->stream), "write state");
    const int grid = (int)std::min<long long>((nd + 255) / 256, 1024);
    unpack_state<<<grid, 256, 0, s->stream>>>(s->d_bodies, s->d_nodes, s->d_stage, s->nbodies, s->nnodes);
    CK(cudaGetLastError(), "unpack state");
    return SIM_OK;
}

int sim_sizes(sim_t s, long long out[9])
{
    if (!s || !out) return SIM_EINVAL;
    int rc = finalize(s);
    if (rc) return rc;
    out[0] = s->nscenes;
    out[1] = (long long)s->subs.size();
    out[2] = s->dof;
    out[3] = (long long)s->cons.size();
    out[4] = s->nrows;
    out[5] = s->nsr;
    out[6] = s->nbodies;
    out[7] = s->max_smem;
    out[8] = s->nnodes;
    return SIM_OK;
}

int sim_scene_info(sim_t s, int scene, long long out[4])
{
    if (!s || !out) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    if (scene < 0 || scene >= s->nscenes) return fail(s, SIM_EINVAL, "scene out of range");
    const SceneDesc &S = s->scenes[scene];
    out[0] = S.g_scene >= 0 ? 3 : S.sub_global + S.hot_global;
    out[1] = S.smem_bytes;
    out[2] = S.nsub;
    out[3] = s->work_bytes;
    return SIM_OK;
}

int sim_iteration_stats(sim_t s, long long out[5], long long *per_scene)
{
    if (!s || !out) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    if (!s->finalized) return fail(s, SIM_EINVAL, "no step has run");
    CK(cudaStreamSynchronize(s->stream), "stream synchronize");
    std::vector<long long> st((size_t)5 * std::max(1, s->nscenes));
    CK(cudaMemcpy(st.data(), s->d_stats, sizeof(long long) * 5 * s->nscenes, cudaMemcpyDeviceToHost), "stats");
    out[0] = out[1] = out[2] = out[3] = out[4] = 0;
    for (int k = 0; k < s->nscenes; ++k) {
        out[0] += st[5 * k];
        out[1] = std::max(out[1], st[5 * k + 1]);
        out[2] += st[5 * k + 2];
        out[3] += st[5 * k + 3];
        out[4] += st[5 * k + 4];
    }
    if (per_scene) std::copy(st.begin(), st.begin() + 5 * (size_t)s->nscenes, per_scene);
    CK(cudaMemset(s->d_stats, 0, sizeof(long long) * 5 * s->nscenes), "stats clear");
    return SIM_OK;
}

int sim_phase_trace(sim_t s, int enable, long long out[8])
{
    if (!s) return SIM_EINVAL;
    ON_DEVICE(s->opt.device);
    int rc = finalize(s);
    if (rc) return rc;
    const size_t bytes = sizeof(long long) * 8 * std::max(1, s->nscenes);
    if (out) {
        for (int k = 0; k < 8; ++k) out[k] = 0;
        if (s->d_phase) {
            CK(cudaStreamSynchronize(s->stream), "stream synchronize");
            std::vector<long long> v((size_t)8 * std::max(1, s->nscenes));
            CK(cudaMemcpy(v.data(), s->d_phase, bytes, cudaMemcpyDeviceToHost), "phase trace");
            for (int sc = 0; sc < s->nscenes; ++sc)
                for (int k = 0; k < 8; ++k) out[k] += v[(size_t)8 * sc + k];
        }
    }
    // a captured graph holds the tracer pointer of its capture: capture again
    if (s->graph || s->graph_learned) {
        CK(cudaStreamSynchronize(s->stream), "stream synchronize");
        drop_graphs(s);
    }
    if (enable && !s->d_phase) {
        cudaError_t e = cudaMalloc((void **)&s->d_phase, bytes);
        if (e != cudaSuccess) return fail(s, SIM_ENOMEM, "cudaMalloc phase trace");
    }
    if (enable) {
        CK(cudaMemsetAsync(s->d_phase, 0, bytes, s->stream), "phase trace clear");
    } else if (s->d_phase) {
        CK(cudaStreamSynchronize(s->stream), "stream synchronize");
        cudaFree(s->d_phase);
        s->d_phase = nullptr;
    }
    return SIM_OK;
}

const char *sim_last_error(sim_t s)
{
    return s ? s->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
