// Device-side description of a batch of scenes, built once by the host runtime when the
// topology is fixed and read by the step kernel.  Internal to libsubadmm.
#pragma once

#define SUBADMM_MAXS 8          // most sides one constraint may have (|S_j|)
#define SUBADMM_THREADS 256     // threads of one scene's block
#define SUBADMM_WARPS (SUBADMM_THREADS / 32)
#define SUBADMM_WIDE 512        // threads of the wide block-kernel variant (one block per SM)
#define SUBADMM_MAXWARPS (SUBADMM_WIDE / 32)
#define SUBADMM_MAXN 2048       // largest subsystem DOF
#define SUBADMM_MAXM 2048       // largest side-row count of one subsystem
#define SUBADMM_PARAMS 23       // doubles of a rigid-model constraint's parameters
#define SUBADMM_BODY 17         // doubles of a body record

// constraint sources (how the rows are obtained) -- values of the public SIM_IF_* kinds
enum { SRC_EQUALITY = 0, SRC_HARD = 1, SRC_SOFT = 2, SRC_CONTACT = 3, SRC_BALL = 4,
       SRC_REVOLUTE = 5, SRC_ANGLE_PD = 6, SRC_PLANE = 7, SRC_SPHERE = 8 };
// projection types (Sec. III-C)
enum { TYPE_EQUALITY = 0, TYPE_HARD = 1, TYPE_SOFT = 2, TYPE_CONTACT = 3 };
// subsystem kinds
enum { KIND_GENERIC = 0, KIND_RIGID = 1, KIND_LINEAR = 2 };
#define SUBADMM_NODE 6          // doubles of a node state record: x[3], v[3]
// phase counters (clock64 cycles seen by thread 0 of a scene's block)
enum { PHASE_ASSEMBLE = 0, PHASE_FACTOR = 1, PHASE_VSTEP = 2, PHASE_ZSTEP = 3, PHASE_EXIT = 4,
       PHASE_RECOVER = 5, PHASE_ITERS = 6, PHASE_STEPS = 7 };
// per-scene status words
enum { ST_OK = 0, ST_NOTSPD = -3, ST_NAN = -4, ST_TIMEOUT = -6 };

// One scene: a set of subsystems and constraints solved by one thread block.  The on-chip
// working set lives in dynamic shared memory: a double region (factors), a region of the
// iteration type T, and an int region (tables).  Offsets are in elements of each region.
struct SceneDesc {
    int sub0, nsub;        // global subsystem range
    int con0, ncon;        // global constraint range
    int nsr, nrow;         // side-rows and rows of the scene
    int nitem, nlist;      // projection items (a row, or a whole contact) and their side lists
    int max_sides;         // most sides of one constraint of the scene
    // register-cached iteration: ipool offset of the thread map for 1, 2 and 4 lanes per
    // side-row (-1: the scene's items do not pack into one block that way).  Entry of
    // thread k: int2 {side-row (-1: idle), leader lane | slot << 5 | group lane << 8 |
    // item << 11}
    int fmap_off[3];
    // grid kernel: bytes of one staged D row (the longest row, whole 16-byte vectors)
    int row_bytes;
    int item_g0, list_g0;  // global offsets of the scene's item / list tables
    int nasm, asm_g0;      // assembly slots (constraint indices grouped by kind, -1 = idle)
    // ipool offset of three prefix sums over the subsystems (nsub + 1 each): chunks of 32
    // columns of W, items of c, items of D (the setup's scene-wide work lists)
    int pre_off;
    int ord_off;           // ipool offset: the subsystems in decreasing order of per-warp setup
                           // work (the order the per-warp loops take them in)
    int sr_g0, row_g0;     // global offset of the scene's side-rows / rows (z, lambda state)
    // double region
    int od_beta;           // beta per subsystem
    int od_flag;           // mixed form: 1 if the subsystem was factorised in FP64
    // T region (element offsets)
    int ot_x, ot_y, ot_z, ot_yo, ot_zo, ot_w0, ot_w1, ot_invb, ot_b;  // per side-row
    int ot_lam, ot_e, ot_invs, ot_kf, ot_al, ot_mu;              // per row
    // byte offsets of the T and int regions; total bytes
    int t_base, i_base, smem_bytes;
    // per-subsystem arrays: in shared memory (sub_global = 0, offsets in the regions above)
    // or in the global workspace at byte g_base (doubles) and g_base + g_tbase (T).  The
    // iteration arrays D and c stay in the T region of shared memory unless hot_global, when
    // they follow the others in the workspace.
    int sub_global, hot_global;
    long long g_base, g_tbase;
    // grid kernel: the scene arrays and tables (shared memory in the block kernel) live in
    // the workspace at byte g_scene (-1: block kernel)
    long long g_scene;
};

struct SubDesc {
    int kind, n, m;        // DOF, side-rows (rows of J_ci)
    int mpad;              // m rounded up to a whole 16-byte vector of the iteration type
    int ldd;               // row stride of D (mpad, or mpad + one vector to keep it odd)
    int sr0;               // scene-local first side-row (16-byte aligned in the T region)
    int local;             // index inside its scene
    int body0, nb;         // first global body (rigid) or node (linear), and their count
    int gen_off;           // pool offset of A (n*n) then b (n) (generic); of mass (nb), f (n),
                           // X0 (n), K values (linear)
    int csr_off;           // linear: ipool offset of the K row pointers (n+1), then columns
    int env_off;           // ipool offset of the profile of K_i: env (n), lastr (n), jlo (m), jhi (m)
    int grp_off, ngrp;     // ipool offset of the row groups of J_ci: maximal runs of consecutive
                           // rows with one column span, as ngrp + 1 first rows (the last = m)
    int cst;               // 1 if K_i is the same at every step (its factor may be kept)
    int od_J, od_L, od_b;  // double region: J_ci rows (m x n), K then its factor L (n x n), b (n)
    int od_v, od_id;       // double region: v-hat (n); 1 / L_pp (FP64 factor) or rhs (mixed) (n)
    int od_t;              // double region: J v in the mixed refinement (m)
    int ot_L, ot_W;        // T region: L (n x n, 1/L_pp on the diagonal); W = L^-1 [J^T b]
                           // (n x (m + 1), column-major: W[p (m + 1) + t], column m = g)
    int ot_s;              // T region: solve vector of the mixed recovery (n)
    int ot_D, ot_c;        // iteration region: D (m rows of mpad, ldd apart), c (m)
    int v_off;             // global offset of v-hat
    int ne, tet_off, ke_off;   // co-rotational linear block: elements, ipool offset of their
                               // 4 node indices each, pool offset of their 12 x 12 rest
                               // stiffness matrices (ne = 0: the constant linear model)
    int tc;                // grid scenes, mixed form: when refactorised, W's columns are solved
                           // by all warps and D, c formed by the tensor-core Gram kernel
};

struct ConDesc {
    int src, type, rows, ns;
    int row0;              // scene-local first row (lambda, e)
    int par_off;           // pool offset: model params (23), or k, alpha, mu, e[rows], J blocks
    int sub[SUBADMM_MAXS]; // scene-local subsystem of each side
    int sr[SUBADMM_MAXS];  // scene-local side-row of row 0 of each side
    int ba, bb;            // model: body index inside its subsystem (column block 6*ba)
    int gb_a, gb_b;        // model: global body or node index of a and b (-1: the world)
    int node_a, node_b;    // model: 1 if that side is a node of a linear block
    int side_b;            // model: side that holds body b (-1 for the world)
};

// One z-step work item: a row of an equality / hard / soft constraint, or a whole contact
// (type -1: an idle slot that aligns the next type's items to a warp).
// list[lo .. lo+ns) holds the scene-local side-row of each side (row 0 for a contact).
struct Item {
    int type, ns, row, lo;
};

// Scratch of the grid kernel (one scene over the whole grid) in global memory, zeroed
// before every launch: the barrier, the scene status, and the reduction slots.
struct GridScratch {
    unsigned count, gen;           // grid barrier
    int err;                       // a barrier wait timed out
    int status;                    // ST_* of the step
    unsigned long long umax[3];    // per iteration: max(|x - z|, |dz|) bits (rotating slots)
    double theta[3];               // per iteration: theta (rotating slots)
    double tsum;                   // exit residuals: theta, max |x - z|, max beta |dz| (bits)
    unsigned long long pmax, dmax;
    unsigned long long chk;        // mixed form: FP64 max |J v - z| (bits)
};

struct StepParams {
    int pj;                // 1: Projected Jacobi (the comparison solver) instead of ADMM
    double pj_omega;       // its relaxation factor
    const SceneDesc *scenes;
    const int *scene_ids;  // the scenes of this launch (indices into scenes)
    const SubDesc *subs;
    const ConDesc *cons;
    const Item *items;
    const int *lists;
    const int *asm_order;  // per scene: constraint index of each assembly slot
    const double *pool;    // constant data and generic A, b
    double *work;          // per-subsystem arrays of scenes too large for shared memory
    double *bodies;        // 17 doubles per body (state in and out)
    double *nodes;         // 6 doubles per node of linear blocks (state in and out)
    const int *ipool;      // integer constant data (sparse K of linear blocks, profiles)
    int *subflag;          // per subsystem: bit 0 its kept factor is valid, bit 1 it is FP64
    int *pending;          // per subsystem, this step (set by the factorisation loop of the
                           // setup): 4 its factor is left to the blocked factorisation, then
                           // W, D and c; 3 W, D and c are to be formed; 2 D and c; 1 only c;
                           // 0 none (or a failed factorisation); -1 not set yet
    int keep_factors;      // 0: refactor constant blocks every step too (Algorithm 1 literally)
    int tc_phase;          // grid kernel: 0 the whole step; 1 up to the map's W (the Gram
                           // kernel forms D, c of the tc subsystems next); 2 from the duals on;
                           // 3 only the W of the subsystems whose factor was deferred
    int tc_factor;         // tc_phase 1: the FP32 factors of the tc subsystems are left to the
                           // blocked tensor-core factorisation (step flag 4), run before phase 3
    double *vhat;          // per DOF
    double *lam;           // per row: lambda of the last step (warm start state)
    const double *lam0;    // per row: learned initial lambda of this step (NULL: not learned)
    unsigned long long *ref10;   // per scene: bits of the residual after 10 iterations of the
                                 // last plain start (the learned start's reference)
    int *learn_skip;       // per scene: steps left to start plain, and the fallback streak
    double *z;             // per side-row: z of the last step (warm start state)
    double *beta;          // per subsystem
    const double *beta_scale;  // per subsystem: beta = scale x (trace rule or rho)
    double *beta_used;     // per subsystem: the scale a kept factor was computed with
    double *res;           // 6 per scene
    long long *stats;      // 5 per scene: sum iters, max iters, not converged, steps,
                           // fallbacks of the learned start
    long long *phase;      // 8 per scene (or null): SM clock cycles per phase, see PHASE_*
    GridScratch *grid;     // grid kernel scratch
    int grid_stage;        // grid kernel: bytes per staged D row in shared memory (filled
                           // by bulk copies), 0: rows read directly
    int grid_nstage;       // grid kernel: staged rows per warp (2 to 4)
    int nscenes;           // scenes of this launch
    int n_steps;
    double h, g0, g1, g2, gamma, rho, tol, theta_th;
    int beta_fixed, warm_prev, stop_theta, max_iters;
};
