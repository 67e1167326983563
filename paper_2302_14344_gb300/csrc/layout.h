// Device-side description of a batch of scenes, built once by the host runtime when the
// topology is fixed and read by the step kernel.  Internal to libsubadmm.
#pragma once

#define SUBADMM_MAXS 8          // most sides one constraint may have (|S_j|)
#define SUBADMM_THREADS 256     // threads of one scene's block
#define SUBADMM_WARPS (SUBADMM_THREADS / 32)
#define SUBADMM_MAXN 64         // largest subsystem DOF of the on-chip path
#define SUBADMM_MAXM 96         // largest side-row count of one subsystem (on-chip path)
#define SUBADMM_PARAMS 23       // doubles of a rigid-model constraint's parameters
#define SUBADMM_BODY 17         // doubles of a body record

// constraint sources (how the rows are obtained) -- values of the public SIM_IF_* kinds
enum { SRC_EQUALITY = 0, SRC_HARD = 1, SRC_SOFT = 2, SRC_CONTACT = 3, SRC_BALL = 4,
       SRC_REVOLUTE = 5, SRC_ANGLE_PD = 6, SRC_PLANE = 7 };
// projection types (Sec. III-C)
enum { TYPE_EQUALITY = 0, TYPE_HARD = 1, TYPE_SOFT = 2, TYPE_CONTACT = 3 };
// subsystem kinds
enum { KIND_GENERIC = 0, KIND_RIGID = 1 };
// per-scene status words
enum { ST_OK = 0, ST_NOTSPD = -3, ST_NAN = -4 };

// One scene: a set of subsystems and constraints solved by one thread block.  The on-chip
// working set lives in dynamic shared memory at the offsets below (in doubles, then ints).
struct SceneDesc {
    int sub0, nsub;        // global subsystem range
    int con0, ncon;        // global constraint range
    int nsr, nrow;         // side-rows and rows of the scene
    int sr_g0, row_g0;     // global offset of the scene's side-rows / rows (z, lambda state)
    // shared-memory offsets (doubles)
    int o_x, o_y, o_z, o_w0, o_w1, o_lam, o_e, o_beta;
    int o_int;             // first int slot (after all doubles): side-row -> row, -> subsystem
    int smem_bytes;
};

struct SubDesc {
    int kind, n, m;        // DOF, side-rows (rows of J_ci)
    int sr0;               // scene-local first side-row of this subsystem
    int local;             // index inside its scene
    int body0, nb;         // first global body, body count (rigid)
    int gen_off;           // pool offset of A (n*n) then b (n) (generic)
    int o_W, o_L, o_D, o_b, o_c;   // shared-memory offsets (doubles)
    int v_off;             // global offset of v-hat
};

struct ConDesc {
    int src, type, rows, ns;
    int row0;              // scene-local first row (lambda, e)
    int par_off;           // pool offset: model params (23), or k, alpha, mu, e[rows], J blocks
    int sub[SUBADMM_MAXS]; // scene-local subsystem of each side
    int sr[SUBADMM_MAXS];  // scene-local side-row of row 0 of each side
    int ba, bb;            // model: body index inside its subsystem (column block 6*ba)
    int gb_a, gb_b;        // model: global body index of a and b (-1: the world)
    int side_b;            // model: side that holds body b (-1 for the world)
};

struct StepParams {
    const SceneDesc *scenes;
    const SubDesc *subs;
    const ConDesc *cons;
    const double *pool;    // constant data and generic A, b
    double *bodies;        // 17 doubles per body (state in and out)
    double *vhat;          // per DOF
    double *lam;           // per row: lambda of the last step (warm start state)
    double *z;             // per side-row: z of the last step (warm start state)
    double *beta;          // per subsystem
    double *res;           // 6 per scene
    long long *stats;      // 4 per scene: sum iters, max iters, not converged, steps
    int nscenes;
    int n_steps;
    double h, g0, g1, g2, gamma, rho, tol, theta_th;
    int beta_fixed, warm_prev, stop_theta, max_iters;
};
