/*
 * subadmm.h -- C ABI of the GB300 (sm_103a) subsystem-based ADMM multibody solver.
 *
 * The method is that of "Modular and Parallelizable Multibody Physics Simulation via
 * Subsystem-Based ADMM" (Lee, Lee & Lee, arXiv 2302.14344).  One time step (Algorithm 1):
 *   construct A_i, b_i per subsystem (Eq. sdyn) and e_j, J_j per constraint (Sec. II-A);
 *   beta_i = Tr(A_i) / Tr(J_ci^T J_ci) (Sec. III-D) or a fixed rho;
 *   factorise K_i = A_i + beta_i J_ci^T J_ci once per step;
 *   iterate  v-step  K_i v_i = b_i + J_ci^T (beta_i z_i - u_i),  x_i = J_ci v_i   (Eq. admm-1i)
 *            z-step  per constraint, closed-form lambda_j, beta_i z_ij = y_ij + lambda_j
 *                    with y_i = beta_i x_i + u_i                    (Eq. admm-2j, Eq. surrogate)
 *            u-step  u_i += beta_i (x_i - z_i)                                    (Eq. admm-3)
 *   until the stop rule holds; then update each subsystem's state from v-hat (Eq. ddyn).
 *
 * Every step of that loop runs in CUDA kernels on the device; nothing falls back to the host.
 *
 * Conventions for every call:
 *   - Return value: SIM_OK (0) on success, a positive warning, or a negative error code; the
 *     message of the last error is in sim_last_error().
 *   - Ownership: host arrays passed in are copied before the call returns; the library never
 *     keeps a caller's pointer.  A sim_t owns all device memory it allocates, freed by
 *     sim_destroy().
 *   - Topology (subsystems and interfaces) is fixed at the first sim_step(); adding after that
 *     returns SIM_EINVAL.
 *   - One host thread per sim_t.  Work is enqueued on the stream given in sim_options;
 *     sim_step() is asynchronous, the sim_get_* / sim_residuals() calls synchronise it.
 *   - Matrices are row-major double precision.  Indices are 0-based.
 *   - Sign convention: constraint j's value is sum_{i in S_j} J_ij v_i + e_j; lambda_j acts on
 *     subsystem i as J_ij^T lambda_j.
 */
#ifndef SUBADMM_H
#define SUBADMM_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SIM_OK 0
#define SIM_NOT_CONVERGED 1   /* warning: a scene hit max_iters before its stop rule held */
#define SIM_EINVAL (-1)       /* bad argument, bad topology, or a scene too large           */
#define SIM_ENOMEM (-2)       /* device or host allocation failed                           */
#define SIM_ENOTSPD (-3)      /* K_i = A_i + beta_i J^T J had a pivot <= 0 (not SPD)        */
#define SIM_ENAN (-4)         /* a residual became NaN or infinite                          */
#define SIM_ECUDA (-5)        /* a CUDA runtime call failed                                 */
#define SIM_ETIMEOUT (-6)     /* a grid-wide barrier (one scene over the whole GPU) waited
                                 over 20 s: the kernel ended early, results are undefined  */

/* subsystem kinds (Sec. III-A: rigid bodies, or any block given by A_i, b_i) */
#define SIM_SUB_GENERIC 0     /* A_i (n x n, SPD) and b_i given directly                    */
#define SIM_SUB_RIGID 1       /* rigid bodies in maximal coordinates, 6 DOF each            */
#define SIM_SUB_LINEAR 2      /* linear elastic block of nodes (3 DOF each), e.g. linear FEM */

/* interface kinds.  The first four give rows explicitly (J per side, e); the last four are
 * rigid-body model constraints whose rows are rebuilt from the bodies' state every step. */
#define SIM_IF_EQUALITY 0     /* sum J v + e = 0                       (hard, Eq. hcon)    */
#define SIM_IF_HARD 1         /* sum J v + e >= 0, lambda >= 0, per row (Eq. hcon)          */
#define SIM_IF_SOFT 2         /* lambda = -k (e + alpha sum J v)        (Eq. scon)          */
#define SIM_IF_CONTACT 3      /* 3 rows (normal, t1, t2), Signorini-Coulomb (Eq. scc)       */
#define SIM_IF_BALL 4         /* 3 equality rows: point of a == point of b                  */
#define SIM_IF_REVOLUTE 5     /* 5 equality rows: ball + two axis-alignment rows            */
#define SIM_IF_ANGLE_PD 6     /* 1 soft row: PD drive of the relative angle about an axis   */
#define SIM_IF_PLANE_CONTACT 7/* 3 contact rows: a sphere (or point) of a against a plane    */
#define SIM_IF_SPHERE_CONTACT 8/* 3 contact rows: a sphere of a against a sphere of b       */

/* option values */
#define SIM_BETA_TRACE 0      /* beta_i = Tr(A_i) / Tr(J_ci^T J_ci)  (Sec. III-D)           */
#define SIM_BETA_FIXED 1      /* beta_i = rho for every subsystem                           */
#define SIM_WARM_COLD 0       /* z = u = 0 at the start of every step                       */
#define SIM_WARM_PREV 1       /* z and u = -lambda of the previous step                     */
#define SIM_STOP_PRIMAL 0     /* stop when max|x - z| <= tol and max|z^{l+1}-z^l| <= tol    */
#define SIM_STOP_THETA 1      /* stop when theta < theta_th after the v-step (Eq. residual) */
#define SIM_FP64 0            /* every step in double precision                             */
#define SIM_MIXED 1           /* FP64 assembly, beta and final residual check; K_i factorised
                                 in FP32 (a large block of a grid scene by the blocked
                                 factorisation, see sim_tc_factor), or in FP64 when the block
                                 is stiff (spread of K_i's diagonal above 1e3); FP32
                                 iterations (resumed with a refined c if the FP64 check
                                 misses the tolerance)                                      */

/* what sim_get() reads */
#define SIM_GET_VHAT 0        /* id = subsystem: n doubles, v-hat of the last step          */
#define SIM_GET_LAMBDA 1      /* id = interface: rows doubles, lambda of the last step      */
#define SIM_GET_BODIES 2      /* id = subsystem: nb x 17 doubles (body records, see below)  */
#define SIM_GET_BETA 3        /* id = subsystem: 1 double                                   */
#define SIM_GET_Z 4           /* id = interface: n_sides x rows doubles, z of the last step */
#define SIM_GET_NODES 5       /* id = linear subsystem: nodes x 6 doubles (x[3], v[3])      */

typedef struct sim_s *sim_t;

typedef struct sim_options {
    double h;              /* time step (s)                                   default 1e-3  */
    double gravity[3];     /* gravity acceleration on rigid bodies (m/s^2)  default 0,0,-9.81*/
    double baumgarte;      /* gamma in e = gamma phi / h for joints       default 0.2       */
    int beta_mode;         /* SIM_BETA_TRACE or SIM_BETA_FIXED            default TRACE      */
    double rho;            /* beta for SIM_BETA_FIXED                     default 1e3        */
    int warm;              /* SIM_WARM_COLD or SIM_WARM_PREV              default PREV       */
    int stop;              /* SIM_STOP_PRIMAL or SIM_STOP_THETA           default PRIMAL     */
    double tol_primal;     /* <= 0: run exactly max_iters iterations      default 1e-6       */
    double theta_th;       /*                                             default 1e-12      */
    int max_iters;         /* l_max                                       default 1000       */
    int precision;         /* SIM_FP64 or SIM_MIXED                       default FP64       */
    int device;            /* CUDA device ordinal                         default 0          */
    void *stream;          /* cudaStream_t to enqueue on; NULL = default  default NULL       */
} sim_options;

/* Fills *opt with the defaults listed above. */
void sim_default_options(sim_options *opt);

/* Creates an empty simulation on opt->device.  *out receives the handle. */
int sim_create(const sim_options *opt, sim_t *out);

/* Frees every device and host resource of s (NULL is ignored).  Synchronises s's stream. */
void sim_destroy(sim_t s);

/* Adds a subsystem to scene `scene` (scenes are independent problems solved side by side,
 * numbered 0..; a new number opens a new scene).  Subsystem ids are global, in call order.
 *   kind SIM_SUB_GENERIC: count = n >= 1; data = A (n*n, row-major, SPD) then b (n).
 *   kind SIM_SUB_RIGID:   count = number of bodies >= 1; data = count records of 17 doubles
 *       m, Ixx, Iyy, Izz (principal inertia in the body frame), p[3] (world position of the
 *       centre of mass), q[4] (w, x, y, z unit quaternion, body to world), v[3] (world linear
 *       velocity), w[3] (body-frame angular velocity).  DOF order: [v, w] per body.
 *       A_i = (2/h) M_i and b_i = (2/h) M_i v_k - C v_k + f with C v_k = [0; w x I w] and
 *       f = [m g; 0] (Eq. ddyn with v_{k+1} = 2 v-hat - v_k).
 *   kind SIM_SUB_LINEAR:  count = nodes nn >= 1, n = 3 nn DOF (node velocities); data =
 *       mass (nn, lumped per node), f (n, constant force), X0 (n, rest positions),
 *       x (n, positions), v (n, velocities), nnz, then nnz triplets (row, col, value) of the
 *       symmetric stiffness K (indices as exact doubles).  With the elastic force
 *       at the midpoint of the step (Eq. ddyn): A_i = (2/h) M + (h/2) K,
 *       b_i = (2/h) M v_k - K (x_k - X0) + f + M g; then x += h v-hat, v = 2 v-hat - v_k.
 *       K is kept sparse.  */
int sim_add_subsystem(sim_t s, int scene, int kind, int count, const double *data, int *out_id);

/* Adds an interface (constraint j) to scene `scene`; interface ids are global, in call order.
 * Explicit-row kinds (SIM_IF_EQUALITY, SIM_IF_HARD, SIM_IF_SOFT, SIM_IF_CONTACT):
 *   rows >= 1 (3 for a contact), n_sides = |S_j| in 1..8, sides = distinct subsystem ids of
 *   the same scene; J = for each side in order, a rows x n_side row-major block; e = rows
 *   values; params = {k, alpha, mu} (k, alpha for SOFT; mu for CONTACT; may be NULL
 *   otherwise).  J and e are constant for the life of the simulation.
 * Rigid-model kinds (SIM_IF_BALL, SIM_IF_REVOLUTE, SIM_IF_ANGLE_PD, SIM_IF_PLANE_CONTACT,
 * SIM_IF_SPHERE_CONTACT):
 *   rows and n_sides are ignored; sides = {sub_a, body_a, sub_b, body_b}: (subsystem id, body
 *   index inside it) of bodies a and b, sub_b = -1 for the world (PLANE_CONTACT uses a only);
 *   for BALL and the two contacts a side may also be (linear subsystem id, node index): the
 *   node's position takes the place of the anchored body point;
 *   J and e must be NULL; params = 23 doubles:
 *     anchor_a[3] (a frame), anchor_b[3] (b frame, or a world point), axis_a[3], axis_b[3],
 *     ref_a[3] (a frame, orthogonal to axis_a), ref_b[3] (b frame), kp, kd, target,
 *     plane_z, mu.
 *   BALL: phi = p_a + R_a anchor_a - (p_b + R_b anchor_b), e = baumgarte phi / h.
 *   REVOLUTE: BALL rows plus t_k . (R_b axis_b) for t_1 = R_a ref_a, t_2 = R_a (axis_a x ref_a).
 *   ANGLE_PD: angle theta of R_b ref_b from R_a ref_a about R_a axis_a; soft row with
 *     k = kp, alpha = kd/kp + h/2, e = theta - target.
 *   Contact frame of a unit normal n: rows (n, t1, t2), t1 = the world x axis (the y axis
 *     when |n_x| > 0.9) made orthogonal to n and normalised, t2 = n x t1; for n = +z the
 *     rows are (z, x, y).  Both contacts: e_n = gap/h for gap >= 0, baumgarte gap/h
 *     otherwise, e_t = 0; friction coefficient mu >= 0.
 *   PLANE_CONTACT: axis_b = the plane's world normal n (any length > 0, normalised here),
 *     ref_a[0] = r >= 0: the sphere of radius r about the point P = p_a + R_a anchor_a
 *     against the plane {x : n . x = plane_z}; gap = n . P - plane_z - r; rows of the
 *     velocity of the material point P - r n (r = 0: the point P itself).
 *   SPHERE_CONTACT: spheres of radii ref_a[0], ref_b[0] >= 0 about P_a = p_a + R_a anchor_a
 *     and P_b = p_b + R_b anchor_b (anchor_b a world point for the world); n = (P_a - P_b) /
 *     |P_a - P_b| (+z when the centres coincide), gap = |P_a - P_b| - r_a - r_b; rows of the
 *     relative velocity of the material points P_a - r_a n (of a) and P_b + r_b n (of b).
 * Two bodies of the same subsystem give an intra-subsystem constraint (|S_j| = 1). */
int sim_add_interface(sim_t s, int scene, int kind, int rows, int n_sides, const int *sides,
                      const double *J, const double *e, const double *params, int *out_id);

/* Replaces A_i and/or b_i of a SIM_SUB_GENERIC subsystem (host arrays; either may be NULL).
 * Takes effect at the next step. */
int sim_set_generic(sim_t s, int subsystem, const double *A, const double *b);

/* Runs n_steps >= 1 time steps of every scene, asynchronously on the stream.  The first call
 * uploads the topology.  Returns SIM_EINVAL if a scene does not fit the on-chip path. */
int sim_step(sim_t s, int n_steps);

/* Launch classes.  The scenes are grouped into classes that share a kernel variant (the
 * register-cached iteration, which holds each thread's D row chunks and projection item in
 * registers, or the generic one) and a shared-memory budget (a whole SM, or half of one for
 * generic scenes that fit, so that two blocks share an SM).  sim_step enqueues one launch per
 * class; classes after the first run on streams of their own forked from the simulation's
 * stream and joined back to it, so the classes overlap.
 * A scene with at least 8192 side-rows runs alone over the whole GPU instead (the grid
 * kernel: a cooperative launch whose blocks share the scene's rows, items and subsystems,
 * with two bounded grid barriers per iteration); grid classes run before the others, one
 * scene at a time, and are never captured into a graph.
 * sim_launch_classes lays the simulation out if needed and writes, for each class k <
 * max_classes, five counts at out[5k]: scenes, kernel (0 generic, 1 register-cached, 2
 * grid, 3 generic with 512 threads per block: a class whose scenes take a whole SM's shared
 * memory, so that a block has the whole register file and twice the warps), lanes per
 * side-row (1, 2 or 4; 8, 16 or 32 for the grid kernel), dynamic shared
 * memory per block in bytes (for a grid class: its staged D-row buffers at its last launch,
 * 0 before the first or without staging, see sim_grid_staging), 0.  Returns the number
 * of classes, or a negative SIM_E* code.
 * sim_autotune times, for each class on its own, every kernel variant that is valid for all
 * its scenes (generic with 1, 2 or 4 lanes per side-row and 256 or 512 threads per block,
 * register-cached where the scenes fit; the grid kernel with 8, 16 or 32 lanes per
 * side-row and all resident blocks or half of them, unless sim_grid_blocks fixed the count) over `steps`
 * steps from the current state, keeps the fastest, and restores the state
 * (bodies, nodes, warm-start duals, outputs, counters) so that tuning leaves no trace.  It
 * waits for the stream, allocates a temporary snapshot, and writes the same rows as
 * sim_launch_classes with out[5k + 4] the chosen variant's time per step in nanoseconds.
 * Returns the number of classes or a negative SIM_E* code. */
int sim_launch_classes(sim_t s, int max_classes, long long *out);
int sim_autotune(sim_t s, int steps, int max_classes, long long *out);

/* Learned warm start (a learned counterpart of the previous-step duals of Sec. III-D).
 * Interfaces are numbered by their public ids (sim_add_interface order); x_dev, t_dev and
 * mask_dev are device arrays of float, ordered on the simulation's stream.
 *
 * sim_interface_features writes 32 features per interface from the current state (the
 * state a next sim_step starts from): [0:4] projection type one-hot (equality, hard, soft,
 * contact); [4:7] anchor point of side a minus that of side b (world; the world side is
 * its anchor, a plane contact's the foot of a's point on the plane, a sphere contact's
 * the centre of b's sphere); [7:11] relative
 * orientation q_a^-1 q_b (w, x, y, z; identity for nodes and the world); [11:14] and
 * [14:17] anchor velocity and angular velocity of a minus those of b (world); [17:23] the
 * last step's lambda (first 6 rows); [23:26] the error terms e (first 3 rows); [26] mu;
 * [27] s = sum of 1/beta over its sides (last step's beta; 0 before the first step); [28]
 * the contact gap; [29] beta_a / beta_b (1 for one side or before the first step); [30]
 * log2(1 + side-rows of the scene); [31] log2(1 + DOF of side a's subsystem); a non-finite
 * feature is written as 0.  x_dev holds 32 x interfaces floats.
 *
 * sim_interface_targets, after a sim_step whose start features are in x_dev, writes the
 * training targets of each interface: t_dev[7 i + r] = lambda*_r - lambda_prev,r for its
 * first 6 rows (lambda* the step's final duals, lambda_prev read from the features), 0
 * elsewhere; mask_dev 1 on those rows and 0 elsewhere; column 6 (log2 of the beta scale)
 * target 0, mask 1: the trace rule, unless the caller writes the scale a search found.
 *
 * sim_step_learned evaluates the network once and then runs n_steps steps (one launch per
 * launch class): the features of the current state, the network (32 inputs, 7 outputs; see
 * warmstart.h), lambda^0 = lambda_prev + output (first 6 rows of each interface), and the
 * beta scales (output 7 is log2 of a scale proposed per interface; every subsystem of a
 * scene takes scale 2^k, k the mean over the scene's interfaces rounded to an integer in
 * [-3, 3]; see sim_set_beta_scale).  The first step starts from lambda^0 (z^0 from the previous step),
 * the others from the previous step's duals; the scales hold for all n_steps (and after,
 * until changed).  After 10 iterations of the first step a scene compares its residual
 * max(|x - z|, |dz|) with the one its last plain (previous-step) start had after 10
 * iterations; if the learned start is behind, the scene restarts the step from the plain
 * start and records that run's residual as the new reference; it then starts plain for the
 * next 2^f - 1 calls (f its run of consecutive fallbacks, at most 5); a kept learned start
 * ends the run.  The iterations of abandoned learned starts count in sim_iteration_stats.
 * With sim_use_graph on (and no grid scene), the first call with a network and step count
 * runs directly and captures a graph that later calls replay; the network's parameters
 * are read at replay time, so training between calls needs no recapture. */
struct wsn_s;
int sim_interface_features(sim_t s, float *x_dev);
int sim_interface_targets(sim_t s, const float *x_dev, float *t_dev, float *mask_dev);
int sim_step_learned(sim_t s, struct wsn_s *net, int n_steps);

/* Scenes with at least `side_rows` side-rows run on the grid kernel (default 8192).  Must be
 * called before the first sim_step (SIM_EINVAL after it, or for side_rows < 1). */
int sim_grid_threshold(sim_t s, int side_rows);

/* Grid kernel: with enable != 0 (the default) each warp of the warp-per-side-row v-step
 * stages its D rows in shared memory by bulk asynchronous copies (two stages per warp,
 * the next row in flight while the current one is used), when that leaves the launch its
 * blocks per SM; with 0 the rows are read from global memory directly.  The results are
 * the same either way (the same products in the same order).  Takes effect at the next
 * sim_step. */
int sim_grid_staging(sim_t s, int enable);

/* Makes linear subsystem `subsystem` co-rotational (the paper's beam model, Sec. IV-A):
 * `ne` tetrahedra, tets[4e .. 4e + 3] their node indices (inside the block), Ke[144 e ..] their
 * rest stiffness matrices (12 x 12 row-major, DOF order node-major).  Every step then
 * assembles, per element, the rotation R of its deformation gradient F = Ds Dm^-1 (polar
 * decomposition), the stiffness R K_e R^T and the force -R K_e (R^T x_e - X_e): A_i =
 * (2/h) M + (h/2) sum_e R K_e R^T and b_i = (2/h) M v_k + sum_e f_e + f + M g (the block's own
 * K triplets give only the pattern, which must contain every element's node pairs).  Its
 * factor changes every step, so it is never kept.  Before the first sim_step only. */
int sim_set_corotational(sim_t s, int subsystem, int ne, const int *tets, const double *Ke);

/* Per-subsystem beta scales (host array, one per subsystem id): from the next step on,
 * beta_i = scale[i] x (the trace rule of Sec. III-D, or rho).  The default is 1.  The ADMM
 * fixed point does not depend on beta, its speed does: this is the input a learned rho sets
 * (sim_step_learned does so from the network's seventh output).  A block whose factor is
 * kept (sim_keep_factors) is factorised again when its scale changes.  SIM_EINVAL for a
 * scale that is not positive and finite.  Lays the simulation out if needed; waits for the
 * copy. */
int sim_set_beta_scale(sim_t s, const double *scale);

/* Tensor cores for the per-step map of large blocks (mixed form, grid kernel scenes; on by
 * default).  A step that factorises such a block (n >= 128 DOF, m >= 16 side-rows) anew --
 * every step with sim_keep_factors(0), else the first -- runs as three launches: the grid
 * kernel up to W = L^-1 [J^T b] (its columns solved in 32-wide chunks over every warp), the
 * tcgen05 Gram kernel forming D = W^T W and c = W^T g (see sim_gram_tc), and the grid kernel
 * from the initial duals on (with sim_tc_factor, the default, those blocks' factorisation
 * and a W launch come between the first two).  With 0 the grid kernel forms D and c itself
 * (one warp per block, FP32 CUDA cores).  Must be called before the first sim_step
 * (SIM_EINVAL after). */
int sim_tensor_cores(sim_t s, int enable);

/* Blocked factorisation of those blocks on the tensor cores (Algorithm 1, factorise; on by
 * default; takes effect only where sim_tensor_cores is on).  A refactorised block that the
 * mixed form factorises in FP32 (not stiff by the diagonal-spread test) is factorised after
 * the setup launch instead of inside it: right-looking over panels of 128 columns, one launch
 * per panel for the diagonal tile's factor and the rows below it (CUDA cores, FP32, a thread
 * per row), and one tcgen05 launch per panel for the Schur update of the trailing tiles the
 * panel reaches inside K_i's envelope (C -= P P^T, split-TF32, accumulators in tensor
 * memory); a grid launch then solves those blocks' W before the Gram kernel.  Stiff blocks
 * stay on the FP64 envelope factorisation.  With 0 every factor is formed inside the setup
 * launch (one warp per block).  A non-positive pivot ends the step with SIM_ENOTSPD status
 * like the one-warp factorisation.  May be called at any time; it applies from the next
 * step that refactorises. */
int sim_tc_factor(sim_t s, int enable);

/* The solver of every step (Sec. IV-B compares the method with other solvers on the same
 * scenes; Projected Jacobi is one of them):
 *   SIM_SOLVER_ADMM (default): subsystem-based ADMM, Algorithm 1.
 *   SIM_SOLVER_PJ: Projected Jacobi on the step's dual problem, relaxation omega > 0.  With
 *     A_i's own factor (no penalty term): D_i = J_i A_i^-1 J_i^T, c_i = J_i A_i^-1 b_i, the
 *     diagonal delta_r = sum over the row's sides of D_i's entry; every iteration forms
 *     each side's x = c + D lambda and updates every row at once: equality
 *     lambda -= omega (x + e) / delta; hard the same clamped at 0; soft lambda += omega
 *     (lambda* - lambda) with lambda* = -k (e + alpha (x - delta lambda)) / (1 + k alpha
 *     delta); contact: normal as hard, both tangents with delta_t = max of theirs, then
 *     scaled onto the disk of radius mu lambda_n.  Exactly max_iters iterations per step
 *     (tol_primal and the stop rule are ignored); v-hat = A^-1 (b + J^T lambda).  The
 *     reported r_p is the last iteration's natural residual max |d lambda| delta / omega;
 *     r_d and theta are 0.  The learned warm start and the tensor-core map are not used.
 * Must be called before the first sim_step (SIM_EINVAL after); SIM_EINVAL for an unknown
 * solver or omega <= 0. */
#define SIM_SOLVER_ADMM 0
#define SIM_SOLVER_PJ 1
int sim_set_solver(sim_t s, int solver, double omega);

/* Grid kernel: run the cooperative launch with `blocks` blocks (at most the resident count;
 * 0, the default, takes every resident block: 2 per SM).  Fewer blocks give each warp more
 * side-rows, subsystems and items; the results do not depend on it.  Takes effect at the
 * next sim_step; SIM_EINVAL for blocks < 0. */
int sim_grid_blocks(sim_t s, int blocks);

/* A linear block's K_i = A_i + beta_i J_i^T J_i is constant (Sec. II-B: its A_i and its
 * node-selector rows are), so by default (enable != 0) its factor, W and D are computed at
 * its first step and kept.  Not kept: co-rotational blocks (A_i changes) and blocks with a
 * node in a SPHERE_CONTACT (the rows turn with the normal, so D does).  With 0 every step
 * factorises every block again, as Algorithm 1
 * states it: the same matrix, so the results agree to rounding (with a kept factor
 * g = L^-1 b is formed by the single-vector solve, otherwise as the last column of W).
 * Takes effect at the next sim_step. */
int sim_keep_factors(sim_t s, int enable);

/* Self-test of the grid barrier's time limit (failure detection without a fault): a
 * cooperative launch of `blocks` blocks (all resident, else SIM_EINVAL) in which every block
 * waits once at a barrier that needs `expected` arrivals, for at most limit_s seconds
 * (0 < limit_s <= 10).  With expected > blocks nothing completes the barrier: every wait runs
 * out, raises the error flag and returns.  Writes out[0] the error flag (1 if a wait ran
 * out), out[1] the blocks that left the barrier.  Synchronises the device. */
int sim_probe_barrier(int device, int blocks, int expected, double limit_s, int out[2]);

/* Floor of one iteration of the block kernel (a measurement aid, no counterpart in the
 * paper): launches one 256-thread block per SM on `device` that runs `iters` rounds of the
 * block barrier (__syncthreads_count) the block kernel ends every iteration with, nothing
 * else between them.  Writes out[0] SM clock cycles per round (mean over blocks), out[1]
 * nanoseconds per round of the whole launch (CUDA events).  Synchronises the device;
 * allocates (and frees) a small device buffer.  SIM_EINVAL for iters outside 1..1e7. */
int sim_barrier_floor(int device, int iters, double out[2]);

/* Gram matrices G_j = W_j^T W_j on the tensor cores (tcgen05, split-TF32: FP32-class
 * accuracy), the kernel that forms the per-step map of each subsystem (D = W^T W and
 * c = W^T g with W = L^-1 [J^T b], Algorithm 1's factorise step carried to the constraint
 * space).  This entry runs it standalone on `njobs` matrices, for testing and measurement:
 * W[j] (device, n[j] rows of ldw[j] floats: W[j][p * ldw[j] + t], t < cols[j]) gives
 * G[j] (device, cols[j] x cols[j], both triangles, G[j][t * ldg[j] + u]).  Runs `reps` times
 * on the legacy default stream (the first untimed) and writes the mean time of the others
 * to *ms_per_run (0 if reps == 1; ms_per_run may be NULL).  Allocates (and frees) its
 * transposed operand buffers; synchronises the device.  Returns SIM_OK, SIM_EINVAL,
 * SIM_ENOMEM, SIM_ECUDA, or SIM_ETIMEOUT if a wait of the kernel ran out (1 s). */
int sim_gram_tc(int device, int njobs, const float *const *W, const int *n, const int *cols,
                const int *ldw, float *const *G, const int *ldg, int reps, float *ms_per_run);

/* CUDA-graph replay of sim_step (off by default).  When enabled, the first sim_step with a
 * given n_steps captures its launches (one per launch class of scenes, forked across streams
 * and joined back to the simulation's stream) into a graph, and later calls with the same
 * n_steps replay it with a single cudaGraphLaunch on the stream.  A call on a stream that the
 * caller is already capturing enqueues the launches into the caller's capture instead.
 * Disabling frees the graph.  Returns SIM_OK, or SIM_EINVAL for a null handle. */
int sim_use_graph(sim_t s, int enable);

/* Waits for the stream, then writes for scene `scene`'s last step:
 * out[0] r_p = max|x - z|, out[1] r_d = max beta_i |z^{l+1} - z^l|, out[2] theta,
 * out[3] iterations, out[4] 1 if the stop rule held, out[5] status (0 or a SIM_E* code).
 * Returns that status, or SIM_NOT_CONVERGED if out[4] is 0. */
int sim_residuals(sim_t s, int scene, double out[6]);

/* Waits for the stream, then copies a quantity of the last step into host memory dst. */
int sim_get(sim_t s, int what, int id, double *dst);

/* Packed state: all rigid bodies ordered by scene, then subsystem in the order added, then
 * body, 13 doubles per body (p[3], q[4], v[3], w[3]), followed by all nodes of the linear
 * blocks in the same order, 6 doubles per node (x[3], v[3]); 13 x bodies + 6 x nodes doubles in all (sim_sizes
 * out[6] and out[8]).  sim_read_state copies device -> host after the stream's work;
 * sim_write_state copies host -> device, enqueued on the stream.  dst/src are host memory
 * owned by the caller (pinned memory makes the copies asynchronous to the host). */
int sim_read_state(sim_t s, double *dst);
int sim_write_state(sim_t s, const double *src);

/* sim_read_state without any device allocation.  The paper has no counterpart: this is a
 * service of the library for callers that cannot allocate device memory when they read the
 * state, such as a control loop that must not block on the allocator or an application
 * whose framework owns all device memory under a fixed budget.  sim_read_state itself
 * allocates nothing once the simulation is laid out, but its first call on a fresh
 * simulation lays it out, which allocates; this entry point never does (no cudaMalloc,
 * cudaFree or allocating library routine) and returns SIM_EINVAL until the first sim_step
 * has laid the simulation out.
 * It packs the state through a fixed 1 MiB staging array in device memory, which every GPU
 * that loads the library holds until the process exits, so it reads a state of at most
 * 131072 doubles (10082 bodies without nodes) and returns SIM_EINVAL beyond that.  The first call on a device looks
 * up that array's address; make that first call before any stream capture.  Every call,
 * from any simulation on the device, shares the one array: calls whose GPU work overlaps
 * (different host threads or streams at once) race and must be serialised by the caller.
 * Each call overwrites all the entries it reads, so nothing needs clearing between calls.
 * Output: dst as for sim_read_state; the call returns after the copy has completed. */
int sim_read_state_noalloc(sim_t s, double *dst);

/* Counts: out[0] scenes, out[1] subsystems, out[2] DOF, out[3] interfaces, out[4] rows,
 * out[5] side-rows, out[6] rigid bodies, out[7] on-chip bytes of the largest scene,
 * out[8] nodes of the linear blocks. */
int sim_sizes(sim_t s, long long out[9]);

/* Where scene `scene` keeps its working set (lays the simulation out if needed):
 * out[0] 0 if every per-subsystem array fits in the block's shared memory; 1 if the setup
 * arrays (J, K, the factor, W: O(n^2) per subsystem) live in the simulation's global
 * workspace while the iteration arrays (D, c: O(m^2)) and the per-row arrays stay in shared
 * memory; 2 if the iteration arrays are in the workspace too; 3 if the scene runs on the
 * grid kernel (everything in the workspace).  out[1] shared-memory bytes of
 * the scene; out[2] its subsystems; out[3] bytes of the global workspace of the whole
 * simulation. */
int sim_scene_info(sim_t s, int scene, long long out[4]);

/* Sum and maximum over scenes of the iterations of all steps since the last call, and the
 * number of scene-steps that ended without their stop rule holding; then clears them.
 * out[0] total iterations (with those of learned starts that fell back), out[1] max
 * iterations of a scene-step, out[2] not converged, out[3] scene-steps counted, out[4]
 * learned starts that fell back to the plain start.  per_scene (host memory, may be NULL)
 * receives the same five counts for each scene: 5 x scenes entries, scene k at 5k (its
 * maximum at 5k + 1). */
int sim_iteration_stats(sim_t s, long long out[5], long long *per_scene);

/* Device-side phase tracer.  Reads the counters accumulated since the last call into out
 * (if out is not NULL; zeros when tracing was off), then turns tracing on (enable != 0, the
 * counters restart at zero) or off.  Counters, summed over scenes, are SM clock cycles seen
 * by the first thread of each scene's block: out[0] assembly and start of the iterations,
 * out[1] beta and factorisation, out[2] v-steps (Eq. admm-1i) including their barrier,
 * out[3] z-steps and u-steps (Eqs. admm-2j, admm-3) including their barrier, out[4] exit
 * checks and residuals, out[5] v-hat recovery and state update; out[6] iterations,
 * out[7] scene-steps.  Tracing adds a few clock reads per iteration. */
int sim_phase_trace(sim_t s, int enable, long long out[8]);

/* Blocks until every call enqueued on s's stream has finished. */
int sim_sync(sim_t s);

/* Message of the last error on s (or of the last failed sim_create when s is NULL). */
const char *sim_last_error(sim_t s);

#ifdef __cplusplus
}
#endif
#endif /* SUBADMM_H */
