/*
 * oracle.c -- plain, slow FP64 CPU oracle of subsystem-based ADMM multibody simulation
 * (Lee, Lee & Lee, "Modular and Parallelizable Multibody Physics Simulation via
 * Subsystem-Based ADMM", arXiv 2302.14344).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header, table or helper
 * with the CUDA library, and it includes nothing from it.
 *
 * What it computes, in the paper's order (Algorithm 1), for one scene:
 *   construct A_i, b_i                         (Eq. ddyn -> Eq. sdyn; rigid bodies below)
 *   construct e_j, J_j                         (Sec. II-A: soft, hard, contact rows)
 *   beta_i = Tr(A_i) / Tr(J_ci^T J_ci)         (Sec. III-D), or a fixed rho, times a
 *                                              per-subsystem scale (input, default 1)
 *   factorise K_i = A_i + beta_i J_ci^T J_ci   (plain Cholesky, no pivoting)
 *   loop l = 0 .. l_max-1
 *     v-step   K_i v_i = b_i + J_ci^T (beta_i z_i - u_i)      (Eq. admm-1i)
 *              x_i = J_ci v_i,  y_i = beta_i x_i + u_i          (Eq. surrogate)
 *     theta    = sum_i |y_i^{l+1} - y_i^l|^2                    (Eq. residual)
 *     z-step   per constraint j: lambda_j from the closed forms of Sec. III-C, then
 *              beta_i z_ij = y_ij + lambda_j                    (Eq. surrogate)
 *     u-step   u_i += beta_i (x_i - z_i)                        (Eq. admm-3)
 *     r_p = max |x - z|, r_d = max beta_i |z^{l+1} - z^l|       (Boyd's residuals)
 *   update each subsystem state from v-hat                      (Eq. ddyn)
 *
 * Readings where the paper is silent or garbled:
 *   - A_i = (2/h) M_i and b_i = (2/h) M_i v_k - C v_k + f: Eq. ddyn with
 *     v_{k+1} = 2 v-hat - v_k substituted; lambda is in force units.
 *   - Soft: lambda = -k (e + alpha q) / (1 + s alpha k) with q = sum beta_i^-1 y_i and
 *     s = sum beta_i^-1 (the printed formula has an unbalanced parenthesis).
 *   - Contact: with lambda* = -(q + e)/s, lambda_n = max(0, lambda*_n) and the tangent
 *     lambda*_t scaled onto the disk of radius mu lambda_n: the exact solution of
 *     Eq. contact12 under the isotropic metric s I (open / stick / slip cases).
 *   - Stop rule "primal": r_p = max|x - z| <= tol and max|z^{l+1} - z^l| <= tol after the
 *     u-step (both in constraint-velocity units; tol <= 0: exactly l_max iterations).  The
 *     second test is Boyd's dual residual divided by beta: without it an open contact seen
 *     twice in a row has x = z exactly while v is still moving.  Stop rule "theta":
 *     theta < theta_th after the v-step, from l >= 1.
 *   - Baumgarte error e = gamma phi / h for joints; contact normal e_n = gap/h for an
 *     open gap, gamma gap/h for penetration; tangential e = 0.
 *
 * Rounding: build with -O2 -ffp-contract=off (no fused multiply-add).
 *
 * Threads: the plain build is single-threaded.  Built with -fopenmp (the benchmark's
 * multi-core timing baseline only, as the paper times its own solver with OpenMP) the
 * factorisation and v-step run one subsystem per thread and the constraint loops one
 * constraint per thread; every per-element result is the same, only the order of theta's
 * sum differs.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXSIDES 8

enum { T_EQUALITY = 0, T_HARD = 1, T_SOFT = 2, T_CONTACT = 3 };
enum { SRC_ROWS = 0, SRC_BALL = 1, SRC_REVOLUTE = 2, SRC_ANGLE_PD = 3, SRC_PLANE = 4,
       SRC_SPHERE = 5 };
enum { SUB_GENERIC = 0, SUB_RIGID = 1, SUB_LINEAR = 2 };

typedef struct {
    double m, I[3], p[3], q[4], v[3], w[3];
} body_t;

typedef struct {
    int kind, n, nb;           /* nb: bodies (rigid) or nodes (linear) */
    body_t *bodies;
    double *mass, *Kel, *fext, *X0, *x, *vel;   /* linear: per node mass, K (n x n), f,
                                                   rest, position, velocity (n each) */
    double *A, *b;   /* n*n, n */
    double *L;       /* Cholesky factor of K (lower, row-major n*n) */
    double *v;       /* v-hat */
    double *rhs;
    double beta;
    double beta_scale;         /* multiplies the trace rule's (or the fixed) beta; 1 default */
    int ne;                    /* co-rotational linear block: elements (0: linear model) */
    int *tets;                 /* 4 node indices per element */
    double *Ke;                /* rest stiffness per element (12 x 12, row-major) */
} sub_t;

typedef struct {
    int src, type, rows, ns;
    int sub[MAXSIDES];
    double *J[MAXSIDES];  /* rows x n_sub, row-major */
    double *e;
    double k, alpha, mu;
    /* rigid-model parameters */
    int sa, ba, sb, bb;
    double anc_a[3], anc_b[3], ax_a[3], ax_b[3], ref_a[3], ref_b[3];
    double kp, kd, target, plane_z;
    /* iteration state per side-row, index s*rows + r */
    double *x, *z, *u, *y, *yold, *zold, *zprev;
    double *lam, *lamprev;
    int has_prev;
} con_t;

typedef struct orc_scene {
    double h, g[3], gamma, rho, tol, theta_th;
    int beta_fixed, warm_prev, stop_theta, max_iters;
    int pj;                    /* 1: the step runs Projected Jacobi instead of ADMM */
    double pj_omega;           /* its relaxation factor */
    int nsub, ncon, capsub, capcon;
    sub_t *subs;
    con_t *cons;
    /* last solve */
    int iters, converged, status;
    double r_p, r_d, theta;
    double *trace;
    int trace_cap;
} orc_scene;

/* ------------------------------------------------------------------------------------ */
/* small dense helpers                                                                   */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* plain Cholesky K = L L^T; returns 0 on success, -1 on a pivot <= 0 or non-finite */
static int cholesky(int n, const double *K, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j <= i; j++) {
            double s = K[i * n + j];
            for (int k = 0; k < j; k++) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0) || !isfinite(s)) return -1;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    }
    return 0;
}

/* solve L L^T x = r in place */
static void chol_solve(int n, const double *L, double *x)
{
    for (int i = 0; i < n; i++) {
        double s = x[i];
        for (int k = 0; k < i; k++) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

static void quat_to_mat(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void matvec3(const double R[9], const double a[3], double out[3])
{
    for (int i = 0; i < 3; i++) out[i] = R[3 * i] * a[0] + R[3 * i + 1] * a[1] + R[3 * i + 2] * a[2];
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* row vector c^T R (i.e. R^T c) */
static void rowtimesR(const double c[3], const double R[9], double out[3])
{
    for (int j = 0; j < 3; j++) out[j] = c[0] * R[j] + c[1] * R[3 + j] + c[2] * R[6 + j];
}

/* ------------------------------------------------------------------------------------ */
/* construction                                                                          */

orc_scene *orc_new(const double *o)
{
    orc_scene *S = (orc_scene *)xcalloc(1, sizeof(orc_scene));
    S->h = o[0]; S->g[0] = o[1]; S->g[1] = o[2]; S->g[2] = o[3];
    S->gamma = o[4];
    S->beta_fixed = (int)o[5];
    S->rho = o[6];
    S->warm_prev = (int)o[7];
    S->stop_theta = (int)o[8];
    S->tol = o[9];
    S->theta_th = o[10];
    S->max_iters = (int)o[11];
    return S;
}

static sub_t *new_sub(orc_scene *S)
{
    if (S->nsub == S->capsub) {
        S->capsub = S->capsub ? 2 * S->capsub : 8;
        S->subs = (sub_t *)realloc(S->subs, sizeof(sub_t) * S->capsub);
    }
    sub_t *u = &S->subs[S->nsub++];
    memset(u, 0, sizeof(*u));
    u->beta_scale = 1.0;
    return u;
}

static void sub_alloc(sub_t *u)
{
    int n = u->n;
    u->A = (double *)xcalloc((size_t)n * n, sizeof(double));
    u->b = (double *)xcalloc(n, sizeof(double));
    u->L = (double *)xcalloc((size_t)n * n, sizeof(double));
    u->v = (double *)xcalloc(n, sizeof(double));
    u->rhs = (double *)xcalloc(n, sizeof(double));
}

int orc_add_generic(orc_scene *S, int n, const double *A, const double *b)
{
    if (n <= 0) return -1;
    sub_t *u = new_sub(S);
    u->kind = SUB_GENERIC; u->n = n;
    sub_alloc(u);
    memcpy(u->A, A, sizeof(double) * (size_t)n * n);
    memcpy(u->b, b, sizeof(double) * n);
    return S->nsub - 1;
}

/* bodies: nb records of 17 doubles: m, I[3], p[3], q[4] (w,x,y,z), v[3], w[3] */
int orc_add_rigid(orc_scene *S, int nb, const double *rec)
{
    if (nb <= 0) return -1;
    sub_t *u = new_sub(S);
    u->kind = SUB_RIGID; u->nb = nb; u->n = 6 * nb;
    u->bodies = (body_t *)xcalloc(nb, sizeof(body_t));
    for (int k = 0; k < nb; k++) {
        const double *r = rec + 17 * k;
        body_t *B = &u->bodies[k];
        B->m = r[0];
        memcpy(B->I, r + 1, 3 * sizeof(double));
        memcpy(B->p, r + 4, 3 * sizeof(double));
        memcpy(B->q, r + 7, 4 * sizeof(double));
        memcpy(B->v, r + 11, 3 * sizeof(double));
        memcpy(B->w, r + 14, 3 * sizeof(double));
    }
    sub_alloc(u);
    return S->nsub - 1;
}

/* linear elastic block of nn nodes (3 DOF each): data = mass (nn), K (n x n row-major),
 * f (n), rest positions X0 (n), positions x (n), velocities v (n), n = 3 nn */
static void assemble_corot(orc_scene *S, sub_t *u);

/* Makes linear block i co-rotational: ne elements of 4 node indices (tets) with their rest
   stiffness matrices (Ke, 144 per element); its K and elastic force are assembled from them
   at every step (assemble_corot) instead of from the constant K. */
int orc_set_corot(orc_scene *S, int i, int ne, const int *tets, const double *Ke)
{
    sub_t *u = &S->subs[i];
    if (u->kind != SUB_LINEAR || ne < 1) return -1;
    for (int q = 0; q < 4 * ne; q++)
        if (tets[q] < 0 || tets[q] >= u->nb) return -1;
    u->ne = ne;
    u->tets = (int *)xcalloc((size_t)4 * ne, sizeof(int));
    u->Ke = (double *)xcalloc((size_t)144 * ne, sizeof(double));
    memcpy(u->tets, tets, sizeof(int) * 4 * (size_t)ne);
    memcpy(u->Ke, Ke, sizeof(double) * 144 * (size_t)ne);
    return 0;
}

/* Elastic force of a linear block at its current positions (n doubles) and its stiffness
   (n x n): the assembly's own terms, for tests.  */
void orc_elastic(orc_scene *S, int i, double *f, double *K)
{
    sub_t *u = &S->subs[i];
    int n = u->n;
    if (u->ne > 0) {
        assemble_corot(S, u);
        memcpy(f, u->rhs, sizeof(double) * n);
    } else {
        for (int p = 0; p < n; p++) {
            double kx = 0.0;
            for (int q = 0; q < n; q++) kx += u->Kel[p * n + q] * (u->x[q] - u->X0[q]);
            f[p] = -kx;
        }
    }
    memcpy(K, u->Kel, sizeof(double) * (size_t)n * n);
}

int orc_add_linear(orc_scene *S, int nn, const double *data)
{
    if (nn <= 0) return -1;
    sub_t *u = new_sub(S);
    u->kind = SUB_LINEAR; u->nb = nn; u->n = 3 * nn;
    int n = u->n;
    u->mass = (double *)xcalloc(nn, sizeof(double));
    u->Kel = (double *)xcalloc((size_t)n * n, sizeof(double));
    u->fext = (double *)xcalloc(n, sizeof(double));
    u->X0 = (double *)xcalloc(n, sizeof(double));
    u->x = (double *)xcalloc(n, sizeof(double));
    u->vel = (double *)xcalloc(n, sizeof(double));
    const double *p = data;
    memcpy(u->mass, p, nn * sizeof(double)); p += nn;
    memcpy(u->Kel, p, (size_t)n * n * sizeof(double)); p += (size_t)n * n;
    memcpy(u->fext, p, n * sizeof(double)); p += n;
    memcpy(u->X0, p, n * sizeof(double)); p += n;
    memcpy(u->x, p, n * sizeof(double)); p += n;
    memcpy(u->vel, p, n * sizeof(double));
    sub_alloc(u);
    return S->nsub - 1;
}

static con_t *new_con(orc_scene *S)
{
    if (S->ncon == S->capcon) {
        S->capcon = S->capcon ? 2 * S->capcon : 8;
        S->cons = (con_t *)realloc(S->cons, sizeof(con_t) * S->capcon);
    }
    con_t *c = &S->cons[S->ncon++];
    memset(c, 0, sizeof(*c));
    return c;
}

static void con_alloc(orc_scene *S, con_t *c)
{
    int nr = c->rows * c->ns;
    for (int s = 0; s < c->ns; s++)
        c->J[s] = (double *)xcalloc((size_t)c->rows * S->subs[c->sub[s]].n, sizeof(double));
    c->e = (double *)xcalloc(c->rows, sizeof(double));
    c->x = (double *)xcalloc(nr, sizeof(double));
    c->z = (double *)xcalloc(nr, sizeof(double));
    c->u = (double *)xcalloc(nr, sizeof(double));
    c->y = (double *)xcalloc(nr, sizeof(double));
    c->yold = (double *)xcalloc(nr, sizeof(double));
    c->zold = (double *)xcalloc(nr, sizeof(double));
    c->zprev = (double *)xcalloc(nr, sizeof(double));
    c->lam = (double *)xcalloc(c->rows, sizeof(double));
    c->lamprev = (double *)xcalloc(c->rows, sizeof(double));
}

/* explicit rows: J holds, side after side, rows x n_{subs[s]} row-major blocks */
int orc_add_rows(orc_scene *S, int type, int rows, int ns, const int *subs, const double *J,
                 const double *e, double k, double alpha, double mu)
{
    if (ns < 1 || ns > MAXSIDES || rows < 1) return -1;
    if (type == T_CONTACT && rows != 3) return -1;
    for (int s = 0; s < ns; s++) {
        if (subs[s] < 0 || subs[s] >= S->nsub) return -1;
        for (int t = 0; t < s; t++) if (subs[t] == subs[s]) return -1;
    }
    con_t *c = new_con(S);
    c->src = SRC_ROWS; c->type = type; c->rows = rows; c->ns = ns;
    c->k = k; c->alpha = alpha; c->mu = mu;
    for (int s = 0; s < ns; s++) c->sub[s] = subs[s];
    con_alloc(S, c);
    const double *Jp = J;
    for (int s = 0; s < ns; s++) {
        size_t cnt = (size_t)rows * S->subs[subs[s]].n;
        memcpy(c->J[s], Jp, cnt * sizeof(double));
        Jp += cnt;
    }
    memcpy(c->e, e, rows * sizeof(double));
    return S->ncon - 1;
}

/* rigid-model constraint.  p: anchor_a[3] anchor_b[3] axis_a[3] axis_b[3] ref_a[3]
 * ref_b[3] kp kd target plane_z mu   (23 doubles).  sb < 0 means the world.
 * PLANE: axis_b is the plane's world normal (any length > 0; stored normalised); a sphere
 * of radius ref_a[0] (>= 0; 0 for a point) about anchor_a touches the plane.
 * SPHERE: anchor_a / anchor_b are the sphere centres in a's / b's frame (b: a world point
 * for the world), ref_a[0] and ref_b[0] the radii (>= 0). */
int orc_add_joint(orc_scene *S, int kind, int sa, int ba, int sb, int bb, const double *p)
{
    /* a node of a linear block may be a side of a ball joint or a contact */
    const int node_ok = (kind == SRC_BALL || kind == SRC_PLANE || kind == SRC_SPHERE);
    if (sa < 0 || sa >= S->nsub || S->subs[sa].kind == SUB_GENERIC) return -1;
    if (S->subs[sa].kind == SUB_LINEAR && !node_ok) return -1;
    if (ba < 0 || ba >= S->subs[sa].nb) return -1;
    if (kind == SRC_PLANE) sb = -1;
    if (sb >= 0) {
        if (sb >= S->nsub || S->subs[sb].kind == SUB_GENERIC) return -1;
        if (S->subs[sb].kind == SUB_LINEAR && !node_ok) return -1;
        if (bb < 0 || bb >= S->subs[sb].nb) return -1;
        if (sb == sa && bb == ba) return -1;
    }
    if (kind == SRC_PLANE) sb = -1;
    con_t *c = new_con(S);
    c->src = kind;
    c->sa = sa; c->ba = ba; c->sb = sb; c->bb = bb;
    memcpy(c->anc_a, p + 0, 3 * sizeof(double));
    memcpy(c->anc_b, p + 3, 3 * sizeof(double));
    memcpy(c->ax_a, p + 6, 3 * sizeof(double));
    memcpy(c->ax_b, p + 9, 3 * sizeof(double));
    memcpy(c->ref_a, p + 12, 3 * sizeof(double));
    memcpy(c->ref_b, p + 15, 3 * sizeof(double));
    c->kp = p[18]; c->kd = p[19]; c->target = p[20]; c->plane_z = p[21]; c->mu = p[22];
    switch (kind) {
    case SRC_BALL: c->rows = 3; c->type = T_EQUALITY; break;
    case SRC_REVOLUTE: c->rows = 5; c->type = T_EQUALITY; break;
    case SRC_ANGLE_PD: c->rows = 1; c->type = T_SOFT; break;
    case SRC_PLANE: c->rows = 3; c->type = T_CONTACT; break;
    case SRC_SPHERE: c->rows = 3; c->type = T_CONTACT; break;
    default: S->ncon--; return -1;
    }
    if (kind == SRC_PLANE) {
        double len = sqrt(dot3(c->ax_b, c->ax_b));
        if (!(len > 0.0)) { S->ncon--; return -1; }
        for (int d = 0; d < 3; d++) c->ax_b[d] /= len;
    }
    if (kind == SRC_PLANE && !(c->ref_a[0] >= 0.0)) { S->ncon--; return -1; }
    if (kind == SRC_SPHERE && !(c->ref_a[0] >= 0.0 && c->ref_b[0] >= 0.0)) { S->ncon--; return -1; }
    c->ns = 1;
    c->sub[0] = sa;
    if (sb >= 0 && sb != sa) { c->ns = 2; c->sub[1] = sb; }
    con_alloc(S, c);
    return S->ncon - 1;
}

/* ------------------------------------------------------------------------------------ */
/* rigid-body model: A_i, b_i (Eq. ddyn) and constraint rows (Sec. II-A)                 */

static void assemble_rigid(orc_scene *S, sub_t *u)
{
    int n = u->n;
    double c2h = 2.0 / S->h;
    memset(u->A, 0, sizeof(double) * (size_t)n * n);
    for (int k = 0; k < u->nb; k++) {
        body_t *B = &u->bodies[k];
        int o = 6 * k;
        double mass[6] = {B->m, B->m, B->m, B->I[0], B->I[1], B->I[2]};
        for (int d = 0; d < 6; d++) u->A[(o + d) * n + (o + d)] = c2h * mass[d];
        /* b = (2/h) M v_k - C v_k + f ;  C v_k = [0; w x I w] (body frame) ; f = [m g; 0] */
        double Iw[3] = {B->I[0] * B->w[0], B->I[1] * B->w[1], B->I[2] * B->w[2]};
        double gyro[3];
        cross3(B->w, Iw, gyro);
        for (int d = 0; d < 3; d++) {
            u->b[o + d] = c2h * B->m * B->v[d] + B->m * S->g[d];
            u->b[o + 3 + d] = c2h * Iw[d] - gyro[d];
        }
    }
}

/* Linear elastic block (Eq. ddyn with the elastic force at the midpoint):
 * A = (2/h) M + (h/2) K ;  b = (2/h) M v_k - K (x_k - X0) + f + M g */
/* Rotation part of F (polar decomposition F = R S, S symmetric positive definite) by
   Newton's iteration R <- (R + R^-T) / 2 from R = F (Higham), to convergence. */
static void polar_rotation(const double F[9], double R[9])
{
    memcpy(R, F, 9 * sizeof(double));
    for (int it = 0; it < 60; it++) {
        /* R^-T = cofactor(R) / det(R) */
        double c[9];
        c[0] = R[4] * R[8] - R[5] * R[7];
        c[1] = R[5] * R[6] - R[3] * R[8];
        c[2] = R[3] * R[7] - R[4] * R[6];
        c[3] = R[2] * R[7] - R[1] * R[8];
        c[4] = R[0] * R[8] - R[2] * R[6];
        c[5] = R[1] * R[6] - R[0] * R[7];
        c[6] = R[1] * R[5] - R[2] * R[4];
        c[7] = R[2] * R[3] - R[0] * R[5];
        c[8] = R[0] * R[4] - R[1] * R[3];
        double det = R[0] * c[0] + R[1] * c[1] + R[2] * c[2];
        double d = 0.0, nrm = 0.0;
        for (int k = 0; k < 9; k++) {
            double nk = 0.5 * (R[k] + c[k] / det);
            d += (nk - R[k]) * (nk - R[k]);
            nrm += nk * nk;
            R[k] = nk;
        }
        if (d <= 1e-30 * nrm) break;
    }
}

/* Co-rotational linear elasticity (the paper's beam model, Sec. IV-A): per element the
   rotation R of its deformation gradient F = D_s D_m^-1 (edge matrices of the current and
   rest positions), the rotated stiffness R K_e R^T (R on each node's 3 x 3 block) and the
   elastic force -R K_e (R^T x_e - X_e); the stiffness is that of the step's start, like the
   linear block's (A = (2/h) M + (h/2) K, b = (2/h) M v_k + f_el + f + M g). */
static void assemble_corot(orc_scene *S, sub_t *u)
{
    int n = u->n;
    double c2h = 2.0 / S->h;
    memset(u->Kel, 0, sizeof(double) * (size_t)n * n);
    double *fel = u->rhs;                     /* scratch: elastic force (n) */
    memset(fel, 0, sizeof(double) * n);
    for (int e = 0; e < u->ne; e++) {
        const int *t = u->tets + 4 * e;
        const double *K = u->Ke + 144 * e;
        double Dm[9], Ds[9];                  /* columns: node k - node 0, k = 1..3 */
        for (int k = 0; k < 3; k++)
            for (int d = 0; d < 3; d++) {
                Dm[3 * d + k] = u->X0[3 * t[k + 1] + d] - u->X0[3 * t[0] + d];
                Ds[3 * d + k] = u->x[3 * t[k + 1] + d] - u->x[3 * t[0] + d];
            }
        /* F = Ds Dm^-1 */
        double c[9], Mi[9], F[9], R[9];
        c[0] = Dm[4] * Dm[8] - Dm[5] * Dm[7];
        c[1] = Dm[5] * Dm[6] - Dm[3] * Dm[8];
        c[2] = Dm[3] * Dm[7] - Dm[4] * Dm[6];
        c[3] = Dm[2] * Dm[7] - Dm[1] * Dm[8];
        c[4] = Dm[0] * Dm[8] - Dm[2] * Dm[6];
        c[5] = Dm[1] * Dm[6] - Dm[0] * Dm[7];
        c[6] = Dm[1] * Dm[5] - Dm[2] * Dm[4];
        c[7] = Dm[2] * Dm[3] - Dm[0] * Dm[5];
        c[8] = Dm[0] * Dm[4] - Dm[1] * Dm[3];
        double det = Dm[0] * c[0] + Dm[1] * c[1] + Dm[2] * c[2];
        for (int a = 0; a < 3; a++)                 /* inverse = cofactor^T / det */
            for (int b = 0; b < 3; b++) Mi[3 * a + b] = c[3 * b + a] / det;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += Ds[3 * a + k] * Mi[3 * k + b];
                F[3 * a + b] = acc;
            }
        polar_rotation(F, R);
        /* w = R^T x_e - X_e ; g = K w ; force -R g */
        double w[12], g[12];
        for (int a = 0; a < 4; a++)
            for (int d = 0; d < 3; d++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += R[3 * k + d] * u->x[3 * t[a] + k];
                w[3 * a + d] = acc - u->X0[3 * t[a] + d];
            }
        for (int i = 0; i < 12; i++) {
            double acc = 0.0;
            for (int j = 0; j < 12; j++) acc += K[12 * i + j] * w[j];
            g[i] = acc;
        }
        for (int a = 0; a < 4; a++)
            for (int d = 0; d < 3; d++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += R[3 * d + k] * g[3 * a + k];
                fel[3 * t[a] + d] -= acc;
            }
        /* Kel block (a, b) += R K_ab R^T */
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                double T[9];
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        double acc = 0.0;
                        for (int k = 0; k < 3; k++) acc += R[3 * i + k] * K[12 * (3 * a + k) + 3 * b + j];
                        T[3 * i + j] = acc;
                    }
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        double acc = 0.0;
                        for (int k = 0; k < 3; k++) acc += T[3 * i + k] * R[3 * j + k];
                        u->Kel[(size_t)(3 * t[a] + i) * n + 3 * t[b] + j] += acc;
                    }
            }
    }
    for (int p = 0; p < n; p++) {
        for (int q = 0; q < n; q++) u->A[p * n + q] = 0.5 * S->h * u->Kel[p * n + q];
        u->A[p * n + p] += c2h * u->mass[p / 3];
        u->b[p] = c2h * u->mass[p / 3] * u->vel[p] + fel[p] + u->fext[p] + u->mass[p / 3] * S->g[p % 3];
    }
}

static void assemble_linear(orc_scene *S, sub_t *u)
{
    if (u->ne > 0) { assemble_corot(S, u); return; }
    int n = u->n;
    double c2h = 2.0 / S->h;
    for (int p = 0; p < n; p++) {
        for (int q = 0; q < n; q++) u->A[p * n + q] = 0.5 * S->h * u->Kel[p * n + q];
        u->A[p * n + p] += c2h * u->mass[p / 3];
        double kx = 0.0;
        for (int q = 0; q < n; q++) kx += u->Kel[p * n + q] * (u->x[q] - u->X0[q]);
        u->b[p] = c2h * u->mass[p / 3] * u->vel[p] - kx + u->fext[p] + u->mass[p / 3] * S->g[p % 3];
    }
}

/* Row of the velocity of body point P = p + R r along the world direction dir.
 * dP/dt = v + R (w x r) with w in the body frame, so
 * dir . dP/dt = dir . v + (R^T dir) . (w x r) = dir . v + w . (r x R^T dir). */
static void point_row(const double dir[3], const double R[9], const double r[3], double row[6])
{
    double Rd[3];
    rowtimesR(dir, R, Rd);          /* R^T dir */
    row[0] = dir[0]; row[1] = dir[1]; row[2] = dir[2];
    cross3(r, Rd, row + 3);
}

/* A side of a model constraint: a rigid body (6 columns from 6 idx: [v, w]) or a node of a
 * linear block (3 columns from 3 idx: its velocity). */
typedef struct { int node; const double *p; double R[9]; } side_t;

static void side_of(orc_scene *S, int sub, int idx, side_t *sd)
{
    if (S->subs[sub].kind == SUB_LINEAR) {
        sd->node = 1;
        sd->p = S->subs[sub].x + 3 * idx;
        memset(sd->R, 0, sizeof sd->R);
        sd->R[0] = sd->R[4] = sd->R[8] = 1.0;
    } else {
        body_t *B = &S->subs[sub].bodies[idx];
        sd->node = 0;
        sd->p = B->p;
        quat_to_mat(B->q, sd->R);
    }
}

/* world point of a side (a node ignores the anchor) and its velocity row along dir */
static void side_point(const side_t *sd, const double anc[3], double P[3])
{
    if (sd->node) { P[0] = sd->p[0]; P[1] = sd->p[1]; P[2] = sd->p[2]; return; }
    double ra[3];
    matvec3(sd->R, anc, ra);
    for (int d = 0; d < 3; d++) P[d] = sd->p[d] + ra[d];
}

static void side_row(const side_t *sd, const double dir[3], const double anc[3], double *row)
{
    if (sd->node) { row[0] = dir[0]; row[1] = dir[1]; row[2] = dir[2]; return; }
    point_row(dir, sd->R, anc, row);
}

/* Contact frame of a unit normal n: rows (n, t1, t2) with t1 the world x axis (the y axis
 * when n is within ~25 degrees of x) made orthogonal to n and normalised, t2 = n x t1.  For
 * n = +z this is (z, x, y). */
static void contact_frame(const double n[3], double F[3][3])
{
    double e[3] = {1.0, 0.0, 0.0};
    if (fabs(n[0]) > 0.9) { e[0] = 0.0; e[1] = 1.0; }
    double en = dot3(e, n), t1[3];
    for (int d = 0; d < 3; d++) t1[d] = e[d] - en * n[d];
    double len = sqrt(dot3(t1, t1));
    for (int d = 0; d < 3; d++) { t1[d] /= len; F[0][d] = n[d]; F[1][d] = t1[d]; }
    cross3(n, t1, F[2]);
}

/* phi (rows) and the blocks Ja, Jb (rows x 6, of which the first 3 columns are used for a
 * node side) of a model constraint */
static void joint_rows(orc_scene *S, con_t *c, double *phi, double *Ja, double *Jb)
{
    side_t sa, sbd;
    side_of(S, c->sa, c->ba, &sa);
    const int hasb = c->sb >= 0;
    if (hasb) side_of(S, c->sb, c->bb, &sbd);
    const double *Ra = sa.R, *Rb = hasb ? sbd.R : NULL;
    body_t *B = (hasb && !sbd.node) ? &S->subs[c->sb].bodies[c->bb] : NULL;
    memset(Ja, 0, sizeof(double) * 6 * c->rows);
    memset(Jb, 0, sizeof(double) * 6 * c->rows);
    static const double E[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (c->src == SRC_BALL || c->src == SRC_REVOLUTE) {
        double pa[3], pb[3];
        side_point(&sa, c->anc_a, pa);
        if (hasb) side_point(&sbd, c->anc_b, pb);
        else { for (int d = 0; d < 3; d++) pb[d] = c->anc_b[d]; }
        for (int d = 0; d < 3; d++) {
            phi[d] = pa[d] - pb[d];
            side_row(&sa, E[d], c->anc_a, Ja + 6 * d);
            if (hasb) {
                side_row(&sbd, E[d], c->anc_b, Jb + 6 * d);
                for (int q = 0; q < 6; q++) Jb[6 * d + q] = -Jb[6 * d + q];
            }
        }
        if (c->src == SRC_REVOLUTE) {
            double ub[3], t[2][3], tmp[3];
            if (B) matvec3(Rb, c->ax_b, ub); else memcpy(ub, c->ax_b, sizeof ub);
            matvec3(Ra, c->ref_a, t[0]);
            cross3(c->ax_a, c->ref_a, tmp);
            matvec3(Ra, tmp, t[1]);
            for (int k = 0; k < 2; k++) {
                int r = 3 + k;
                double txu[3], ja[3], jb[3];
                phi[r] = dot3(t[k], ub);
                cross3(t[k], ub, txu);       /* d/dt (t . u_b) = (t x u_b) . (w_a - w_b) */
                rowtimesR(txu, Ra, ja);
                for (int q = 0; q < 3; q++) Ja[6 * r + 3 + q] = ja[q];
                if (B) {
                    rowtimesR(txu, Rb, jb);
                    for (int q = 0; q < 3; q++) Jb[6 * r + 3 + q] = -jb[q];
                }
            }
        }
    } else if (c->src == SRC_ANGLE_PD) {
        double u[3], na[3], nb[3], cr[3], ja[3], jb[3];
        matvec3(Ra, c->ax_a, u);
        matvec3(Ra, c->ref_a, na);
        if (B) matvec3(Rb, c->ref_b, nb); else memcpy(nb, c->ref_b, sizeof nb);
        cross3(na, nb, cr);
        phi[0] = atan2(dot3(cr, u), dot3(na, nb));
        /* d theta / dt = u . (w_b - w_a) */
        rowtimesR(u, Ra, ja);
        for (int q = 0; q < 3; q++) Ja[3 + q] = -ja[q];
        if (B) {
            rowtimesR(u, Rb, jb);
            for (int q = 0; q < 3; q++) Jb[3 + q] = jb[q];
        }
    } else if (c->src == SRC_PLANE) {
        /* the plane {x : n . x = plane_z}; the gap along n of the sphere of radius r about
         * point a; rows of the velocity of its surface point a - r n */
        double pa[3], F[3][3], ca[3], tmp[3];
        const double *n = c->ax_b, r = c->ref_a[0];
        side_point(&sa, c->anc_a, pa);
        phi[0] = dot3(n, pa) - c->plane_z - r;
        phi[1] = 0.0; phi[2] = 0.0;
        contact_frame(n, F);
        rowtimesR(n, Ra, tmp);
        for (int d = 0; d < 3; d++) ca[d] = c->anc_a[d] - r * tmp[d];
        for (int d = 0; d < 3; d++) side_row(&sa, F[d], ca, Ja + 6 * d);
    } else if (c->src == SRC_SPHERE) {
        /* spheres of radii r_a, r_b about the centres P_a, P_b: normal n = (P_a - P_b)/|.|
         * (+z for coincident centres), gap |P_a - P_b| - r_a - r_b; rows of the relative
         * velocity of the two surface points P_a - r_a n and P_b + r_b n */
        double Pa[3], Pb[3], dv[3], n[3] = {0.0, 0.0, 1.0}, F[3][3];
        side_point(&sa, c->anc_a, Pa);
        if (hasb) side_point(&sbd, c->anc_b, Pb);
        else { for (int d = 0; d < 3; d++) Pb[d] = c->anc_b[d]; }
        for (int d = 0; d < 3; d++) dv[d] = Pa[d] - Pb[d];
        double dist = sqrt(dot3(dv, dv));
        if (dist > 0.0) for (int d = 0; d < 3; d++) n[d] = dv[d] / dist;
        const double ra = c->ref_a[0], rb = c->ref_b[0];
        phi[0] = dist - ra - rb;
        phi[1] = 0.0; phi[2] = 0.0;
        contact_frame(n, F);
        /* surface points as offsets in each body's frame: anchor + R^T (-/+ r n) */
        double ca[3], cb[3] = {c->anc_b[0], c->anc_b[1], c->anc_b[2]}, tmp[3];
        rowtimesR(n, Ra, tmp);
        for (int d = 0; d < 3; d++) ca[d] = c->anc_a[d] - ra * tmp[d];
        if (hasb && !sbd.node) {
            rowtimesR(n, Rb, tmp);
            for (int d = 0; d < 3; d++) cb[d] = c->anc_b[d] + rb * tmp[d];
        }
        for (int d = 0; d < 3; d++) {
            side_row(&sa, F[d], ca, Ja + 6 * d);
            if (hasb) {
                side_row(&sbd, F[d], cb, Jb + 6 * d);
                for (int q = 0; q < 6; q++) Jb[6 * d + q] = -Jb[6 * d + q];
            }
        }
    }
}

static void assemble_joint(orc_scene *S, con_t *c)
{
    double phi[5], Ja[30], Jb[30];
    joint_rows(S, c, phi, Ja, Jb);
    int na = S->subs[c->sa].n;
    /* a body side fills 6 columns at 6 * index, a node side 3 columns at 3 * index */
    int wa = S->subs[c->sa].kind == SUB_LINEAR ? 3 : 6;
    for (int s = 0; s < c->ns; s++) memset(c->J[s], 0, sizeof(double) * c->rows * S->subs[c->sub[s]].n);
    for (int r = 0; r < c->rows; r++)
        for (int q = 0; q < wa; q++) c->J[0][r * na + wa * c->ba + q] += Ja[r * 6 + q];
    if (c->sb >= 0) {
        int side = (c->sb == c->sa) ? 0 : 1;
        int nb = S->subs[c->sb].n;
        int wb = S->subs[c->sb].kind == SUB_LINEAR ? 3 : 6;
        for (int r = 0; r < c->rows; r++)
            for (int q = 0; q < wb; q++) c->J[side][r * nb + wb * c->bb + q] += Jb[r * 6 + q];
    }
    double h = S->h;
    if (c->src == SRC_BALL || c->src == SRC_REVOLUTE) {
        for (int r = 0; r < c->rows; r++) c->e[r] = S->gamma * phi[r] / h;
    } else if (c->src == SRC_ANGLE_PD) {
        c->e[0] = phi[0] - c->target;
        c->k = c->kp;
        c->alpha = c->kd / c->kp + 0.5 * h;
    } else if (c->src == SRC_PLANE || c->src == SRC_SPHERE) {
        double gap = phi[0];
        c->e[0] = gap >= 0.0 ? gap / h : S->gamma * gap / h;
        c->e[1] = 0.0; c->e[2] = 0.0;
    }
}

/* ------------------------------------------------------------------------------------ */
/* z-step of one constraint (Sec. III-C, Eq. admm-2j via Eq. surrogate)                   */

/* y: ns x rows, beta: ns.  Writes lambda (rows).  Returns nothing. */
void orc_project(int type, int rows, int ns, const double *beta, const double *y,
                 const double *e, double k, double alpha, double mu, double *lam)
{
    double s = 0.0;
    for (int i = 0; i < ns; i++) s += 1.0 / beta[i];
    double q[8];
    for (int r = 0; r < rows; r++) {
        q[r] = 0.0;
        for (int i = 0; i < ns; i++) q[r] += y[i * rows + r] / beta[i];
    }
    if (type == T_EQUALITY) {
        for (int r = 0; r < rows; r++) lam[r] = -(q[r] + e[r]) / s;
    } else if (type == T_HARD) {
        for (int r = 0; r < rows; r++) {
            double l = -(q[r] + e[r]) / s;
            lam[r] = l > 0.0 ? l : 0.0;
        }
    } else if (type == T_SOFT) {
        for (int r = 0; r < rows; r++)
            lam[r] = -k * (e[r] + alpha * q[r]) / (1.0 + s * alpha * k);
    } else { /* contact: rows (n, t1, t2) */
        double ln = -(q[0] + e[0]) / s;
        double l1 = -(q[1] + e[1]) / s;
        double l2 = -(q[2] + e[2]) / s;
        if (ln <= 0.0) { lam[0] = 0.0; lam[1] = 0.0; lam[2] = 0.0; return; }
        double t = sqrt(l1 * l1 + l2 * l2);
        double lim = mu * ln;
        lam[0] = ln;
        if (t > lim) { lam[1] = l1 * (lim / t); lam[2] = l2 * (lim / t); }
        else { lam[1] = l1; lam[2] = l2; }
    }
}

/* ------------------------------------------------------------------------------------ */
/* one time step (Algorithm 1)                                                            */

static double beta_of(orc_scene *S, int i)
{
    return S->subs[i].beta;
}

/* v_i = A_i^-1 (b_i + sum_j J_ij^T lambda_j) for every subsystem (A_i's factor in L) */
static void pj_velocities(orc_scene *S)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < S->nsub; i++) {
        sub_t *u = &S->subs[i];
        memcpy(u->v, u->b, sizeof(double) * u->n);
        for (int j = 0; j < S->ncon; j++) {
            con_t *c = &S->cons[j];
            for (int s = 0; s < c->ns; s++) {
                if (c->sub[s] != i) continue;
                for (int r = 0; r < c->rows; r++)
                    for (int p = 0; p < u->n; p++) u->v[p] += c->J[s][r * u->n + p] * c->lam[r];
            }
        }
        chol_solve(u->n, u->L, u->v);
    }
}

/* The subsystem-based ADMM loop of one step (Algorithm 1) on the assembled A_i, b_i, J, e:
 * leaves v-hat in each subsystem and lambda, z in each constraint. */
static int admm_solve(orc_scene *S)
{
    /* beta_i (Sec. III-D): the trace rule, or a fixed rho; times the subsystem's scale (an
       input: 1 unless a learned rho sets it) */
    for (int i = 0; i < S->nsub; i++) {
        sub_t *u = &S->subs[i];
        if (S->beta_fixed) { u->beta = S->rho * u->beta_scale; continue; }
        double trA = 0.0, trJ = 0.0;
        for (int d = 0; d < u->n; d++) trA += u->A[d * u->n + d];
        for (int j = 0; j < S->ncon; j++) {
            con_t *c = &S->cons[j];
            for (int s = 0; s < c->ns; s++) {
                if (c->sub[s] != i) continue;
                for (int q = 0; q < c->rows * u->n; q++) trJ += c->J[s][q] * c->J[s][q];
            }
        }
        u->beta = (trJ > 0.0 ? trA / trJ : 1.0) * u->beta_scale;
    }
    /* factorise K_i = A_i + beta_i J_ci^T J_ci (subsystems are independent: the OpenMP
       build of the timing baseline runs them on separate threads) */
    int notspd = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : notspd)
    for (int i = 0; i < S->nsub; i++) {
        sub_t *u = &S->subs[i];
        int n = u->n;
        double *K = (double *)xcalloc((size_t)n * n, sizeof(double));
        memcpy(K, u->A, sizeof(double) * (size_t)n * n);
        for (int j = 0; j < S->ncon; j++) {
            con_t *c = &S->cons[j];
            for (int s = 0; s < c->ns; s++) {
                if (c->sub[s] != i) continue;
                const double *J = c->J[s];
                for (int r = 0; r < c->rows; r++)
                    for (int p = 0; p < n; p++)
                        for (int q = 0; q < n; q++)
                            K[p * n + q] += u->beta * J[r * n + p] * J[r * n + q];
            }
        }
        int rc = cholesky(n, K, u->L);
        free(K);
        if (rc) notspd = 1;
    }
    if (notspd) { S->status = -3; return -3; }
    /* initial z, u (cold: zeros; warm: previous step's z and -lambda) */
    for (int j = 0; j < S->ncon; j++) {
        con_t *c = &S->cons[j];
        for (int s = 0; s < c->ns; s++) {
            double be = beta_of(S, c->sub[s]);
            for (int r = 0; r < c->rows; r++) {
                int q = s * c->rows + r;
                if (S->warm_prev && c->has_prev) {
                    c->z[q] = c->zprev[q];
                    c->u[q] = -c->lamprev[r];
                } else {
                    c->z[q] = 0.0;
                    c->u[q] = 0.0;
                }
                c->yold[q] = be * c->z[q] + c->u[q];
            }
        }
    }
    S->iters = 0; S->converged = 0;
    S->r_p = INFINITY; S->r_d = INFINITY; S->theta = INFINITY;
    int L = S->max_iters;
    for (int l = 0; l < L; l++) {
        /* v-step: rhs_i = b_i + J_ci^T (beta_i z_i - u_i); K_i v_i = rhs_i.  Each subsystem
           gathers its constraints' terms in constraint order (independent per subsystem) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < S->nsub; i++) {
            sub_t *u = &S->subs[i];
            memcpy(u->rhs, u->b, sizeof(double) * u->n);
            for (int j = 0; j < S->ncon; j++) {
                con_t *c = &S->cons[j];
                for (int s = 0; s < c->ns; s++) {
                    if (c->sub[s] != i) continue;
                    for (int r = 0; r < c->rows; r++) {
                        int q = s * c->rows + r;
                        double w = u->beta * c->z[q] - c->u[q];
                        for (int p = 0; p < u->n; p++) u->rhs[p] += c->J[s][r * u->n + p] * w;
                    }
                }
            }
            memcpy(u->v, u->rhs, sizeof(double) * u->n);
            chol_solve(u->n, u->L, u->v);
        }
        /* x_i = J_ci v_i ; y_i = beta_i x_i + u_i ; theta */
        double theta = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : theta)
        for (int j = 0; j < S->ncon; j++) {
            con_t *c = &S->cons[j];
            for (int s = 0; s < c->ns; s++) {
                sub_t *u = &S->subs[c->sub[s]];
                for (int r = 0; r < c->rows; r++) {
                    int q = s * c->rows + r;
                    double acc = 0.0;
                    for (int p = 0; p < u->n; p++) acc += c->J[s][r * u->n + p] * u->v[p];
                    c->x[q] = acc;
                    c->y[q] = u->beta * acc + c->u[q];
                    double d = c->y[q] - c->yold[q];
                    theta += d * d;
                    c->yold[q] = c->y[q];
                }
            }
        }
        S->theta = theta;
        S->iters = l + 1;
        if (S->stop_theta && l >= 1 && theta < S->theta_th) {
            S->converged = 1;
            if (S->trace && l < S->trace_cap) {
                S->trace[3 * l] = theta; S->trace[3 * l + 1] = NAN; S->trace[3 * l + 2] = NAN;
            }
            break;
        }
        /* z-step per constraint, then u-step, then residuals (independent per constraint) */
        double rp = 0.0, rd = 0.0, rz = 0.0;
#pragma omp parallel for schedule(static) reduction(max : rp, rd, rz)
        for (int j = 0; j < S->ncon; j++) {
            con_t *c = &S->cons[j];
            double beta[MAXSIDES];
            for (int s = 0; s < c->ns; s++) beta[s] = beta_of(S, c->sub[s]);
            orc_project(c->type, c->rows, c->ns, beta, c->y, c->e, c->k, c->alpha, c->mu, c->lam);
            for (int s = 0; s < c->ns; s++) {
                for (int r = 0; r < c->rows; r++) {
                    int q = s * c->rows + r;
                    c->zold[q] = c->z[q];
                    c->z[q] = (c->y[q] + c->lam[r]) / beta[s];
                    c->u[q] = c->u[q] + beta[s] * (c->x[q] - c->z[q]);
                    double a = fabs(c->x[q] - c->z[q]);
                    if (a > rp) rp = a;
                    double dz = fabs(c->z[q] - c->zold[q]);
                    if (dz > rz) rz = dz;
                    double b = beta[s] * dz;
                    if (b > rd) rd = b;
                }
            }
        }
        S->r_p = rp; S->r_d = rd;
        if (S->trace && l < S->trace_cap) {
            S->trace[3 * l] = theta; S->trace[3 * l + 1] = rp; S->trace[3 * l + 2] = rd;
        }
        if (!S->stop_theta && S->tol > 0.0 && rp <= S->tol && rz <= S->tol) {
            S->converged = 1;
            break;
        }
        if (!isfinite(rp) || !isfinite(theta)) { S->status = -4; break; }
    }
    return S->status;
}

/* Projected Jacobi on the same step (the comparison solver of Sec. IV-B, written from the
 * standard method, as its details are not printed): the dual problem over the impulses
 * lambda with the subsystems' own A_i (no penalty term), v_i = A_i^-1 (b_i + J_i^T lambda).
 *   delta_r = sum_i J_ir A_i^-1 J_ir^T   (the diagonal of the Delassus operator, per row)
 *   loop l = 0 .. l_max - 1 (a fixed count: the step has no stop rule)
 *     v_i = A_i^-1 (b_i + sum_j J_ij^T lambda_j);  x_r = sum_i J_ir v_i;  c_r = x_r + e_r
 *     every row at once from these values, with relaxation omega:
 *       equality  lambda_r -= omega c_r / delta_r
 *       hard      lambda_r = max(0, lambda_r - omega c_r / delta_r)
 *       soft      lambda*_r = -k (e_r + alpha (x_r - delta_r lambda_r)) / (1 + k alpha delta_r)
 *                 (the soft law with x_r linearised in its own lambda), then
 *                 lambda_r += omega (lambda*_r - lambda_r)
 *       contact   lambda_n = max(0, lambda_n - omega c_n / delta_n); both tangent rows
 *                 lambda_t -= omega c_t / delta_t with one delta_t = max(delta_t1, delta_t2)
 *                 (an isotropic step, so that a sliding contact's exact impulse, on the
 *                 cone's edge against the slip, is a fixed point), then (lambda_t1,
 *                 lambda_t2) scaled onto the disk of radius mu lambda_n when outside it
 *     r_p = max_r |lambda_r^{l+1} - lambda_r^l| delta_r / omega (the natural residual, in
 *     constraint-velocity units)
 *   v-hat = A^-1 (b + J^T lambda) with the last lambda.
 * Starts from the previous step's lambda (warm) or zero. */
static int pj_solve(orc_scene *S)
{
    int notspd = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : notspd)
    for (int i = 0; i < S->nsub; i++) {
        sub_t *u = &S->subs[i];
        u->beta = 0.0;
        if (cholesky(u->n, u->A, u->L)) notspd = 1;
    }
    if (notspd) { S->status = -3; return -3; }
    /* delta per row: J_r A^-1 J_r^T summed over the sides */
    double **delta = (double **)xcalloc(S->ncon, sizeof(double *));
    for (int j = 0; j < S->ncon; j++) {
        con_t *c = &S->cons[j];
        delta[j] = (double *)xcalloc(c->rows, sizeof(double));
        for (int s = 0; s < c->ns; s++) {
            sub_t *u = &S->subs[c->sub[s]];
            double *y = (double *)xcalloc(u->n, sizeof(double));
            for (int r = 0; r < c->rows; r++) {
                memcpy(y, c->J[s] + (size_t)r * u->n, sizeof(double) * u->n);
                chol_solve(u->n, u->L, y);
                double acc = 0.0;
                for (int p = 0; p < u->n; p++) acc += c->J[s][r * u->n + p] * y[p];
                delta[j][r] += acc;
            }
            free(y);
        }
    }
    for (int j = 0; j < S->ncon; j++) {
        con_t *c = &S->cons[j];
        for (int r = 0; r < c->rows; r++)
            c->lam[r] = (S->warm_prev && c->has_prev) ? c->lamprev[r] : 0.0;
    }
    const double om = S->pj_omega;
    S->iters = 0; S->converged = 0;
    S->r_p = INFINITY; S->r_d = 0.0; S->theta = 0.0;
    for (int l = 0; l < S->max_iters; l++) {
        pj_velocities(S);
        double rp = 0.0;
        for (int j = 0; j < S->ncon; j++) {
            con_t *c = &S->cons[j];
            double *x = (double *)xcalloc(c->rows, sizeof(double));
            double *lo = (double *)xcalloc(c->rows, sizeof(double));
            for (int r = 0; r < c->rows; r++) {
                x[r] = 0.0;
                for (int s = 0; s < c->ns; s++) {
                    sub_t *u = &S->subs[c->sub[s]];
                    for (int p = 0; p < u->n; p++) x[r] += c->J[s][r * u->n + p] * u->v[p];
                }
                lo[r] = c->lam[r];
            }
            double *dl = delta[j];
            if (c->type == T_EQUALITY) {
                for (int r = 0; r < c->rows; r++) c->lam[r] = lo[r] - om * (x[r] + c->e[r]) / dl[r];
            } else if (c->type == T_HARD) {
                for (int r = 0; r < c->rows; r++) {
                    double t = lo[r] - om * (x[r] + c->e[r]) / dl[r];
                    c->lam[r] = t > 0.0 ? t : 0.0;
                }
            } else if (c->type == T_SOFT) {
                for (int r = 0; r < c->rows; r++) {
                    double ka = c->k * c->alpha;
                    double ls = -c->k * (c->e[r] + c->alpha * (x[r] - dl[r] * lo[r])) / (1.0 + ka * dl[r]);
                    c->lam[r] = lo[r] + om * (ls - lo[r]);
                }
            } else {
                double ln = lo[0] - om * (x[0] + c->e[0]) / dl[0];
                ln = ln > 0.0 ? ln : 0.0;
                const double dt = dl[1] > dl[2] ? dl[1] : dl[2];
                dl[1] = dt;
                dl[2] = dt;
                double l1 = lo[1] - om * (x[1] + c->e[1]) / dt;
                double l2 = lo[2] - om * (x[2] + c->e[2]) / dt;
                double lim = c->mu * ln, t2 = l1 * l1 + l2 * l2;
                if (t2 > lim * lim) {
                    double f = lim / sqrt(t2);
                    l1 *= f; l2 *= f;
                }
                c->lam[0] = ln; c->lam[1] = l1; c->lam[2] = l2;
            }
            for (int r = 0; r < c->rows; r++) {
                double a = fabs(c->lam[r] - lo[r]) * dl[r] / om;
                if (a > rp) rp = a;
            }
            free(x);
            free(lo);
        }
        S->r_p = rp;
        S->iters = l + 1;
        if (S->trace && l < S->trace_cap) {
            S->trace[3 * l] = 0.0; S->trace[3 * l + 1] = rp; S->trace[3 * l + 2] = 0.0;
        }
        if (!isfinite(rp)) { S->status = -4; break; }
    }
    pj_velocities(S);
    for (int j = 0; j < S->ncon; j++) free(delta[j]);
    free(delta);
    return S->status;
}

int orc_step(orc_scene *S)
{
    S->status = 0;
    /* construct A_i, b_i */
    for (int i = 0; i < S->nsub; i++) {
        if (S->subs[i].kind == SUB_RIGID) assemble_rigid(S, &S->subs[i]);
        else if (S->subs[i].kind == SUB_LINEAR) assemble_linear(S, &S->subs[i]);
    }
    /* construct e_j, J_j */
    for (int j = 0; j < S->ncon; j++)
        if (S->cons[j].src != SRC_ROWS) assemble_joint(S, &S->cons[j]);
    int rc = S->pj ? pj_solve(S) : admm_solve(S);
    if (rc == -3) return rc;
    /* keep lambda and z for the next step's warm start */
    for (int j = 0; j < S->ncon; j++) {
        con_t *c = &S->cons[j];
        memcpy(c->lamprev, c->lam, sizeof(double) * c->rows);
        memcpy(c->zprev, c->z, sizeof(double) * c->rows * c->ns);
        c->has_prev = 1;
    }
    /* state update from v-hat (Eq. ddyn): v_{k+1} = 2 v-hat - v_k ; p += h v-hat ;
       R <- R Exp(h w-hat) with the body-frame angular velocity */
    for (int i = 0; i < S->nsub; i++) {
        sub_t *u = &S->subs[i];
        if (u->kind == SUB_LINEAR) {
            for (int p = 0; p < u->n; p++) {
                u->x[p] += S->h * u->v[p];
                u->vel[p] = 2.0 * u->v[p] - u->vel[p];
            }
            continue;
        }
        if (u->kind != SUB_RIGID) continue;
        for (int k = 0; k < u->nb; k++) {
            body_t *B = &u->bodies[k];
            const double *vh = u->v + 6 * k;
            for (int d = 0; d < 3; d++) {
                B->p[d] += S->h * vh[d];
                B->v[d] = 2.0 * vh[d] - B->v[d];
                B->w[d] = 2.0 * vh[3 + d] - B->w[d];
            }
            double a[3] = {S->h * vh[3], S->h * vh[4], S->h * vh[5]};
            double th = sqrt(dot3(a, a));
            double dq[4];
            if (th > 0.0) {
                double sn = sin(0.5 * th) / th;
                dq[0] = cos(0.5 * th); dq[1] = a[0] * sn; dq[2] = a[1] * sn; dq[3] = a[2] * sn;
            } else { dq[0] = 1.0; dq[1] = dq[2] = dq[3] = 0.0; }
            double *q = B->q, nq[4];
            nq[0] = q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] - q[3] * dq[3];
            nq[1] = q[0] * dq[1] + q[1] * dq[0] + q[2] * dq[3] - q[3] * dq[2];
            nq[2] = q[0] * dq[2] - q[1] * dq[3] + q[2] * dq[0] + q[3] * dq[1];
            nq[3] = q[0] * dq[3] + q[1] * dq[2] - q[2] * dq[1] + q[3] * dq[0];
            double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
            for (int d = 0; d < 4; d++) q[d] = nq[d] / nn;
        }
    }
    return S->status;
}

/* ------------------------------------------------------------------------------------ */
/* accessors                                                                             */

void orc_set_trace(orc_scene *S, double *buf, int cap) { S->trace = buf; S->trace_cap = cap; }
/* Projected Jacobi instead of ADMM for every later step (on != 0), relaxation omega > 0 */
int orc_set_pj(orc_scene *S, int on, double omega)
{
    if (on && !(omega > 0.0)) return -1;
    S->pj = on ? 1 : 0;
    S->pj_omega = omega;
    return 0;
}
int orc_nsub(orc_scene *S) { return S->nsub; }
int orc_ncon(orc_scene *S) { return S->ncon; }
int orc_n(orc_scene *S, int i) { return S->subs[i].n; }
int orc_rows(orc_scene *S, int j) { return S->cons[j].rows; }
int orc_nsides(orc_scene *S, int j) { return S->cons[j].ns; }
double orc_beta(orc_scene *S, int i) { return S->subs[i].beta; }

/* Scales subsystem i's beta (from the next step on): beta_i = scale * trace rule (or rho). */
void orc_set_beta_scale(orc_scene *S, int i, double scale) { S->subs[i].beta_scale = scale; }

void orc_get_vhat(orc_scene *S, int i, double *out) { memcpy(out, S->subs[i].v, sizeof(double) * S->subs[i].n); }

void orc_get_Ab(orc_scene *S, int i, double *A, double *b)
{
    sub_t *u = &S->subs[i];
    if (A) memcpy(A, u->A, sizeof(double) * (size_t)u->n * u->n);
    if (b) memcpy(b, u->b, sizeof(double) * u->n);
}

void orc_get_L(orc_scene *S, int i, double *L) { memcpy(L, S->subs[i].L, sizeof(double) * (size_t)S->subs[i].n * S->subs[i].n); }

void orc_get_lambda(orc_scene *S, int j, double *out) { memcpy(out, S->cons[j].lam, sizeof(double) * S->cons[j].rows); }

/* which: 0 x, 1 z, 2 u, 3 y */
void orc_get_side(orc_scene *S, int j, int which, double *out)
{
    con_t *c = &S->cons[j];
    double *src = which == 0 ? c->x : which == 1 ? c->z : which == 2 ? c->u : c->y;
    memcpy(out, src, sizeof(double) * c->rows * c->ns);
}

/* the rows of constraint j as assembled for the last step: e (rows) and J per side */
void orc_get_rows(orc_scene *S, int j, double *e, double *J)
{
    con_t *c = &S->cons[j];
    if (e) memcpy(e, c->e, sizeof(double) * c->rows);
    if (J) {
        double *p = J;
        for (int s = 0; s < c->ns; s++) {
            size_t cnt = (size_t)c->rows * S->subs[c->sub[s]].n;
            memcpy(p, c->J[s], cnt * sizeof(double));
            p += cnt;
        }
    }
}

int orc_con_sub(orc_scene *S, int j, int s) { return S->cons[j].sub[s]; }

/* assemble (without solving) so tests can read A, b, J, e at the current state */
void orc_assemble(orc_scene *S)
{
    for (int i = 0; i < S->nsub; i++) {
        if (S->subs[i].kind == SUB_RIGID) assemble_rigid(S, &S->subs[i]);
        else if (S->subs[i].kind == SUB_LINEAR) assemble_linear(S, &S->subs[i]);
    }
    for (int j = 0; j < S->ncon; j++)
        if (S->cons[j].src != SRC_ROWS) assemble_joint(S, &S->cons[j]);
}

/* position-level value phi of a rigid-model constraint at the current state */
void orc_joint_phi(orc_scene *S, int j, double *phi)
{
    double Ja[30], Jb[30];
    joint_rows(S, &S->cons[j], phi, Ja, Jb);
}

/* node k of linear block i: x[3], v[3] */
void orc_get_node(orc_scene *S, int i, int k, double *out)
{
    sub_t *u = &S->subs[i];
    memcpy(out, u->x + 3 * k, 3 * sizeof(double));
    memcpy(out + 3, u->vel + 3 * k, 3 * sizeof(double));
}

void orc_set_node(orc_scene *S, int i, int k, const double *in)
{
    sub_t *u = &S->subs[i];
    memcpy(u->x + 3 * k, in, 3 * sizeof(double));
    memcpy(u->vel + 3 * k, in + 3, 3 * sizeof(double));
}

void orc_get_body(orc_scene *S, int i, int k, double *out)
{
    body_t *B = &S->subs[i].bodies[k];
    out[0] = B->m;
    memcpy(out + 1, B->I, 3 * sizeof(double));
    memcpy(out + 4, B->p, 3 * sizeof(double));
    memcpy(out + 7, B->q, 4 * sizeof(double));
    memcpy(out + 11, B->v, 3 * sizeof(double));
    memcpy(out + 14, B->w, 3 * sizeof(double));
}

void orc_set_body(orc_scene *S, int i, int k, const double *in)
{
    body_t *B = &S->subs[i].bodies[k];
    B->m = in[0];
    memcpy(B->I, in + 1, 3 * sizeof(double));
    memcpy(B->p, in + 4, 3 * sizeof(double));
    memcpy(B->q, in + 7, 4 * sizeof(double));
    memcpy(B->v, in + 11, 3 * sizeof(double));
    memcpy(B->w, in + 14, 3 * sizeof(double));
}

/* Sets constraint j's warm-start state, as a finished step leaves it: lambda (rows) and z
   (sides x rows).  Lets a test start the oracle from a state reached elsewhere. */
void orc_set_warm(orc_scene *S, int j, const double *lam, const double *z)
{
    con_t *c = &S->cons[j];
    memcpy(c->lamprev, lam, sizeof(double) * c->rows);
    memcpy(c->zprev, z, sizeof(double) * c->rows * c->ns);
    c->has_prev = 1;
}

void orc_set_generic(orc_scene *S, int i, const double *A, const double *b)
{
    sub_t *u = &S->subs[i];
    if (A) memcpy(u->A, A, sizeof(double) * (size_t)u->n * u->n);
    if (b) memcpy(u->b, b, sizeof(double) * u->n);
}

/* out: r_p, r_d, theta, iters, converged, status */
void orc_residuals(orc_scene *S, double *out)
{
    out[0] = S->r_p; out[1] = S->r_d; out[2] = S->theta;
    out[3] = S->iters; out[4] = S->converged; out[5] = S->status;
}

/* standalone dense SPD solve through the oracle's Cholesky (for pins) */
int orc_chol_solve(int n, const double *K, const double *r, double *x)
{
    double *L = (double *)xcalloc((size_t)n * n, sizeof(double));
    int rc = cholesky(n, K, L);
    if (!rc) { memcpy(x, r, sizeof(double) * n); chol_solve(n, L, x); }
    free(L);
    return rc;
}

void orc_free(orc_scene *S)
{
    if (!S) return;
    for (int i = 0; i < S->nsub; i++) {
        sub_t *u = &S->subs[i];
        free(u->A); free(u->b); free(u->L); free(u->v); free(u->rhs); free(u->bodies);
        free(u->mass); free(u->Kel); free(u->fext); free(u->X0); free(u->x); free(u->vel);
        free(u->tets); free(u->Ke);
    }
    for (int j = 0; j < S->ncon; j++) {
        con_t *c = &S->cons[j];
        for (int s = 0; s < c->ns; s++) free(c->J[s]);
        free(c->e); free(c->x); free(c->z); free(c->u); free(c->y); free(c->yold);
        free(c->zold); free(c->zprev); free(c->lam); free(c->lamprev);
    }
    free(S->subs); free(S->cons); free(S);
}
