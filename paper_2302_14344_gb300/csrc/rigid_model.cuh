// Rigid-body model on the device: the per-step construction of A_i, b_i (Eq. ddyn with
// v_{k+1} = 2 v-hat - v_k substituted, so A_i = (2/h) M_i, b_i = (2/h) M_i v_k - C v_k + f)
// and of the rows J_j, e_j of ball, revolute, PD-drive and plane-contact constraints
// (Sec. II-A), plus the state update that ends each step of Algorithm 1.
//
// Body record (17 doubles): m, I[3] (principal, body frame), p[3], q[4] (w, x, y, z),
// v[3] (world), w[3] (body frame).  Generalized velocity per body: [v, w].
#pragma once
#include "layout.h"

namespace subadmm {

struct Rot { double r[9]; };

__device__ __forceinline__ Rot quat_rot(const double *q)
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    Rot R;
    R.r[0] = 1.0 - 2.0 * (y * y + z * z); R.r[1] = 2.0 * (x * y - w * z); R.r[2] = 2.0 * (x * z + w * y);
    R.r[3] = 2.0 * (x * y + w * z); R.r[4] = 1.0 - 2.0 * (x * x + z * z); R.r[5] = 2.0 * (y * z - w * x);
    R.r[6] = 2.0 * (x * z - w * y); R.r[7] = 2.0 * (y * z + w * x); R.r[8] = 1.0 - 2.0 * (x * x + y * y);
    return R;
}

__device__ __forceinline__ void mul(const Rot &R, const double *a, double *o)
{
    o[0] = R.r[0] * a[0] + R.r[1] * a[1] + R.r[2] * a[2];
    o[1] = R.r[3] * a[0] + R.r[4] * a[1] + R.r[5] * a[2];
    o[2] = R.r[6] * a[0] + R.r[7] * a[1] + R.r[8] * a[2];
}

// R^T c, i.e. the row vector c^T R
__device__ __forceinline__ void mulT(const Rot &R, const double *c, double *o)
{
    o[0] = R.r[0] * c[0] + R.r[3] * c[1] + R.r[6] * c[2];
    o[1] = R.r[1] * c[0] + R.r[4] * c[1] + R.r[7] * c[2];
    o[2] = R.r[2] * c[0] + R.r[5] * c[1] + R.r[8] * c[2];
}

__device__ __forceinline__ void cross(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Row of the velocity of body point p + R r along world direction d:
// d . (v + R (w x r)) = d . v + w . (r x R^T d)
__device__ __forceinline__ void point_row(const double *d, const Rot &R, const double *r, double *row)
{
    double Rd[3];
    mulT(R, d, Rd);
    row[0] = d[0]; row[1] = d[1]; row[2] = d[2];
    cross(r, Rd, row + 3);
}

// Contact frame of a unit normal n: rows n, t1, t2 with t1 the world x axis (y when
// |n_x| > 0.9) with its n component removed, normalised, and t2 = n x t1; for n = +z the
// frame is (z, x, y).
__device__ __forceinline__ void contact_frame(const double *n, double F[3][3])
{
    const bool near_x = fabs(n[0]) > 0.9;
    const double ex = near_x ? 0.0 : 1.0, ey = near_x ? 1.0 : 0.0;
    const double en = ex * n[0] + ey * n[1];
    double t[3] = {ex - en * n[0], ey - en * n[1], -en * n[2]};
    const double inv = 1.0 / sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int q = 0; q < 3; ++q) { t[q] *= inv; F[0][q] = n[q]; F[1][q] = t[q]; }
    cross(n, t, F[2]);
}

// A side of a model constraint: a rigid body (its point p + R anchor, rows of 6 columns
// [v, w]) or a node of a linear block (its position, rows of 3 columns: its velocity).
struct Side {
    bool node;
    const double *p;
    Rot R;
};

__device__ __forceinline__ Side make_side(bool node, const double *rec)
{
    Side s;
    s.node = node;
    if (node) {
        s.p = rec;                                  // x[3], then v[3]
        for (int q = 0; q < 9; ++q) s.R.r[q] = (q % 4 == 0) ? 1.0 : 0.0;
    } else {
        s.p = rec + 4;
        s.R = quat_rot(rec + 7);
    }
    return s;
}

__device__ __forceinline__ void side_point(const Side &s, const double *anc, double *P)
{
    if (s.node) { P[0] = s.p[0]; P[1] = s.p[1]; P[2] = s.p[2]; return; }
    double r[3];
    mul(s.R, anc, r);
    for (int d = 0; d < 3; ++d) P[d] = s.p[d] + r[d];
}

__device__ __forceinline__ void side_row(const Side &s, const double *dir, const double *anc, double *row)
{
    if (s.node) { row[0] = dir[0]; row[1] = dir[1]; row[2] = dir[2]; return; }
    point_row(dir, s.R, anc, row);
}

// Rows of a model constraint: Ja, Jb are rows x 6 blocks of sides a and b (a node side
// uses the first 3 columns), e the error terms; k, alpha (soft) are returned for ANGLE_PD.
__device__ void model_rows(const ConDesc &c, const double *prm, const double *bodies,
                           const double *nodes, double h, double gamma, double *Ja, double *Jb,
                           double *e, double *k_out, double *alpha_out)
{
    const double ih = 1.0 / h;
    const Side sa = make_side(c.node_a, c.node_a ? nodes + (size_t)c.gb_a * SUBADMM_NODE
                                                 : bodies + (size_t)c.gb_a * SUBADMM_BODY);
    const bool hasb = c.gb_b >= 0;
    Side sb;
    if (hasb)
        sb = make_side(c.node_b, c.node_b ? nodes + (size_t)c.gb_b * SUBADMM_NODE
                                          : bodies + (size_t)c.gb_b * SUBADMM_BODY);
    const Rot &Ra = sa.R;
    const double *anc_a = prm + 0, *anc_b = prm + 3, *ax_a = prm + 6, *ax_b = prm + 9;
    const double *ref_a = prm + 12, *ref_b = prm + 15;
    for (int q = 0; q < 6 * c.rows; ++q) { Ja[q] = 0.0; Jb[q] = 0.0; }
    if (c.src == SRC_BALL || c.src == SRC_REVOLUTE) {
        double pa[3], pb[3];
        side_point(sa, anc_a, pa);
        if (hasb) side_point(sb, anc_b, pb);
        else { pb[0] = anc_b[0]; pb[1] = anc_b[1]; pb[2] = anc_b[2]; }
        for (int d = 0; d < 3; ++d) {
            const double E[3] = {d == 0 ? 1.0 : 0.0, d == 1 ? 1.0 : 0.0, d == 2 ? 1.0 : 0.0};
            side_row(sa, E, anc_a, Ja + 6 * d);
            if (hasb) {
                side_row(sb, E, anc_b, Jb + 6 * d);
                for (int q = 0; q < 6; ++q) Jb[6 * d + q] = -Jb[6 * d + q];
            }
            e[d] = gamma * (pa[d] - pb[d]) * ih;
        }
        if (c.src == SRC_REVOLUTE) {
            // revolute joints join rigid bodies only (the host rejects node sides)
            double ub[3], t[2][3], axr[3];
            if (hasb) mul(sb.R, ax_b, ub); else { ub[0] = ax_b[0]; ub[1] = ax_b[1]; ub[2] = ax_b[2]; }
            mul(Ra, ref_a, t[0]);
            cross(ax_a, ref_a, axr);
            mul(Ra, axr, t[1]);
            for (int kk = 0; kk < 2; ++kk) {
                const int r = 3 + kk;
                double txu[3], ja[3];
                cross(t[kk], ub, txu);          // d/dt (t . u_b) = (t x u_b) . (w_a - w_b)
                mulT(Ra, txu, ja);
                for (int q = 0; q < 3; ++q) Ja[6 * r + 3 + q] = ja[q];
                if (hasb) {
                    double jb[3];
                    mulT(sb.R, txu, jb);
                    for (int q = 0; q < 3; ++q) Jb[6 * r + 3 + q] = -jb[q];
                }
                e[r] = gamma * dot(t[kk], ub) * ih;
            }
        }
    } else if (c.src == SRC_ANGLE_PD) {
        double u[3], na[3], nb[3], cr[3], ja[3];
        mul(Ra, ax_a, u);
        mul(Ra, ref_a, na);
        if (hasb) mul(sb.R, ref_b, nb); else { nb[0] = ref_b[0]; nb[1] = ref_b[1]; nb[2] = ref_b[2]; }
        cross(na, nb, cr);
        const double theta = atan2(dot(cr, u), dot(na, nb));
        mulT(Ra, u, ja);                        // d theta / dt = u . (w_b - w_a)
        for (int q = 0; q < 3; ++q) Ja[3 + q] = -ja[q];
        if (hasb) {
            double jb[3];
            mulT(sb.R, u, jb);
            for (int q = 0; q < 3; ++q) Jb[3 + q] = jb[q];
        }
        const double kp = prm[18], kd = prm[19];
        e[0] = theta - prm[20];
        *k_out = kp;
        *alpha_out = kd / kp + 0.5 * h;
    } else if (c.src == SRC_PLANE || c.src == SRC_SPHERE) {
        // a sphere of radius ref_a[0] about point a against the plane n . x = plane_z (n =
        // axis_b, unit), or against the sphere of radius ref_b[0] about point b (n from b's
        // centre to a's, +z for coincident centres); rows of the relative velocity of the
        // two surface points along the contact frame of n
        double pa[3], n[3], gap;
        const double ra = ref_a[0];
        side_point(sa, anc_a, pa);
        if (c.src == SRC_PLANE) {
            n[0] = ax_b[0]; n[1] = ax_b[1]; n[2] = ax_b[2];
            gap = dot(n, pa) - prm[21] - ra;
        } else {
            double pb[3];
            if (hasb) side_point(sb, anc_b, pb);
            else { pb[0] = anc_b[0]; pb[1] = anc_b[1]; pb[2] = anc_b[2]; }
            const double d[3] = {pa[0] - pb[0], pa[1] - pb[1], pa[2] - pb[2]};
            const double dist = sqrt(dot(d, d));
            n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
            if (dist > 0.0) { n[0] = d[0] / dist; n[1] = d[1] / dist; n[2] = d[2] / dist; }
            gap = dist - ra - ref_b[0];
        }
        double F[3][3];
        contact_frame(n, F);
        double ca[3], cb[3], rn[3];
        mulT(Ra, n, rn);
        for (int q = 0; q < 3; ++q) ca[q] = anc_a[q] - ra * rn[q];
        if (c.src == SRC_SPHERE && hasb && !sb.node) {
            mulT(sb.R, n, rn);
            for (int q = 0; q < 3; ++q) cb[q] = anc_b[q] + ref_b[0] * rn[q];
        } else {
            for (int q = 0; q < 3; ++q) cb[q] = anc_b[q];
        }
        for (int d = 0; d < 3; ++d) {
            side_row(sa, F[d], ca, Ja + 6 * d);
            if (c.src == SRC_SPHERE && hasb) {
                side_row(sb, F[d], cb, Jb + 6 * d);
                for (int q = 0; q < 6; ++q) Jb[6 * d + q] = -Jb[6 * d + q];
            }
        }
        e[0] = gap >= 0.0 ? gap * ih : gamma * gap * ih;
        e[1] = 0.0;
        e[2] = 0.0;
    }
}

// Diagonal of A_i = (2/h) M and b_i for one body (6 entries each).
__device__ __forceinline__ void body_dynamics(const double *B, double h, double g0, double g1,
                                              double g2, double *Adiag, double *b)
{
    const double c2h = 2.0 / h;
    const double m = B[0];
    const double *I = B + 1, *v = B + 11, *w = B + 14;
    const double g[3] = {g0, g1, g2};
    double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]};
    double gyro[3];
    cross(w, Iw, gyro);
    for (int d = 0; d < 3; ++d) {
        Adiag[d] = c2h * m;
        Adiag[3 + d] = c2h * I[d];
        b[d] = c2h * m * v[d] + m * g[d];
        b[3 + d] = c2h * Iw[d] - gyro[d];
    }
}

// Linear elastic block (Eq. ddyn with the elastic force at the midpoint): the diagonal part
// (2/h) m of A and b_p = (2/h) m v_p - (K (x - X0))_p + f_p + m g_p (K sparse, CSR), a lane
// per row; ux = x - X0 staged by the caller.  Two partial sums keep two gathers in flight.
__device__ __forceinline__ double linear_b(int p, const double *mass, const double *f,
                                           const double *ux, const double *Kval, const int *rowp,
                                           const int *col, const double *nodes, double h,
                                           const double *g)
{
    double k0 = 0.0, k1 = 0.0;
    int q = rowp[p];
    const int q1 = rowp[p + 1];
    for (; q + 1 < q1; q += 2) {
        k0 += Kval[q] * ux[col[q]];
        k1 += Kval[q + 1] * ux[col[q + 1]];
    }
    if (q < q1) k0 += Kval[q] * ux[col[q]];
    const double m = mass[p / 3];
    return (2.0 / h) * m * nodes[(p / 3) * SUBADMM_NODE + 3 + p % 3] - (k0 + k1) + f[p] + m * g[p % 3];
}

// Co-rotational tetrahedron (the beam model of Sec. IV-A): R, the rotation of the element's
// deformation gradient F = Ds Dm^-1 (Ds, Dm: edge matrices of the current and rest positions)
// by Newton's polar iteration R <- (R + R^-T) / 2 from R = F; then (h/2) R K_e R^T (R on every
// node's 3 x 3 block) is added into the block's K and -R K_e (R^T x_e - X_e) into b.  K row-
// major n x n, full symmetric band; atomics, since elements share nodes.
__device__ __forceinline__ void inv3_cof(const double *M, double *c, double &det)
{
    c[0] = M[4] * M[8] - M[5] * M[7];
    c[1] = M[5] * M[6] - M[3] * M[8];
    c[2] = M[3] * M[7] - M[4] * M[6];
    c[3] = M[2] * M[7] - M[1] * M[8];
    c[4] = M[0] * M[8] - M[2] * M[6];
    c[5] = M[1] * M[6] - M[0] * M[7];
    c[6] = M[1] * M[5] - M[2] * M[4];
    c[7] = M[2] * M[3] - M[0] * M[5];
    c[8] = M[0] * M[4] - M[1] * M[3];
    det = M[0] * c[0] + M[1] * c[1] + M[2] * c[2];
}

__device__ void corot_element(const int *tet, const double *Ke, const double *X0,
                              const double *nodes, double h, int n, double *K, double *b)
{
    double Dm[9], Ds[9];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) {
            Dm[3 * d + k] = X0[3 * tet[k + 1] + d] - X0[3 * tet[0] + d];
            Ds[3 * d + k] = nodes[tet[k + 1] * SUBADMM_NODE + d] - nodes[tet[0] * SUBADMM_NODE + d];
        }
    double c[9], det;
    inv3_cof(Dm, c, det);
    double F[9], R[9];
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 3; ++q) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += Ds[3 * a + k] * c[3 * q + k];
            F[3 * a + q] = acc / det;
        }
    for (int k = 0; k < 9; ++k) R[k] = F[k];
    for (int it = 0; it < 60; ++it) {
        double rd;
        inv3_cof(R, c, rd);
        double dd = 0.0, nrm = 0.0;
        for (int k = 0; k < 9; ++k) {
            const double nk = 0.5 * (R[k] + c[k] / rd);
            dd += (nk - R[k]) * (nk - R[k]);
            nrm += nk * nk;
            R[k] = nk;
        }
        if (dd <= 1e-30 * nrm) break;
    }
    double w[12], g[12];
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) {
            const double *xa = nodes + tet[a] * SUBADMM_NODE;
            w[3 * a + d] = R[d] * xa[0] + R[3 + d] * xa[1] + R[6 + d] * xa[2] - X0[3 * tet[a] + d];
        }
    for (int i = 0; i < 12; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 12; ++j) acc += Ke[12 * i + j] * w[j];
        g[i] = acc;
    }
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d)
            atomicAdd(&b[3 * tet[a] + d],
                      -(R[3 * d] * g[3 * a] + R[3 * d + 1] * g[3 * a + 1] + R[3 * d + 2] * g[3 * a + 2]));
    const double hh = 0.5 * h;
    for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 4; ++q) {
            double T[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * Ke[12 * (3 * a + k) + 3 * q + j];
                    T[3 * i + j] = acc;
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double v = T[3 * i] * R[3 * j] + T[3 * i + 1] * R[3 * j + 1] + T[3 * i + 2] * R[3 * j + 2];
                    atomicAdd(&K[(size_t)(3 * tet[a] + i) * n + 3 * tet[q] + j], hh * v);
                }
        }
}

// v_{k+1} = 2 v-hat - v_k; p += h v-hat; q <- q (x) Exp(h w-hat), renormalised.
__device__ __forceinline__ void body_update(double *B, const double *vh, double h)
{
    for (int d = 0; d < 3; ++d) {
        B[4 + d] += h * vh[d];
        B[11 + d] = 2.0 * vh[d] - B[11 + d];
        B[14 + d] = 2.0 * vh[3 + d] - B[14 + d];
    }
    const double a0 = h * vh[3], a1 = h * vh[4], a2 = h * vh[5];
    const double th = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    double dq[4];
    if (th > 0.0) {
        double sn, cs;
        sincos(0.5 * th, &sn, &cs);
        sn /= th;
        dq[0] = cs; dq[1] = a0 * sn; dq[2] = a1 * sn; dq[3] = a2 * sn;
    } else {
        dq[0] = 1.0; dq[1] = 0.0; dq[2] = 0.0; dq[3] = 0.0;
    }
    double *q = B + 7;
    double nq[4];
    nq[0] = q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] - q[3] * dq[3];
    nq[1] = q[0] * dq[1] + q[1] * dq[0] + q[2] * dq[3] - q[3] * dq[2];
    nq[2] = q[0] * dq[2] - q[1] * dq[3] + q[2] * dq[0] + q[3] * dq[1];
    nq[3] = q[0] * dq[3] + q[1] * dq[2] - q[2] * dq[1] + q[3] * dq[0];
    const double inv = 1.0 / sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int d = 0; d < 4; ++d) q[d] = nq[d] * inv;
}

}  // namespace subadmm
