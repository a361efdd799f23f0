/*
 * FP64 CPU oracle for the boundary-element electrostatics model of
 * Yokota, Bardhan, Knepley, Barba & Hamada (arXiv:1007.4591).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never links, calls or falls back to it.  It shares no
 * code, header, table or constant with the CUDA sources.
 *
 * Everything here is the plain dense definition of the discrete operators:
 * no tree, no expansions, no near/far split, no blocking.  Every pair of
 * distinct panels uses the same quadrature rule.  OpenMP parallelises only
 * the loop over targets (each target's sum is accumulated serially in the
 * source order, so results do not depend on the thread count).
 *
 * Notation (Sec. 2.1, Eqs. ASC and reac):
 *   panels j: vertices v0, v1, v2 (counter-clockwise seen from the solvent),
 *   unit normal n_j = (v1-v0)x(v2-v0)/|.|, area A_j, centroid c_j,
 *   quadrature points y_jq with weights w_q (sum w_q = 1),
 *   Green's function G(r) = 1/(4 pi r),
 *   K'_ij = A_j sum_q w_q [-(c_i - y_jq).n_i] / (4 pi |c_i - y_jq|^3), K'_ii = 0,
 *   (B q)_i = sum_k q_k [-(c_i - x_k).n_i] / (4 pi |c_i - x_k|^3),
 *   (C s)_k = sum_j s_j A_j sum_q w_q / (4 pi |x_k - y_jq|).
 *
 * K'_ii = 0: for a flat panel (c_i - y).n_i vanishes for every y in panel i,
 * so the principal-value self integral of the normal derivative is exactly
 * zero; the jump term of the interior limit is carried by the identity in
 * A = I + Ehat K'.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FOUR_PI 12.566370614359172953850573533118

/* ------------------------------------------------------------------ */
/* Quadrature on a triangle.                                           */
/* nq = 1: the centroid (the paper's one-point rule, Sec. 2.1).        */
/* nq = 7: Radon's degree-5 rule (Stroud, "Approximate Calculation of  */
/*         Multiple Integrals", 1971, formula T2:5-1): the centroid    */
/*         with weight 9/40, the three permutations of (a, a, 1-2a),   */
/*         a = (6 - sqrt15)/21, weight (155 - sqrt15)/1200, and the    */
/*         three permutations of (b, b, 1-2b), b = (6 + sqrt15)/21,    */
/*         weight (155 + sqrt15)/1200.  Weights sum to one.            */
/* ------------------------------------------------------------------ */
int oracle_quad_rule(int nq, double *bary, double *w)
{
    if (nq == 1) {
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 1.0;
        return 0;
    }
    if (nq != 7) return -1;
    const double s15 = sqrt(15.0);
    const double a = (6.0 - s15) / 21.0, b = (6.0 + s15) / 21.0;
    const double wa = (155.0 - s15) / 1200.0, wb = (155.0 + s15) / 1200.0;
    const double pts[7][3] = {
        {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
        {a, a, 1.0 - 2.0 * a}, {a, 1.0 - 2.0 * a, a}, {1.0 - 2.0 * a, a, a},
        {b, b, 1.0 - 2.0 * b}, {b, 1.0 - 2.0 * b, b}, {1.0 - 2.0 * b, b, b},
    };
    const double wt[7] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    for (int q = 0; q < 7; ++q) {
        for (int k = 0; k < 3; ++k) bary[3 * q + k] = pts[q][k];
        w[q] = wt[q];
    }
    return 0;
}

/* Panel geometry: centroid, unit normal, area and quadrature points
 * y_jq = sum_k bary_qk v_k with the weights A_j w_q (Sec. 2.1: flat
 * triangular panels, piecewise-constant basis). */
int oracle_geometry(const double *panels, int64_t n, int nq,
                    double *cen, double *nrm, double *area,
                    double *qp, double *qw)
{
    double bary[21], w[7];
    if (oracle_quad_rule(nq, bary, w)) return -1;
    for (int64_t j = 0; j < n; ++j) {
        const double *v0 = panels + 9 * j, *v1 = v0 + 3, *v2 = v0 + 6;
        double e1[3], e2[3], cr[3];
        for (int k = 0; k < 3; ++k) { e1[k] = v1[k] - v0[k]; e2[k] = v2[k] - v0[k]; }
        cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
        cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
        cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        if (!(len > 0.0)) return -2;
        area[j] = 0.5 * len;
        for (int k = 0; k < 3; ++k) {
            nrm[3 * j + k] = cr[k] / len;
            cen[3 * j + k] = (v0[k] + v1[k] + v2[k]) / 3.0;
        }
        for (int q = 0; q < nq; ++q) {
            for (int k = 0; k < 3; ++k)
                qp[(j * nq + q) * 3 + k] = bary[3 * q] * v0[k] + bary[3 * q + 1] * v1[k]
                                          + bary[3 * q + 2] * v2[k];
            qw[j * nq + q] = area[j] * w[q];
        }
    }
    return 0;
}

/* Normal derivative at target t (normal n) of the potential of a unit
 * source at s:  d/dn_t [1/(4 pi |t - s|)] = -(t - s).n / (4 pi |t - s|^3). */
static inline double dn_green(const double *t, const double *n, const double *s)
{
    double d0 = t[0] - s[0], d1 = t[1] - s[1], d2 = t[2] - s[2];
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    double r = sqrt(r2);
    return -(d0 * n[0] + d1 * n[1] + d2 * n[2]) / (FOUR_PI * r2 * r);
}

static inline double green(const double *a, const double *b)
{
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return 1.0 / (FOUR_PI * sqrt(d0 * d0 + d1 * d1 + d2 * d2));
}

/* K'_ij for one pair (i != j), Eq. ASC discretised by collocation at c_i. */
static inline double kprime_entry(int64_t i, int64_t j, int nq, const double *cen,
                                  const double *nrm, const double *qp, const double *qw)
{
    double acc = 0.0;
    for (int q = 0; q < nq; ++q)
        acc += qw[j * nq + q] * dn_green(cen + 3 * i, nrm + 3 * i, qp + 3 * (j * nq + q));
    return acc;
}

/* y = K' x  (dense, O(n^2)). */
void oracle_kprime(int64_t n, int nq, const double *cen, const double *nrm,
                   const double *qp, const double *qw, const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            acc += kprime_entry(i, j, nq, cen, nrm, qp, qw) * x[j];
        }
        y[i] = acc;
    }
}

/* y = K' x for a subset of target rows only (sampled parity at large n). */
void oracle_kprime_rows(int64_t n, int nq, const double *cen, const double *nrm,
                        const double *qp, const double *qw, const double *x,
                        int64_t nrows, const int64_t *rows, double *y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            acc += kprime_entry(i, j, nq, cen, nrm, qp, qw) * x[j];
        }
        y[r] = acc;
    }
}

/* y = K'^T x, i.e. y_j = sum_{i != j} K'_ij x_i (each output its own serial sum). */
void oracle_kprime_t(int64_t n, int nq, const double *cen, const double *nrm,
                     const double *qp, const double *qw, const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (i == j) continue;
            acc += kprime_entry(i, j, nq, cen, nrm, qp, qw) * x[i];
        }
        y[j] = acc;
    }
}

/* Dense K' (row-major n x n), small n only. */
void oracle_kprime_dense(int64_t n, int nq, const double *cen, const double *nrm,
                         const double *qp, const double *qw, double *K)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            K[i * n + j] = (i == j) ? 0.0 : kprime_entry(i, j, nq, cen, nrm, qp, qw);
}

/* ------------------------------------------------------------------ */
/* Exact integrals over one flat triangle T (vertices a0, a1, a2, unit  */
/* normal nu = (a1-a0)x(a2-a0)/|.|) of the field of a unit surface      */
/* density, for the near-singular pairs (higher-accuracy panel          */
/* integration: Sec. 2.1 names analytic panel integrals for flat      */
/* elements as the alternative to quadrature).  With R = |t - y|       */
/* and h = (t - a0).nu, split t - y into its normal part h nu and its   */
/* in-plane part:                                                       */
/*   * the normal part integrates to nu * W(t), W(t) = int_T h/R^3 dA,  */
/*     the solid angle of T seen from t, positive when t lies on the    */
/*     side nu points to;                                               */
/*   * the in-plane part is the in-plane gradient of 1/R with respect   */
/*     to y, so by the divergence theorem in the plane it becomes       */
/*     sum over edges e = (p -> q) of m_e * int_e dl / R, where m_e is  */
/*     the edge's outward in-plane normal and                           */
/*     int_e dl / R = asinh(s_q / d) - asinh(s_p / d)                   */
/*                  = log((R_q + s_q) / (R_p + s_p)),                   */
/*     s the coordinate along the edge measured from the foot of t.     */
/* So  int_T (t - y)/R^3 dA = nu W(t) + sum_e m_e log(...), and the     */
/* K' entry (collocation at t with normal n) is                         */
/*   int_T -(t - y).n / (4 pi R^3) dA = -n.(nu W + sum_e m_e L_e)/(4pi).*/
/* ------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *c)
{
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* W(t) = int_T h / R^3 dA by the triple-product formula for the solid angle
 * of a triangle (Van Oosterom and Strackee, IEEE Trans. Biomed. Eng. 30,
 * 1983): with r_k = a_k - t,
 *   tan(W'/2) = r0.(r1 x r2) / (|r0||r1||r2| + (r0.r1)|r2| + (r0.r2)|r1| + (r1.r2)|r0|),
 * where W' is positive when the vertices appear counter-clockwise from t,
 * i.e. when t lies on the side opposite to nu; hence W = -W'. */
double oracle_solid_angle(const double *t, const double *tri)
{
    double r0[3], r1[3], r2[3], c[3];
    sub3(tri, t, r0);
    sub3(tri + 3, t, r1);
    sub3(tri + 6, t, r2);
    const double l0 = norm3(r0), l1 = norm3(r1), l2 = norm3(r2);
    cross3(r1, r2, c);
    const double num = dot3(r0, c);
    const double den = l0 * l1 * l2 + dot3(r0, r1) * l2 + dot3(r0, r2) * l1 + dot3(r1, r2) * l0;
    return -2.0 * atan2(num, den);
}

/* int_e dl / |t - y| along the segment p -> q (length > 0). */
static double edge_log(const double *t, const double *p, const double *q)
{
    double e[3], dp[3], dq[3];
    sub3(q, p, e);
    const double len = norm3(e);
    for (int k = 0; k < 3; ++k) e[k] /= len;
    sub3(p, t, dp);
    sub3(q, t, dq);
    const double sp = dot3(dp, e), sq = dot3(dq, e);
    const double Rp = norm3(dp), Rq = norm3(dq);
    /* the two algebraically equal forms; take the one without cancellation */
    if (sp + sq >= 0.0) return log((Rq + sq) / (Rp + sp));
    return log((Rp - sp) / (Rq - sq));
}

/* int_T -(t - y).n / (4 pi |t - y|^3) dA_y for a flat triangle tri[3][3]. */
double oracle_panel_dn(const double *t, const double *n, const double *tri)
{
    double e1[3], e2[3], nu[3];
    sub3(tri + 3, tri, e1);
    sub3(tri + 6, tri, e2);
    cross3(e1, e2, nu);
    const double ln = norm3(nu);
    for (int k = 0; k < 3; ++k) nu[k] /= ln;
    double v[3] = {0.0, 0.0, 0.0};
    const double W = oracle_solid_angle(t, tri);
    for (int k = 0; k < 3; ++k) v[k] = nu[k] * W;
    for (int e = 0; e < 3; ++e) {
        const double *p = tri + 3 * e, *q = tri + 3 * ((e + 1) % 3);
        double te[3], m[3];
        sub3(q, p, te);
        const double lt = norm3(te);
        for (int k = 0; k < 3; ++k) te[k] /= lt;
        cross3(te, nu, m);                     /* outward in-plane normal (CCW about nu) */
        const double L = edge_log(t, p, q);
        for (int k = 0; k < 3; ++k) v[k] += m[k] * L;
    }
    return -dot3(n, v) / FOUR_PI;
}

/* int_T dA_y / (4 pi |t - y|) for a flat triangle tri[3][3] (the single-layer
 * potential of a unit density, Sec. 2.1's G integrated over one panel).  In
 * the plane of T let rho0 be the foot of t, h = (t - a0).nu its height and,
 * for each edge e from p to q with outward in-plane normal m_e,
 * d_e = m_e.(p - t) the distance of rho0 from the edge's line (positive on
 * the inner side).  The 2D field F(rho) = (rho - rho0)(R - |h|)/|rho - rho0|^2
 * has divergence 1/R in the plane, so the divergence theorem gives
 *   int_T dA / R = sum_e d_e int_e (R - |h|)/s^2 dl
 *                = sum_e d_e L_e - |h| int_T |h| / R^3 dA
 * (s = |rho - rho0|, L_e = int_e dl / R), and the last integral is the
 * magnitude of the solid angle W, so |h| |W| = h W. */
double oracle_panel_phi(const double *t, const double *tri)
{
    double e1[3], e2[3], nu[3], a0t[3];
    sub3(tri + 3, tri, e1);
    sub3(tri + 6, tri, e2);
    cross3(e1, e2, nu);
    const double ln = norm3(nu);
    for (int k = 0; k < 3; ++k) nu[k] /= ln;
    sub3(t, tri, a0t);
    const double h = dot3(a0t, nu);
    double acc = -h * oracle_solid_angle(t, tri);
    for (int e = 0; e < 3; ++e) {
        const double *p = tri + 3 * e, *q = tri + 3 * ((e + 1) % 3);
        double te[3], m[3], pt[3];
        sub3(q, p, te);
        const double lt = norm3(te);
        for (int k = 0; k < 3; ++k) te[k] /= lt;
        cross3(te, nu, m);
        sub3(p, t, pt);
        const double d = dot3(m, pt);
        if (d != 0.0) acc += d * edge_log(t, p, q);
    }
    return acc / FOUR_PI;
}

/* grad_t of oracle_panel_phi: -int_T (t - y) / (4 pi |t - y|^3) dA, the
 * field whose projection on n is oracle_panel_dn (solid angle along the
 * normal, one edge logarithm per edge in the plane). */
void oracle_panel_grad_phi(const double *t, const double *tri, double *g)
{
    double e1[3], e2[3], nu[3];
    sub3(tri + 3, tri, e1);
    sub3(tri + 6, tri, e2);
    cross3(e1, e2, nu);
    const double ln = norm3(nu);
    for (int k = 0; k < 3; ++k) nu[k] /= ln;
    const double W = oracle_solid_angle(t, tri);
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = nu[k] * W;
    for (int e = 0; e < 3; ++e) {
        const double *p = tri + 3 * e, *q = tri + 3 * ((e + 1) % 3);
        double te[3], m[3];
        sub3(q, p, te);
        const double lt = norm3(te);
        for (int k = 0; k < 3; ++k) te[k] /= lt;
        cross3(te, nu, m);
        const double L = edge_log(t, p, q);
        for (int k = 0; k < 3; ++k) v[k] += m[k] * L;
    }
    for (int k = 0; k < 3; ++k) g[k] = -v[k] / FOUR_PI;
}

/* Charge-panel entries with the higher-accuracy panel integration of the
 * near-singular pairs: a charge x_k closer than 2.5 sqrt(A_j) to the centroid
 * of panel j takes the exact single-layer integral over the flat panel (and
 * its gradient), every other pair the quadrature rule.  phi = C s, v = C^T u,
 * g = grad_x (C s); panels[n][3][3], cen[n][3], area[n]. */
static int charge_near(const double *x, const double *cen, const double *area, int64_t j)
{
    double d[3];
    sub3(x, cen + 3 * j, d);
    return dot3(d, d) <= 6.25 * area[j];
}

void oracle_c_exact(int64_t n, int nq, const double *qp, const double *qw, const double *cen,
                    const double *area, const double *panels, int64_t nc, const double *xq,
                    const double *s, double *phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        const double *x = xq + 3 * k;
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double pj = 0.0;
            if (charge_near(x, cen, area, j))
                pj = oracle_panel_phi(x, panels + 9 * j);
            else
                for (int q = 0; q < nq; ++q) pj += qw[j * nq + q] * green(x, qp + 3 * (j * nq + q));
            acc += s[j] * pj;
        }
        phi[k] = acc;
    }
}

void oracle_ct_exact(int64_t n, int nq, const double *qp, const double *qw, const double *cen,
                     const double *area, const double *panels, int64_t nc, const double *xq,
                     const double *u, double *v)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t k = 0; k < nc; ++k) {
            const double *x = xq + 3 * k;
            double pj = 0.0;
            if (charge_near(x, cen, area, j))
                pj = oracle_panel_phi(x, panels + 9 * j);
            else
                for (int q = 0; q < nq; ++q) pj += qw[j * nq + q] * green(x, qp + 3 * (j * nq + q));
            acc += u[k] * pj;
        }
        v[j] = acc;
    }
}

void oracle_grad_c_exact(int64_t n, int nq, const double *qp, const double *qw, const double *cen,
                         const double *area, const double *panels, int64_t nc, const double *xq,
                         const double *s, double *g /*[nc][3]*/)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        const double *x = xq + 3 * k;
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (charge_near(x, cen, area, j)) {
                double gj[3];
                oracle_panel_grad_phi(x, panels + 9 * j, gj);
                for (int c = 0; c < 3; ++c) a[c] += s[j] * gj[c];
            } else {
                for (int q = 0; q < nq; ++q) {
                    const double *y = qp + 3 * (j * nq + q);
                    double d[3];
                    sub3(x, y, d);
                    const double r2 = dot3(d, d), r = sqrt(r2);
                    const double f = -s[j] * qw[j * nq + q] / (FOUR_PI * r2 * r);
                    for (int c = 0; c < 3; ++c) a[c] += f * d[c];
                }
            }
        }
        for (int c = 0; c < 3; ++c) g[3 * k + c] = a[c];
    }
}

/* Rows of K' x where every pair (i, j != i) with |c_i - c_j| <= 2.5 sqrt(A_i)
 * uses the exact panel integral above and every other pair the quadrature
 * rule (the near-singular set of the accelerated product). */
void oracle_kprime_rows_near_exact(int64_t n, int nq, const double *cen, const double *nrm,
                                   const double *area, const double *panels, const double *qp,
                                   const double *qw, const double *x, int64_t nrows,
                                   const int64_t *rows, double *y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        const double tau = 2.5 * sqrt(area[i]);
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            sub3(cen + 3 * i, cen + 3 * j, d);
            double kij;
            if (dot3(d, d) <= tau * tau)
                kij = oracle_panel_dn(cen + 3 * i, nrm + 3 * i, panels + 9 * j);
            else
                kij = kprime_entry(i, j, nq, cen, nrm, qp, qw);
            acc += kij * x[j];
        }
        y[r] = acc;
    }
}

/* Galerkin rows (Sec. 2.1 states the problem in Galerkin form; with a
 * piecewise-constant basis and test functions the row of panel i is the
 * average over T_i of the collocation row): the outer integral over T_i by
 * the quadrature rule at the points y_iq (weights w_q = qw/A_i), the inner
 * integral over T_j exact for the near-singular pairs
 * (|c_i - c_j| <= 2.5 sqrt(A_i)) and by the rule for all others.  j = i
 * adds nothing (the outer and inner points lie in one plane). */
void oracle_kprime_rows_galerkin(int64_t n, int nq, const double *cen, const double *nrm,
                                 const double *area, const double *panels, const double *qp,
                                 const double *qw, const double *x, int64_t nrows,
                                 const int64_t *rows, double *y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        const double tau = 2.5 * sqrt(area[i]);
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double *t = qp + 3 * (i * nq + q);
            const double wq = qw[i * nq + q] / area[i];
            double row = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                sub3(cen + 3 * i, cen + 3 * j, d);
                double kij = 0.0;
                if (dot3(d, d) <= tau * tau)
                    kij = oracle_panel_dn(t, nrm + 3 * i, panels + 9 * j);
                else
                    for (int s2 = 0; s2 < nq; ++s2)
                        kij += qw[j * nq + s2] * dn_green(t, nrm + 3 * i, qp + 3 * (j * nq + s2));
                row += kij * x[j];
            }
            acc += wq * row;
        }
        y[r] = acc;
    }
}

/* The transpose of the Galerkin K': y_j = sum_{i != j} x_i (K'_G)_ij with
 * (K'_G)_ij = sum_q (qw_iq / A_i) k_ij(y_iq), the inner integral k_ij over
 * panel j exact when |c_i - c_j| <= 2.5 sqrt(A_i) and by the rule otherwise
 * (entry for entry the matrix of oracle_kprime_rows_galerkin). */
void oracle_kprime_t_galerkin(int64_t n, int nq, const double *cen, const double *nrm,
                              const double *area, const double *panels, const double *qp,
                              const double *qw, const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (i == j) continue;
            const double tau = 2.5 * sqrt(area[i]);
            double d[3];
            sub3(cen + 3 * i, cen + 3 * j, d);
            const int near = dot3(d, d) <= tau * tau;
            double kij = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double *t = qp + 3 * (i * nq + q);
                double k = 0.0;
                if (near)
                    k = oracle_panel_dn(t, nrm + 3 * i, panels + 9 * j);
                else
                    for (int s2 = 0; s2 < nq; ++s2)
                        k += qw[j * nq + s2] * dn_green(t, nrm + 3 * i, qp + 3 * (j * nq + s2));
                kij += qw[i * nq + q] / area[i] * k;
            }
            acc += kij * x[i];
        }
        y[j] = acc;
    }
}

/* The Galerkin B^T v and its gradient in the charge positions:
 * (B_G)_ik = sum_q (qw_iq / A_i) [-(y_iq - x_k).n_i] / (4 pi |y_iq - x_k|^3),
 * u_k = sum_i v_i (B_G)_ik, h_k = sum_i v_i grad_{x_k} (B_G)_ik with
 * grad_{x_k} of one term [n_i / |d|^3 - 3 (d.n_i) d / |d|^5] / (4 pi),
 * d = y_iq - x_k. */
void oracle_bt_galerkin(int64_t n, int nq, const double *nrm, const double *area, const double *qp,
                        const double *qw, int64_t nc, const double *xq, const double *v, double *u,
                        double *h /* [nc][3] or NULL */)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        double a = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            for (int q = 0; q < nq; ++q) {
                const double *t = qp + 3 * (i * nq + q), *ni = nrm + 3 * i;
                const double f = v[i] * qw[i * nq + q] / area[i];
                a += f * dn_green(t, ni, xq + 3 * k);
                if (h) {
                    double d[3];
                    sub3(t, xq + 3 * k, d);
                    const double r2 = dot3(d, d), r = sqrt(r2), dn = dot3(d, ni);
                    for (int c = 0; c < 3; ++c)
                        g[c] += f * (ni[c] / (r2 * r) - 3.0 * dn * d[c] / (r2 * r2 * r)) / FOUR_PI;
                }
            }
        }
        u[k] = a;
        if (h)
            for (int c = 0; c < 3; ++c) h[3 * k + c] = g[c];
    }
}

/* Galerkin right-hand side field: the normal field of the charges averaged
 * over each panel by the rule, E_i = sum_q (qw_iq / A_i) E_n(y_iq). */
void oracle_bq_galerkin(int64_t n, int nq, const double *nrm, const double *area, const double *qp,
                        const double *qw, int64_t nc, const double *xq, const double *q, double *E)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int s2 = 0; s2 < nq; ++s2) {
            double e = 0.0;
            for (int64_t k = 0; k < nc; ++k)
                e += q[k] * dn_green(qp + 3 * (i * nq + s2), nrm + 3 * i, xq + 3 * k);
            acc += qw[i * nq + s2] / area[i] * e;
        }
        E[i] = acc;
    }
}

/* E = B q: normal field of the point charges at the collocation points. */
void oracle_bq(int64_t n, const double *cen, const double *nrm, int64_t nc,
               const double *xq /*[nc][3]*/, const double *q, double *E)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t k = 0; k < nc; ++k)
            acc += q[k] * dn_green(cen + 3 * i, nrm + 3 * i, xq + 3 * k);
        E[i] = acc;
    }
}

/* u = B^T v: u_k = sum_i v_i B_ik. */
void oracle_bt(int64_t n, const double *cen, const double *nrm, int64_t nc,
               const double *xq, const double *v, double *u)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i)
            acc += v[i] * dn_green(cen + 3 * i, nrm + 3 * i, xq + 3 * k);
        u[k] = acc;
    }
}

/* phi = C s: potential at the charges of the surface charge s (Eq. reac). */
void oracle_c(int64_t n, int nq, const double *qp, const double *qw, int64_t nc,
              const double *xq, const double *s, double *phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double pj = 0.0;
            for (int q = 0; q < nq; ++q)
                pj += qw[j * nq + q] * green(xq + 3 * k, qp + 3 * (j * nq + q));
            acc += s[j] * pj;
        }
        phi[k] = acc;
    }
}

/* v = C^T u: v_j = sum_k u_k C_kj. */
void oracle_ct(int64_t n, int nq, const double *qp, const double *qw, int64_t nc,
               const double *xq, const double *u, double *v)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t k = 0; k < nc; ++k) {
            double pj = 0.0;
            for (int q = 0; q < nq; ++q)
                pj += qw[j * nq + q] * green(xq + 3 * k, qp + 3 * (j * nq + q));
            acc += u[k] * pj;
        }
        v[j] = acc;
    }
}

/* g_k = grad_{x_k} (C s)_k = sum_j s_j A_j sum_q w_q * (-(x_k - y)/(4 pi |x_k - y|^3)). */
void oracle_grad_c(int64_t n, int nq, const double *qp, const double *qw, int64_t nc,
                   const double *xq, const double *s, double *g /*[nc][3]*/)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            for (int q = 0; q < nq; ++q) {
                const double *y = qp + 3 * (j * nq + q);
                double d0 = xq[3 * k] - y[0], d1 = xq[3 * k + 1] - y[1], d2 = xq[3 * k + 2] - y[2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2, r = sqrt(r2);
                double f = -s[j] * qw[j * nq + q] / (FOUR_PI * r2 * r);
                a0 += f * d0; a1 += f * d1; a2 += f * d2;
            }
        }
        g[3 * k] = a0; g[3 * k + 1] = a1; g[3 * k + 2] = a2;
    }
}

/* h_k = sum_i v_i grad_{x_k} B_ik, with B_ik = -(d.n_i)/(4 pi |d|^3), d = c_i - x_k:
 * grad_{x_k} B_ik = [n_i/|d|^3 - 3 (d.n_i) d/|d|^5] / (4 pi). */
void oracle_grad_bt(int64_t n, const double *cen, const double *nrm, int64_t nc,
                    const double *xq, const double *v, double *h /*[nc][3]*/)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nc; ++k) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double *c = cen + 3 * i, *nn = nrm + 3 * i;
            double d0 = c[0] - xq[3 * k], d1 = c[1] - xq[3 * k + 1], d2 = c[2] - xq[3 * k + 2];
            double r2 = d0 * d0 + d1 * d1 + d2 * d2, r = sqrt(r2);
            double ir3 = 1.0 / (r2 * r), ir5 = ir3 / r2;
            double dn = d0 * nn[0] + d1 * nn[1] + d2 * nn[2];
            double f = v[i] / FOUR_PI;
            a0 += f * (nn[0] * ir3 - 3.0 * dn * d0 * ir5);
            a1 += f * (nn[1] * ir3 - 3.0 * dn * d1 * ir5);
            a2 += f * (nn[2] * ir3 - 3.0 * dn * d2 * ir5);
        }
        h[3 * k] = a0; h[3 * k + 1] = a1; h[3 * k + 2] = a2;
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
