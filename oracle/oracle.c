/*
 * oracle.c -- plain, slow, FP64 CPU oracle for per-element forward-mode
 * differentiation and gradient / Hessian / Jacobian assembly on triangle
 * meshes (Mahmoud, Goel, Ragan-Kelley, Solomon, "Locality-Aware Automatic
 * Differentiation on the GPU for Mesh-Based Computations").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * bench's CPU-baseline leg load this file.  It shares no code, header, table
 * or helper with the CUDA library; the two meet only on the seeded inputs.
 *
 * What it computes is the plain definition of the method (Sec. 4.1):
 *     F(x) = sum_j f_j(S_j x)                      (Eq. 1)
 *     g    = sum_j S_j^T grad f_j                  (Eq. 2)
 *     H    = sum_j S_j^T Hess f_j S_j              (Eq. 2)
 *     J    = sum_j P_j^T J_j S_j                   (Eq. 3)
 * with the local derivatives taken by two independent routes:
 *   route 0 -- forward-mode AD with a dense hyper-dual number carrying the
 *              value, the k-gradient and the full k x k Hessian (the
 *              "ActiveT" of Sec. 5.1 / Sec. 6.2, with k = stencil x VarDim);
 *   route 1 -- hand-derived closed forms (gradients of every scalar term,
 *              the full Hessian of the StVK membrane).
 * Assembly adds every local block into a CSR/BSR pattern enumerated by brute
 * force from the element stencils (Sec. 6.1): collect all (row, col) vertex
 * pairs, sort, deduplicate.
 *
 * Energies (the paper's own, and the synthetic workloads defined in terms of
 * them):
 *   1  symmetric Dirichlet, area_t (|J|_F^2 + |J^-1|_F^2)      (Sec. 7.2)
 *   2  StVK membrane  t A (mu |E|^2 + lambda/2 tr(E)^2)       (synthetic shell)
 *   3  dihedral hinge bending  k_b (A/3) (theta - theta')^2 h^2 (Sec. 7.7)
 *   4  shell = 2 + 3
 *   5  Neo-Hookean membrane on the three invariants of C       (Sec. 7.7)
 *   7  surface area 1/2 |(x_j - x_i) x (x_k - x_i)|            (Sec. 7.6)
 *  16  ARAP-style residual sqrt(A) vec(J - R(J)), 4 per face  (Sec. 4.1 Eq. 3)
 * The reading taken for each ambiguous passage is stated at the function
 * that implements it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* energy identifiers (the numbering of the library's public interface) */
enum {
    E_SYMDIR = 1, E_STVK = 2, E_HINGE = 3, E_SHELL = 4, E_NH = 5, E_MLP = 6,
    E_AREA = 7, E_ARAP = 16
};

/* ======================================================================
 * 1. Dense hyper-dual numbers: value, gradient g[k], Hessian h[k][k].
 *    Rules are the first- and second-order chain rules; every elementary
 *    function supplies f, f', f'' (or the five partials of a bivariate f).
 * ====================================================================== */
#define KMAX 12

typedef struct {
    int k;
    double v;
    double g[KMAX];
    double h[KMAX][KMAX];
} hd;

/* Scalar floating-point operations of the dense rules below, counted as
 * written (value, k gradient entries, k x k Hessian entries; the scalar
 * derivatives f, f', f'' callers pass in are not counted).  A measurement
 * of what dense forward mode costs per element; it changes no result. */
static int64_t g_hd_flops;
#define HD_COUNT(n) (g_hd_flops += (int64_t)(n))

static hd hd_const(int k, double c)
{
    hd r;
    memset(&r, 0, sizeof r);
    r.k = k;
    r.v = c;
    return r;
}

static hd hd_var(int k, double value, int i)
{
    hd r = hd_const(k, value);
    r.g[i] = 1.0;
    return r;
}

static hd hd_add(hd a, hd b)
{
    HD_COUNT(1 + a.k + a.k * a.k);
    hd r = a;
    r.v = a.v + b.v;
    for (int i = 0; i < a.k; ++i) {
        r.g[i] = a.g[i] + b.g[i];
        for (int j = 0; j < a.k; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j];
    }
    return r;
}

static hd hd_scale(hd a, double s)
{
    HD_COUNT(1 + a.k + a.k * a.k);
    hd r = a;
    r.v = a.v * s;
    for (int i = 0; i < a.k; ++i) {
        r.g[i] = a.g[i] * s;
        for (int j = 0; j < a.k; ++j) r.h[i][j] = a.h[i][j] * s;
    }
    return r;
}

static hd hd_sub(hd a, hd b) { return hd_add(a, hd_scale(b, -1.0)); }

static hd hd_addc(hd a, double c)
{
    HD_COUNT(1);
    a.v += c;
    return a;
}

/* product rule: (ab)'' = a'' b + a b'' + a' b'^T + b' a'^T */
static hd hd_mul(hd a, hd b)
{
    HD_COUNT(1 + 3 * a.k + 7 * a.k * a.k);  /* per Hessian entry: 4 products, 3 sums */
    hd r = hd_const(a.k, a.v * b.v);
    for (int i = 0; i < a.k; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
    for (int i = 0; i < a.k; ++i)
        for (int j = 0; j < a.k; ++j)
            r.h[i][j] = a.h[i][j] * b.v + a.v * b.h[i][j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
    return r;
}

/* univariate chain rule: r = f(a), r' = f1 a', r'' = f1 a'' + f2 a' a'^T */
static hd hd_chain1(hd a, double f, double f1, double f2)
{
    HD_COUNT(a.k + 4 * a.k * a.k);
    hd r = hd_const(a.k, f);
    for (int i = 0; i < a.k; ++i) r.g[i] = f1 * a.g[i];
    for (int i = 0; i < a.k; ++i)
        for (int j = 0; j < a.k; ++j) r.h[i][j] = f1 * a.h[i][j] + f2 * a.g[i] * a.g[j];
    return r;
}

/* bivariate chain rule for r = f(a, b) */
static hd hd_chain2(hd a, hd b, double f, double fa, double fb, double faa, double fab,
                    double fbb)
{
    HD_COUNT(3 * a.k + 14 * a.k * a.k);
    hd r = hd_const(a.k, f);
    for (int i = 0; i < a.k; ++i) r.g[i] = fa * a.g[i] + fb * b.g[i];
    for (int i = 0; i < a.k; ++i)
        for (int j = 0; j < a.k; ++j)
            r.h[i][j] = fa * a.h[i][j] + fb * b.h[i][j] + faa * a.g[i] * a.g[j] +
                        fab * (a.g[i] * b.g[j] + b.g[i] * a.g[j]) + fbb * b.g[i] * b.g[j];
    return r;
}

static hd hd_recip(hd a) { return hd_chain1(a, 1.0 / a.v, -1.0 / (a.v * a.v), 2.0 / (a.v * a.v * a.v)); }
static hd hd_div(hd a, hd b) { return hd_mul(a, hd_recip(b)); }
static hd hd_sqrt(hd a)
{
    double s = sqrt(a.v);
    return hd_chain1(a, s, 0.5 / s, -0.25 / (s * a.v));
}
static hd hd_log(hd a) { return hd_chain1(a, log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v)); }
static hd hd_sin(hd a) { return hd_chain1(a, sin(a.v), cos(a.v), -sin(a.v)); }
static hd hd_cos(hd a) { return hd_chain1(a, cos(a.v), -sin(a.v), -cos(a.v)); }
static hd hd_sq(hd a) { return hd_mul(a, a); }

/* theta = atan2(y, x): d/dy = x/r2, d/dx = -y/r2, d2/dy2 = -2xy/r2^2,
 * d2/dx2 = 2xy/r2^2, d2/dxdy = (y^2 - x^2)/r2^2 */
static hd hd_atan2(hd y, hd x)
{
    double r2 = x.v * x.v + y.v * y.v;
    double r4 = r2 * r2;
    return hd_chain2(y, x, atan2(y.v, x.v), x.v / r2, -y.v / r2, -2.0 * x.v * y.v / r4,
                     (y.v * y.v - x.v * x.v) / r4, 2.0 * x.v * y.v / r4);
}

/* exported elementary-rule probes (used by the tests to pin the rules) */
void orc_hd_probe(int op, const double *in, int n_in, double *out)
{
    /* op: 0 recip, 1 sqrt, 2 log, 3 sin, 4 cos, 5 atan2(in0,in1), 6 mul, 7 div
     * inputs become variables 0..n_in-1 (k = n_in); out = value, gradient
     * (n_in), Hessian row-major (n_in^2) */
    int k = n_in;
    hd a = hd_var(k, in[0], 0);
    hd b = n_in > 1 ? hd_var(k, in[1], 1) : hd_const(k, 0.0);
    hd r;
    switch (op) {
    case 0: r = hd_recip(a); break;
    case 1: r = hd_sqrt(a); break;
    case 2: r = hd_log(a); break;
    case 3: r = hd_sin(a); break;
    case 4: r = hd_cos(a); break;
    case 5: r = hd_atan2(a, b); break;
    case 6: r = hd_mul(a, b); break;
    default: r = hd_div(a, b); break;
    }
    out[0] = r.v;
    for (int i = 0; i < k; ++i) out[1 + i] = r.g[i];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) out[1 + k + i * k + j] = r.h[i][j];
}

/* ======================================================================
 * 2. Material constants (readings: plane-stress Lame parameters).
 * ====================================================================== */
typedef struct {
    double E, nu, t, kb, h;
} params_t;

static params_t params_from(int energy, const double *p, int np)
{
    params_t q;
    q.E = 1.0e5;
    q.nu = 0.3;
    q.t = 1.0e-3;
    q.h = 1.0;
    q.kb = -1.0;
    if (energy == E_HINGE) {
        if (np > 0) q.kb = p[0];
        if (np > 1) q.h = p[1];
    } else {
        if (np > 0) q.E = p[0];
        if (np > 1) q.nu = p[1];
        if (np > 2) q.t = p[2];
        if (np > 3) q.kb = p[3];
        if (np > 4) q.h = p[4];
    }
    /* reading: bending stiffness of a thin plate, k_b = E t^3 / (12 (1 - nu^2)) */
    if (q.kb < 0.0) q.kb = q.E * q.t * q.t * q.t / (12.0 * (1.0 - q.nu * q.nu));
    return q;
}

static double lame_mu(params_t q) { return q.E / (2.0 * (1.0 + q.nu)); }
static double lame_lambda(params_t q) { return q.E * q.nu / (1.0 - q.nu * q.nu); }

/* ======================================================================
 * 3. Rest-state data.
 *    Local frame of a rest triangle (a, b, c): e1 = unit(b - a),
 *    e2 = unit(n x e1) with n the counter-clockwise normal; Dm is the 2x2
 *    matrix of the rest edges [b - a, c - a] in that frame (Sec. 7.2).
 * ====================================================================== */
static void cross3(const double *a, const double *b, double *r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

void orc_tri_rest(int64_t nT, const double *Vrest, const int32_t *F, double *Dinv, double *area)
{
    for (int64_t t = 0; t < nT; ++t) {
        const double *a = Vrest + 3 * (int64_t)F[3 * t + 0];
        const double *b = Vrest + 3 * (int64_t)F[3 * t + 1];
        const double *c = Vrest + 3 * (int64_t)F[3 * t + 2];
        double u[3], w[3], n[3], e1[3], e2[3];
        for (int d = 0; d < 3; ++d) {
            u[d] = b[d] - a[d];
            w[d] = c[d] - a[d];
        }
        cross3(u, w, n);
        double nn = sqrt(dot3(n, n));
        double lu = sqrt(dot3(u, u));
        for (int d = 0; d < 3; ++d) e1[d] = u[d] / lu;
        double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
        cross3(nh, e1, e2);
        double Dm[2][2] = {{dot3(u, e1), dot3(w, e1)}, {dot3(u, e2), dot3(w, e2)}};
        double det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
        Dinv[4 * t + 0] = Dm[1][1] / det;
        Dinv[4 * t + 1] = -Dm[0][1] / det;
        Dinv[4 * t + 2] = -Dm[1][0] / det;
        Dinv[4 * t + 3] = Dm[0][0] / det;
        area[t] = 0.5 * nn;
    }
}

/* ======================================================================
 * 4. Local energies over hyper-dual numbers (route 0).
 *    Local DOF order: vertex-major, x[a * vdim + d].
 * ====================================================================== */

/* J = [b - a, c - a] Dm^-1 for a 2D map (uv) or the 3x2 deformation gradient */
static void deformation_gradient(const hd *x, int dim, const double *Dinv, hd Fm[3][2])
{
    for (int r = 0; r < dim; ++r) {
        hd ds0 = hd_sub(x[1 * dim + r], x[0 * dim + r]);
        hd ds1 = hd_sub(x[2 * dim + r], x[0 * dim + r]);
        for (int c = 0; c < 2; ++c)
            Fm[r][c] = hd_add(hd_scale(ds0, Dinv[0 * 2 + c]), hd_scale(ds1, Dinv[1 * 2 + c]));
    }
}

/* symmetric Dirichlet (Sec. 7.2): area_t (|J|_F^2 + |J^-1|_F^2), area_t the
 * rest area (reading), J^-1 formed explicitly.  det J <= 0 is a domain error. */
static int symdir_hd(const hd *x, const double *Dinv, double area, hd *out)
{
    hd J[3][2];
    deformation_gradient(x, 2, Dinv, J);
    hd det = hd_sub(hd_mul(J[0][0], J[1][1]), hd_mul(J[0][1], J[1][0]));
    if (!(det.v > 0.0)) return 1;
    hd idet = hd_recip(det);
    hd Ji[2][2];
    Ji[0][0] = hd_mul(J[1][1], idet);
    Ji[0][1] = hd_scale(hd_mul(J[0][1], idet), -1.0);
    Ji[1][0] = hd_scale(hd_mul(J[1][0], idet), -1.0);
    Ji[1][1] = hd_mul(J[0][0], idet);
    hd s = hd_const(x[0].k, 0.0);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) s = hd_add(s, hd_add(hd_sq(J[r][c]), hd_sq(Ji[r][c])));
    *out = hd_scale(s, area);
    return 0;
}

/* Green strain E = 1/2 (F^T F - I) of a 3x2 deformation gradient */
static void green_strain(hd Fm[3][2], hd E[2][2])
{
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            hd s = hd_const(Fm[0][0].k, 0.0);
            for (int i = 0; i < 3; ++i) s = hd_add(s, hd_mul(Fm[i][a], Fm[i][b]));
            E[a][b] = hd_scale(hd_addc(s, a == b ? -1.0 : 0.0), 0.5);
        }
}

/* StVK membrane (synthetic shell workload): t A (mu |E|_F^2 + lambda/2 tr(E)^2) */
static int stvk_hd(const hd *x, const double *Dinv, double area, params_t q, hd *out)
{
    hd Fm[3][2], E[2][2];
    deformation_gradient(x, 3, Dinv, Fm);
    green_strain(Fm, E);
    double mu = lame_mu(q), la = lame_lambda(q);
    hd n2 = hd_const(x[0].k, 0.0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) n2 = hd_add(n2, hd_sq(E[a][b]));
    hd tr = hd_add(E[0][0], E[1][1]);
    hd psi = hd_add(hd_scale(n2, mu), hd_scale(hd_sq(tr), 0.5 * la));
    *out = hd_scale(psi, q.t * area);
    return 0;
}

/* Neo-Hookean membrane on the invariants of the right Cauchy-Green tensor.
 * Reading: C3 = diag(F^T F, 1) (unit thickness stretch), I1 = tr C3,
 * I2 = 1/2 (tr(C3)^2 - tr(C3^2)), I3 = det C3, J = sqrt(I3),
 * psi = mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2, f = t A psi. */
static int nh_invariants_hd(const hd *x, const double *Dinv, hd I[3])
{
    hd Fm[3][2];
    deformation_gradient(x, 3, Dinv, Fm);
    int k = x[0].k;
    hd C3[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C3[a][b] = hd_const(k, (a == 2 && b == 2) ? 1.0 : 0.0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            hd s = hd_const(k, 0.0);
            for (int i = 0; i < 3; ++i) s = hd_add(s, hd_mul(Fm[i][a], Fm[i][b]));
            C3[a][b] = s;
        }
    hd tr = hd_add(hd_add(C3[0][0], C3[1][1]), C3[2][2]);
    hd trsq = hd_const(k, 0.0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) trsq = hd_add(trsq, hd_mul(C3[a][b], C3[b][a]));
    I[0] = tr;
    I[1] = hd_scale(hd_sub(hd_sq(tr), trsq), 0.5);
    /* cofactor expansion along the first row */
    hd m0 = hd_sub(hd_mul(C3[1][1], C3[2][2]), hd_mul(C3[1][2], C3[2][1]));
    hd m1 = hd_sub(hd_mul(C3[1][0], C3[2][2]), hd_mul(C3[1][2], C3[2][0]));
    hd m2 = hd_sub(hd_mul(C3[1][0], C3[2][1]), hd_mul(C3[1][1], C3[2][0]));
    I[2] = hd_add(hd_sub(hd_mul(C3[0][0], m0), hd_mul(C3[0][1], m1)), hd_mul(C3[0][2], m2));
    return I[2].v > 0.0 ? 0 : 1;
}

static int nh_hd(const hd *x, const double *Dinv, double area, params_t q, hd *out)
{
    hd I[3];
    if (nh_invariants_hd(x, Dinv, I)) return 1;
    double mu = lame_mu(q), la = lame_lambda(q);
    hd lnJ = hd_scale(hd_log(I[2]), 0.5);
    hd psi = hd_add(hd_sub(hd_scale(hd_addc(I[0], -3.0), 0.5 * mu), hd_scale(lnJ, mu)),
                    hd_scale(hd_sq(lnJ), 0.5 * la));
    *out = hd_scale(psi, q.t * area);
    return 0;
}

/* signed dihedral angle of hinge (x0, x1, xa, xb), face A = (x0, x1, xa),
 * face B = (x1, x0, xb):
 *   nA = (x1 - x0) x (xa - x0),  nB = (x0 - x1) x (xb - x1),
 *   theta = atan2((nA x nB) . e_hat, nA . nB),  e_hat = unit(x1 - x0). */
static int hinge_theta_hd(const hd *x, hd *theta)
{
    int k = x[0].k;
    hd e[3], ua[3], nb0[3], vb[3], nA[3], nB[3], c[3];
    for (int d = 0; d < 3; ++d) {
        e[d] = hd_sub(x[3 + d], x[0 + d]);
        ua[d] = hd_sub(x[6 + d], x[0 + d]);
        nb0[d] = hd_sub(x[0 + d], x[3 + d]);
        vb[d] = hd_sub(x[9 + d], x[3 + d]);
    }
#define HCROSS(a, b, r)                                                               \
    do {                                                                              \
        r[0] = hd_sub(hd_mul(a[1], b[2]), hd_mul(a[2], b[1]));                        \
        r[1] = hd_sub(hd_mul(a[2], b[0]), hd_mul(a[0], b[2]));                        \
        r[2] = hd_sub(hd_mul(a[0], b[1]), hd_mul(a[1], b[0]));                        \
    } while (0)
    HCROSS(e, ua, nA);
    HCROSS(nb0, vb, nB);
    HCROSS(nA, nB, c);
#undef HCROSS
    hd el = hd_const(k, 0.0), cosv = hd_const(k, 0.0), sinv = hd_const(k, 0.0);
    for (int d = 0; d < 3; ++d) {
        el = hd_add(el, hd_sq(e[d]));
        cosv = hd_add(cosv, hd_mul(nA[d], nB[d]));
    }
    el = hd_sqrt(el);
    for (int d = 0; d < 3; ++d) sinv = hd_add(sinv, hd_mul(c[d], hd_div(e[d], el)));
    if (cosv.v == 0.0 && sinv.v == 0.0) return 1;
    *theta = hd_atan2(sinv, cosv);
    return 0;
}

/* hinge bending (Sec. 7.7): k_b (A/3) (theta - theta')^2 h^2, A = the
 * average rest area of the two faces (the paper's "pre-computed area") */
static int hinge_hd(const hd *x, double thetabar, double abar, params_t q, hd *out)
{
    hd th;
    if (hinge_theta_hd(x, &th)) return 1;
    double w = q.kb * abar / 3.0 * q.h * q.h;
    *out = hd_scale(hd_sq(hd_addc(th, -thetabar)), w);
    return 0;
}

/* surface area 1/2 |(x1 - x0) x (x2 - x0)| (Sec. 7.6) */
static int area_hd(const hd *x, hd *out)
{
    int k = x[0].k;
    hd u[3], w[3];
    for (int d = 0; d < 3; ++d) {
        u[d] = hd_sub(x[3 + d], x[d]);
        w[d] = hd_sub(x[6 + d], x[d]);
    }
    hd n0 = hd_sub(hd_mul(u[1], w[2]), hd_mul(u[2], w[1]));
    hd n1 = hd_sub(hd_mul(u[2], w[0]), hd_mul(u[0], w[2]));
    hd n2 = hd_sub(hd_mul(u[0], w[1]), hd_mul(u[1], w[0]));
    hd s = hd_add(hd_add(hd_sq(n0), hd_sq(n1)), hd_sq(n2));
    if (!(s.v > 0.0)) return 1;
    (void)k;
    *out = hd_scale(hd_sqrt(s), 0.5);
    return 0;
}

/* ARAP-style residual (Sec. 4.1 Eq. 3 vector-valued term): with J the 2x2
 * Jacobian of the UV map, R(J) the closest rotation = rotation by
 * phi = atan2(J10 - J01, J00 + J11), r = sqrt(A) vec_rowmajor(J - R(J)). */
static int arap_hd(const hd *x, const double *Dinv, double area, hd r[4])
{
    hd J[3][2];
    deformation_gradient(x, 2, Dinv, J);
    hd p = hd_add(J[0][0], J[1][1]);
    hd s = hd_sub(J[1][0], J[0][1]);
    if (p.v == 0.0 && s.v == 0.0) return 1;
    hd phi = hd_atan2(s, p);
    hd c = hd_cos(phi), sn = hd_sin(phi);
    double sa = sqrt(area);
    r[0] = hd_scale(hd_sub(J[0][0], c), sa);
    r[1] = hd_scale(hd_add(J[0][1], sn), sa);
    r[2] = hd_scale(hd_sub(J[1][0], sn), sa);
    r[3] = hd_scale(hd_sub(J[1][1], c), sa);
    return 0;
}

/* ======================================================================
 * 5. Closed-form local derivatives (route 1).
 * ====================================================================== */

/* rows D_v (v = 0,1,2) with F = sum_v x_v D_v:  D_0 = -(Dinv_0 + Dinv_1) */
static void vertex_rows(const double *Dinv, double D[3][2])
{
    for (int c = 0; c < 2; ++c) {
        D[1][c] = Dinv[0 * 2 + c];
        D[2][c] = Dinv[1 * 2 + c];
        D[0][c] = -D[1][c] - D[2][c];
    }
}

static void defgrad_plain(const double *x, int dim, const double *Dinv, double Fm[3][2])
{
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < 2; ++c)
            Fm[r][c] = (x[1 * dim + r] - x[r]) * Dinv[c] + (x[2 * dim + r] - x[r]) * Dinv[2 + c];
}

/* symmetric Dirichlet: df/dJ = A (2 J - 2 J^-T J^-1 J^-T) */
static int symdir_cf(const double *x, const double *Dinv, double area, double *f, double *g)
{
    double J[3][2], D[3][2];
    defgrad_plain(x, 2, Dinv, J);
    vertex_rows(Dinv, D);
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(det > 0.0)) return 1;
    double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    double n = 0.0;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) n += J[r][c] * J[r][c] + Ji[r][c] * Ji[r][c];
    *f = area * n;
    double JiT[2][2] = {{Ji[0][0], Ji[1][0]}, {Ji[0][1], Ji[1][1]}};
    double M[2][2], P[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) M[r][c] = JiT[r][0] * Ji[0][c] + JiT[r][1] * Ji[1][c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c)
            P[r][c] = area * (2.0 * J[r][c] - 2.0 * (M[r][0] * JiT[0][c] + M[r][1] * JiT[1][c]));
    for (int v = 0; v < 3; ++v)
        for (int r = 0; r < 2; ++r) g[v * 2 + r] = P[r][0] * D[v][0] + P[r][1] * D[v][1];
    return 0;
}

/* StVK: P = F S, S = 2 mu E + lambda tr(E) I;
 * dP_ic/dF_jd = delta_ij S_dc + mu (delta_cd (F F^T)_ij + F_id F_jc) + lambda F_ic F_jd */
static int stvk_cf(const double *x, const double *Dinv, double area, params_t q, double *f,
                   double *g, double *H /* 9x9 row-major or NULL */)
{
    double Fm[3][2], D[3][2], E[2][2], S[2][2], P[3][2];
    defgrad_plain(x, 3, Dinv, Fm);
    vertex_rows(Dinv, D);
    double mu = lame_mu(q), la = lame_lambda(q), s = q.t * area;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double c = 0.0;
            for (int i = 0; i < 3; ++i) c += Fm[i][a] * Fm[i][b];
            E[a][b] = 0.5 * (c - (a == b ? 1.0 : 0.0));
        }
    double tr = E[0][0] + E[1][1];
    double n2 = E[0][0] * E[0][0] + E[0][1] * E[0][1] + E[1][0] * E[1][0] + E[1][1] * E[1][1];
    *f = s * (mu * n2 + 0.5 * la * tr * tr);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) S[a][b] = 2.0 * mu * E[a][b] + (a == b ? la * tr : 0.0);
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 2; ++c) P[i][c] = Fm[i][0] * S[0][c] + Fm[i][1] * S[1][c];
    for (int v = 0; v < 3; ++v)
        for (int i = 0; i < 3; ++i) g[3 * v + i] = s * (P[i][0] * D[v][0] + P[i][1] * D[v][1]);
    if (!H) return 0;
    double FFt[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) FFt[i][j] = Fm[i][0] * Fm[j][0] + Fm[i][1] * Fm[j][1];
    for (int v = 0; v < 3; ++v)
        for (int i = 0; i < 3; ++i)
            for (int w = 0; w < 3; ++w)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int c = 0; c < 2; ++c)
                        for (int d = 0; d < 2; ++d) {
                            double A = (i == j ? S[d][c] : 0.0) +
                                       mu * ((c == d ? FFt[i][j] : 0.0) + Fm[i][d] * Fm[j][c]) +
                                       la * Fm[i][c] * Fm[j][d];
                            acc += D[v][c] * D[w][d] * A;
                        }
                    H[(3 * v + i) * 9 + 3 * w + j] = s * acc;
                }
    return 0;
}

/* Neo-Hookean membrane: P = mu F + (lambda ln J - mu) F C^-1, C = F^T F */
static int nh_cf(const double *x, const double *Dinv, double area, params_t q, double *f,
                 double *g)
{
    double Fm[3][2], D[3][2], C[2][2];
    defgrad_plain(x, 3, Dinv, Fm);
    vertex_rows(Dinv, D);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) C[a][b] = Fm[0][a] * Fm[0][b] + Fm[1][a] * Fm[1][b] + Fm[2][a] * Fm[2][b];
    double detC = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    if (!(detC > 0.0)) return 1;
    double mu = lame_mu(q), la = lame_lambda(q), s = q.t * area;
    double lnJ = 0.5 * log(detC);
    *f = s * (0.5 * mu * (C[0][0] + C[1][1] + 1.0 - 3.0) - mu * lnJ + 0.5 * la * lnJ * lnJ);
    double Ci[2][2] = {{C[1][1] / detC, -C[0][1] / detC}, {-C[1][0] / detC, C[0][0] / detC}};
    double P[3][2];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 2; ++c)
            P[i][c] = mu * Fm[i][c] + (la * lnJ - mu) * (Fm[i][0] * Ci[0][c] + Fm[i][1] * Ci[1][c]);
    for (int v = 0; v < 3; ++v)
        for (int i = 0; i < 3; ++i) g[3 * v + i] = s * (P[i][0] * D[v][0] + P[i][1] * D[v][1]);
    return 0;
}

/* hinge: dtheta/dxa = -|e| nA/|nA|^2, dtheta/dxb = -|e| nB/|nB|^2,
 * dtheta/dx0 = -(1 - sa) dtheta/dxa - (1 - sb) dtheta/dxb,
 * dtheta/dx1 = -sa dtheta/dxa - sb dtheta/dxb,
 * with s_w = (x_w - x0).e/|e|^2 the position of the wing's foot on the edge
 * (discrete-shells bending gradient, Grinspun et al. 2003; Tamstorf 2013).
 * The Hessian of theta is the derivative of these four vectors, taken by the
 * product rule with
 *   d nA = de x u + e x du,  d nB = dm x v + m x dv   (m = x0 - x1, v = xb - x1),
 *   d |e| = e.de / |e|,      d s_w = (dw.e + w.de)/|e|^2 - 2 s_w e.de/|e|^2,
 * and E = w (theta - thetabar)^2 gives
 *   H = 2 w (grad theta grad theta^T + (theta - thetabar) Hess theta). */

/* [a]x, the matrix of b -> a x b */
static void skew3(const double *a, double S[3][3])
{
    S[0][0] = 0.0;   S[0][1] = -a[2]; S[0][2] = a[1];
    S[1][0] = a[2];  S[1][1] = 0.0;   S[1][2] = -a[0];
    S[2][0] = -a[1]; S[2][1] = a[0];  S[2][2] = 0.0;
}

/* derivative of the wing gradient g = -el n / |n|^2 with respect to one
 * vertex, given that vertex's dn (3x3) and d el (3) */
static void dwing(const double *n, double n2, double el, double N[3][3], const double L[3], double out[3][3])
{
    double nN[3];
    for (int j = 0; j < 3; ++j) nN[j] = n[0] * N[0][j] + n[1] * N[1][j] + n[2] * N[2][j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            out[i][j] = -n[i] * L[j] / n2 - el * N[i][j] / n2 + 2.0 * el * n[i] * nN[j] / (n2 * n2);
}

static int hinge_cf(const double *x, double thetabar, double abar, params_t q, double *f,
                    double *g, double *H /* 12x12 row-major or NULL */)
{
    const double *x0 = x, *x1 = x + 3, *xa = x + 6, *xb = x + 9;
    double e[3], u[3], m[3], v[3], nA[3], nB[3], c[3];
    for (int d = 0; d < 3; ++d) {
        e[d] = x1[d] - x0[d];
        u[d] = xa[d] - x0[d];
        m[d] = x0[d] - x1[d];
        v[d] = xb[d] - x1[d];
    }
    cross3(e, u, nA);
    cross3(m, v, nB);
    cross3(nA, nB, c);
    double el = sqrt(dot3(e, e));
    double cs = dot3(nA, nB), sn = dot3(c, e) / el;
    if (cs == 0.0 && sn == 0.0) return 1;
    double th = atan2(sn, cs);
    double w = q.kb * abar / 3.0 * q.h * q.h;
    *f = w * (th - thetabar) * (th - thetabar);
    double dA = dot3(nA, nA), dB = dot3(nB, nB), ee = dot3(e, e);
    double ga[3], gb[3];
    for (int d = 0; d < 3; ++d) {
        ga[d] = -el * nA[d] / dA;
        gb[d] = -el * nB[d] / dB;
    }
    double wb[3];
    for (int d = 0; d < 3; ++d) wb[d] = xb[d] - x0[d];
    double sa = dot3(u, e) / ee, sb = dot3(wb, e) / ee;
    double fp = 2.0 * w * (th - thetabar);
    double gt[12];  /* grad theta, vertex order (x0, x1, xa, xb) */
    for (int d = 0; d < 3; ++d) {
        gt[0 + d] = -(1.0 - sa) * ga[d] - (1.0 - sb) * gb[d];
        gt[3 + d] = -sa * ga[d] - sb * gb[d];
        gt[6 + d] = ga[d];
        gt[9 + d] = gb[d];
    }
    for (int i = 0; i < 12; ++i) g[i] = fp * gt[i];
    if (!H) return 0;
    double Su[3][3], Se[3][3], Sv[3][3], Sm[3][3];
    skew3(u, Su);
    skew3(e, Se);
    skew3(v, Sv);
    skew3(m, Sm);
    double eh[3] = {e[0] / el, e[1] / el, e[2] / el};
    double ue = dot3(u, e), we = dot3(wb, e);
    double Ht[12][12];
    for (int k = 0; k < 4; ++k) {
        double NA[3][3], NB[3][3], L[3] = {0.0, 0.0, 0.0}, dsa[3] = {0.0, 0.0, 0.0}, dsb[3] = {0.0, 0.0, 0.0};
        double de_sign = k == 0 ? -1.0 : (k == 1 ? 1.0 : 0.0);  /* de = de_sign dx_k */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                switch (k) {
                case 0: NA[i][j] = Su[i][j] - Se[i][j]; NB[i][j] = -Sv[i][j]; break;
                case 1: NA[i][j] = -Su[i][j]; NB[i][j] = Sv[i][j] - Sm[i][j]; break;
                case 2: NA[i][j] = Se[i][j]; NB[i][j] = 0.0; break;
                default: NA[i][j] = 0.0; NB[i][j] = Sm[i][j]; break;
                }
            }
        for (int j = 0; j < 3; ++j) {
            L[j] = de_sign * eh[j];
            /* d(u.e) and d(wb.e) for this vertex */
            double due = 0.0, dwe = 0.0;
            if (k == 0) { due = -(e[j] + u[j]); dwe = -(e[j] + wb[j]); }
            if (k == 1) { due = u[j]; dwe = wb[j]; }
            if (k == 2) due = e[j];
            if (k == 3) dwe = e[j];
            double dee = 2.0 * de_sign * e[j];
            dsa[j] = due / ee - ue * dee / (ee * ee);
            dsb[j] = dwe / ee - we * dee / (ee * ee);
        }
        double Da[3][3], Db[3][3];
        dwing(nA, dA, el, NA, L, Da);
        dwing(nB, dB, el, NB, L, Db);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                int col = 3 * k + j;
                Ht[0 + i][col] = -(1.0 - sa) * Da[i][j] + ga[i] * dsa[j] - (1.0 - sb) * Db[i][j] + gb[i] * dsb[j];
                Ht[3 + i][col] = -sa * Da[i][j] - ga[i] * dsa[j] - sb * Db[i][j] - gb[i] * dsb[j];
                Ht[6 + i][col] = Da[i][j];
                Ht[9 + i][col] = Db[i][j];
            }
    }
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) H[i * 12 + j] = 2.0 * w * (gt[i] * gt[j] + (th - thetabar) * Ht[i][j]);
    return 0;
}

/* area gradient printed in Sec. 7.6: dA/dx_i = 1/2 (x_j - x_k) x n (unit n),
 * cyclic in (i, j, k) */
static int area_cf(const double *x, double *f, double *g)
{
    double u[3], w[3], n[3];
    for (int d = 0; d < 3; ++d) {
        u[d] = x[3 + d] - x[d];
        w[d] = x[6 + d] - x[d];
    }
    cross3(u, w, n);
    double nn = sqrt(dot3(n, n));
    if (!(nn > 0.0)) return 1;
    *f = 0.5 * nn;
    for (int d = 0; d < 3; ++d) n[d] /= nn;
    for (int i = 0; i < 3; ++i) {
        const double *xj = x + 3 * ((i + 1) % 3), *xk = x + 3 * ((i + 2) % 3);
        double dj[3] = {xj[0] - xk[0], xj[1] - xk[1], xj[2] - xk[2]}, r[3];
        cross3(dj, n, r);
        for (int d = 0; d < 3; ++d) g[3 * i + d] = 0.5 * r[d];
    }
    return 0;
}

/* ======================================================================
 * 6. Connectivity: hinges in canonical order, brute-force block patterns.
 * ====================================================================== */
typedef struct {
    int64_t key; /* lo * nV + hi */
    int32_t from, to, opp;
} halfedge_t;

static int cmp_he(const void *a, const void *b)
{
    const halfedge_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->from != y->from) return x->from < y->from ? -1 : 1;
    return 0;
}

/* Hinges = interior edges with exactly two incident faces.  Canonical form:
 * (e0, e1, a, b) with e0 < e1, face A containing the directed edge e0->e1
 * with third vertex a, face B containing e1->e0 with third vertex b; sorted
 * by (e0, e1).  Returns the number of hinges, or -1 when an edge has more
 * than two faces or two faces traverse it in the same direction.
 * H may be NULL (count only). */
int64_t orc_hinges(int64_t nV, int64_t nT, const int32_t *F, int32_t *H)
{
    halfedge_t *he = malloc(sizeof(halfedge_t) * 3 * (size_t)(nT > 0 ? nT : 1));
    for (int64_t t = 0; t < nT; ++t)
        for (int c = 0; c < 3; ++c) {
            int32_t a = F[3 * t + c], b = F[3 * t + (c + 1) % 3], o = F[3 * t + (c + 2) % 3];
            int32_t lo = a < b ? a : b, hi = a < b ? b : a;
            halfedge_t h = {(int64_t)lo * nV + hi, a, b, o};
            he[3 * t + c] = h;
        }
    qsort(he, 3 * (size_t)nT, sizeof(halfedge_t), cmp_he);
    int64_t nh = 0;
    for (int64_t i = 0; i < 3 * nT;) {
        int64_t j = i;
        while (j < 3 * nT && he[j].key == he[i].key) ++j;
        if (j - i > 2) {
            free(he);
            return -1;
        }
        if (j - i == 2) {
            if (he[i].from == he[i + 1].from) {
                free(he);
                return -1;
            }
            /* after sorting by 'from', he[i] starts at the smaller id */
            const halfedge_t *A = &he[i], *B = &he[i + 1];
            if (H) {
                H[4 * nh + 0] = A->from;
                H[4 * nh + 1] = A->to;
                H[4 * nh + 2] = A->opp;
                H[4 * nh + 3] = B->opp;
            }
            ++nh;
        }
        i = j;
    }
    free(he);
    return nh;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* block pattern {(i, j): i, j in a common stencil} as CSR over vertices.
 * Stencils: every triangle (3 vertices) and, when nH > 0, every hinge
 * (4 vertices).  Returns nnzb; row_ptr (nV+1) and col may be NULL. */
int64_t orc_pattern(int64_t nV, int64_t nT, const int32_t *F, int64_t nH, const int32_t *H,
                    int32_t *row_ptr, int32_t *col)
{
    /* reading: the pattern is {(i, i)} plus the stencil pairs, so a vertex
       no element touches still has its (zero) diagonal block */
    int64_t cap = nV + 9 * nT + 16 * nH;
    int64_t *keys = malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    int64_t n = 0;
    for (int64_t v = 0; v < nV; ++v) keys[n++] = v * nV + v;
    for (int64_t t = 0; t < nT; ++t)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) keys[n++] = (int64_t)F[3 * t + a] * nV + F[3 * t + b];
    for (int64_t h = 0; h < nH; ++h)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) keys[n++] = (int64_t)H[4 * h + a] * nV + H[4 * h + b];
    qsort(keys, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];
    if (row_ptr) {
        for (int64_t v = 0; v <= nV; ++v) row_ptr[v] = 0;
        for (int64_t i = 0; i < m; ++i) row_ptr[keys[i] / nV + 1]++;
        for (int64_t v = 0; v < nV; ++v) row_ptr[v + 1] += row_ptr[v];
    }
    if (col)
        for (int64_t i = 0; i < m; ++i) col[i] = (int32_t)(keys[i] % nV);
    free(keys);
    return m;
}

/* ======================================================================
 * 7. Element evaluation and assembly.
 * ====================================================================== */
typedef struct {
    int64_t nV;
    int vdim;
    const int32_t *row_ptr, *col;
    const unsigned char *row_mask;
    double *grad, *vals;
    double energy;
    int64_t n_err;
} asm_t;

static int64_t find_block(const asm_t *A, int32_t i, int32_t j)
{
    int64_t lo = A->row_ptr[i], hi = A->row_ptr[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (A->col[mid] == j) return mid;
        if (A->col[mid] < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* add f, g (nv*vdim), H (row-major) of one element with vertices vid[nv] */
static int scatter(asm_t *A, int nv, const int32_t *vid, double f, const double *g, const double *H)
{
    int vd = A->vdim, k = nv * vd;
    A->energy += f;
    for (int a = 0; a < nv; ++a) {
        if (A->row_mask && !A->row_mask[vid[a]]) continue;
        if (A->grad)
            for (int d = 0; d < vd; ++d) A->grad[(int64_t)vid[a] * vd + d] += g[a * vd + d];
        if (!A->vals || !H) continue;
        for (int b = 0; b < nv; ++b) {
            int64_t blk = find_block(A, vid[a], vid[b]);
            if (blk < 0) return -1;
            for (int r = 0; r < vd; ++r)
                for (int s = 0; s < vd; ++s)
                    A->vals[blk * vd * vd + r * vd + s] += H[(a * vd + r) * k + b * vd + s];
        }
    }
    return 0;
}

static void hd_unpack(const hd *r, int k, double *f, double *g, double *H)
{
    *f = r->v;
    for (int i = 0; i < k; ++i) {
        g[i] = r->g[i];
        for (int j = 0; j < k; ++j) H[i * k + j] = r->h[i][j];
    }
}

static int touches(const asm_t *A, int nv, const int32_t *vid)
{
    if (!A->row_mask) return 1;
    for (int a = 0; a < nv; ++a)
        if (A->row_mask[vid[a]]) return 1;
    return 0;
}

/* learned membrane energy (section 9): network parameters set by orc_mlp_set */
static double g_mlp_theta[4481], g_mlp_norm[8];
static int mlp_hd(const hd *x, const double *Dinv, double area, params_t q, hd *out);

/* local derivatives of one triangle term; route 0 = hyper-dual, 1 = closed form */
static int tri_local(int energy, int route, const double *xl, int vd, const double *Dinv,
                     double area, params_t q, double *f, double *g, double *H)
{
    int k = 3 * vd;
    if (route == 1) {
        int err;
        switch (energy) {
        case E_SYMDIR: err = symdir_cf(xl, Dinv, area, f, g); break;
        case E_STVK: err = stvk_cf(xl, Dinv, area, q, f, g, H); break;
        case E_NH: err = nh_cf(xl, Dinv, area, q, f, g); break;
        case E_AREA: err = area_cf(xl, f, g); break;
        default: return -2;
        }
        if (energy != E_STVK) memset(H, 0, sizeof(double) * k * k);
        return err;
    }
    hd xs[KMAX], r;
    for (int i = 0; i < k; ++i) xs[i] = hd_var(k, xl[i], i);
    int err;
    switch (energy) {
    case E_SYMDIR: err = symdir_hd(xs, Dinv, area, &r); break;
    case E_STVK: err = stvk_hd(xs, Dinv, area, q, &r); break;
    case E_NH: err = nh_hd(xs, Dinv, area, q, &r); break;
    case E_AREA: err = area_hd(xs, &r); break;
    case E_MLP: err = mlp_hd(xs, Dinv, area, q, &r); break;
    default: return -2;
    }
    if (err) return err;
    hd_unpack(&r, k, f, g, H);
    return 0;
}

static int hinge_local(int route, const double *xl, double thetabar, double abar, params_t q,
                       double *f, double *g, double *H)
{
    if (route == 1) return hinge_cf(xl, thetabar, abar, q, f, g, H);
    hd xs[12], r;
    for (int i = 0; i < 12; ++i) xs[i] = hd_var(12, xl[i], i);
    if (hinge_hd(xs, thetabar, abar, q, &r)) return 1;
    hd_unpack(&r, 12, f, g, H);
    return 0;
}

static int tri_term(int energy)
{
    return energy == E_SYMDIR || energy == E_STVK || energy == E_SHELL || energy == E_NH ||
           energy == E_AREA || energy == E_MLP;
}

/* Evaluate energy, gradient and BSR Hessian of one energy over a mesh.
 *   x          : nV*vdim current DOFs
 *   tri_Dinv   : 4 per triangle, tri_area : rest areas (orc_tri_rest)
 *   H, thetabar, abar : hinges (orc_hinges) and their rest angle / mean area
 *   row_ptr/col: BSR pattern (orc_pattern); vals nnzb*vdim*vdim
 *   row_mask   : NULL, or only rows with mask != 0 are assembled (elements
 *                touching none of them are skipped; energy then covers the
 *                evaluated elements only)
 *   elem_energy: NULL, or per-element energies (triangles then hinges)
 * Outputs are accumulated (the caller zeroes them).  Returns the number of
 * elements with a domain error (they contribute nothing), or < 0 on a
 * pattern/argument error. */
int64_t orc_assemble(int energy, const double *p, int np, int route, int64_t nV, int vdim,
                     int64_t nT, const int32_t *F, const double *tri_Dinv, const double *tri_area,
                     int64_t nH, const int32_t *H, const double *thetabar, const double *abar,
                     const double *x, const int32_t *row_ptr, const int32_t *col,
                     const unsigned char *row_mask, double *energy_out, double *grad,
                     double *vals, double *elem_energy)
{
    params_t q = params_from(energy, p, np);
    asm_t A = {nV, vdim, row_ptr, col, row_mask, grad, vals, 0.0, 0};
    int tri_energy = energy == E_SHELL ? E_STVK : energy;
    double g[KMAX], Hl[KMAX * KMAX], xl[KMAX], f;
    if (tri_term(energy)) {
        int k = 3 * vdim;
        for (int64_t t = 0; t < nT; ++t) {
            const int32_t *vid = F + 3 * t;
            if (!touches(&A, 3, vid)) continue;
            for (int a = 0; a < 3; ++a)
                for (int d = 0; d < vdim; ++d) xl[a * vdim + d] = x[(int64_t)vid[a] * vdim + d];
            int err = tri_local(tri_energy, route, xl, vdim, tri_Dinv + 4 * t, tri_area[t], q, &f, g, Hl);
            if (err < 0) return err;
            if (err) {
                A.n_err++;
                if (elem_energy) elem_energy[t] = 0.0;
                continue;
            }
            (void)k;
            if (elem_energy) elem_energy[t] = f;
            if (scatter(&A, 3, vid, f, g, Hl)) return -3;
        }
    }
    if (energy == E_HINGE || energy == E_SHELL) {
        if (vdim != 3) return -4;
        for (int64_t h = 0; h < nH; ++h) {
            const int32_t *vid = H + 4 * h;
            if (!touches(&A, 4, vid)) continue;
            for (int a = 0; a < 4; ++a)
                for (int d = 0; d < 3; ++d) xl[a * 3 + d] = x[(int64_t)vid[a] * 3 + d];
            int err = hinge_local(route, xl, thetabar[h], abar[h], q, &f, g, Hl);
            int64_t slot = (energy == E_SHELL ? nT : 0) + h;
            if (err) {
                A.n_err++;
                if (elem_energy) elem_energy[slot] = 0.0;
                continue;
            }
            if (elem_energy) elem_energy[slot] = f;
            if (scatter(&A, 4, vid, f, g, Hl)) return -3;
        }
    }
    *energy_out += A.energy;
    return A.n_err;
}

/* rest dihedral angle and mean rest area of every hinge */
void orc_hinge_rest(int64_t nH, const int32_t *H, const double *Vrest, double *thetabar,
                    double *abar)
{
    for (int64_t h = 0; h < nH; ++h) {
        double xl[12];
        for (int a = 0; a < 4; ++a)
            for (int d = 0; d < 3; ++d) xl[3 * a + d] = Vrest[3 * (int64_t)H[4 * h + a] + d];
        hd xs[12], th;
        for (int i = 0; i < 12; ++i) xs[i] = hd_const(0, xl[i]);
        thetabar[h] = hinge_theta_hd(xs, &th) ? 0.0 : th.v;
        double u[3], w[3], n[3], s = 0.0;
        for (int d = 0; d < 3; ++d) {
            u[d] = xl[3 + d] - xl[d];
            w[d] = xl[6 + d] - xl[d];
        }
        cross3(u, w, n);
        s += 0.5 * sqrt(dot3(n, n));
        for (int d = 0; d < 3; ++d) {
            u[d] = xl[d] - xl[3 + d];
            w[d] = xl[9 + d] - xl[3 + d];
        }
        cross3(u, w, n);
        s += 0.5 * sqrt(dot3(n, n));
        abar[h] = 0.5 * s;
    }
}

/* single-element entry points (for pins and finite differences) */
/* the dense-rule operation count since the last reset (reset != 0 clears it) */
int64_t orc_hd_flops(int reset)
{
    const int64_t v = g_hd_flops;
    if (reset) g_hd_flops = 0;
    return v;
}

int orc_local(int energy, int route, const double *p, int np, const double *xl, int vdim,
              const double *Dinv, double area, double thetabar, double abar, double *f,
              double *g, double *H)
{
    params_t q = params_from(energy, p, np);
    if (energy == E_HINGE) return hinge_local(route, xl, thetabar, abar, q, f, g, H);
    return tri_local(energy, route, xl, vdim, Dinv, area, q, f, g, H);
}

/* ======================================================================
 * 8. Vector-valued term: ARAP-style residual and its CSR Jacobian (Eq. 3).
 *    Row 4t + r belongs to triangle t (disjoint row blocks, Sec. 6.1); the
 *    six columns of a row are the (vertex, coordinate) pairs sorted by
 *    vertex id then coordinate.
 * ====================================================================== */
int64_t orc_arap_jacobian(int64_t nT, const int32_t *F, const double *tri_Dinv,
                          const double *tri_area, const double *uv, double *r,
                          int32_t *jrow_ptr, int32_t *jcol, double *jval)
{
    int64_t nerr = 0;
    for (int64_t t = 0; t < nT; ++t) {
        const int32_t *vid = F + 3 * t;
        hd xs[6], res[4];
        for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 2; ++d) xs[2 * a + d] = hd_var(6, uv[(int64_t)vid[a] * 2 + d], 2 * a + d);
        int err = arap_hd(xs, tri_Dinv + 4 * t, tri_area[t], res);
        if (err) nerr++;
        /* column order: local vertices sorted by global id */
        int ord[3] = {0, 1, 2};
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j)
                if (vid[ord[j]] < vid[ord[i]]) {
                    int tmp = ord[i];
                    ord[i] = ord[j];
                    ord[j] = tmp;
                }
        for (int rr = 0; rr < 4; ++rr) {
            int64_t row = 4 * t + rr;
            r[row] = err ? 0.0 : res[rr].v;
            jrow_ptr[row] = (int32_t)(6 * row);
            int c = 0;
            for (int oi = 0; oi < 3; ++oi)
                for (int d = 0; d < 2; ++d) {
                    int a = ord[oi];
                    jcol[6 * row + c] = vid[a] * 2 + d;
                    jval[6 * row + c] = err ? 0.0 : res[rr].g[2 * a + d];
                    ++c;
                }
        }
    }
    jrow_ptr[4 * nT] = (int32_t)(24 * nT);
    return nerr;
}

/* ======================================================================
 * 9. Learned membrane energy (per-triangle MLP surrogate of the
 *    Neo-Hookean density on the three invariants of C3 = diag(F^T F, 1)).
 *    Parameters theta (4481): W1 (64x3, row j = hidden unit), b1 (64),
 *    W2 (64x64, row i = output unit, column j = input unit), b2 (64),
 *    w3 (64), b3.  norm (8): mean and scale of I1..I3, mean and scale of psi.
 *    Network on standardised inputs u_k = (I_k - m_k)/s_k:
 *      z1 = W1 u + b1, a1 = silu(z1), z2 = W2 a1 + b2, a2 = silu(z2),
 *      y = w3 . a2 + b3,  psi = s_psi y + m_psi,  silu(z) = z / (1 + e^-z).
 * ====================================================================== */
#define MLP_H 64
#define MLP_NP (MLP_H * 3 + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

static void silu3(double z, double *s, double *s1, double *s2)
{
    double sg = 1.0 / (1.0 + exp(-z));
    *s = z * sg;
    *s1 = sg * (1.0 + z * (1.0 - sg));
    *s2 = sg * (1.0 - sg) * (2.0 + z * (1.0 - 2.0 * sg));
}

static hd hd_silu(hd a)
{
    double s, s1, s2;
    silu3(a.v, &s, &s1, &s2);
    return hd_chain1(a, s, s1, s2);
}

/* invariants (I1, I2, I3) of C3 = diag(F^T F, 1) for n samples F (3x2 row-major) */
void orc_invariants_from_F(int64_t n, const double *F, double *I)
{
    for (int64_t s = 0; s < n; ++s) {
        const double *f = F + 6 * s;
        double C[3][3] = {{0}};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int i = 0; i < 3; ++i) C[a][b] += f[2 * i + a] * f[2 * i + b];
        C[2][2] = 1.0;
        double tr = C[0][0] + C[1][1] + C[2][2], trsq = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) trsq += C[a][b] * C[b][a];
        double det = C[0][0] * (C[1][1] * C[2][2] - C[1][2] * C[2][1]) -
                     C[0][1] * (C[1][0] * C[2][2] - C[1][2] * C[2][0]) +
                     C[0][2] * (C[1][0] * C[2][1] - C[1][1] * C[2][0]);
        I[3 * s + 0] = tr;
        I[3 * s + 1] = 0.5 * (tr * tr - trsq);
        I[3 * s + 2] = det;
    }
}

/* Neo-Hookean density psi(I) = mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2,
 * J = sqrt(I3), and its gradient in I, by hyper-duals over (I1, I2, I3) */
void orc_nh_targets(int64_t n, const double *I, const double *p, int np, double *psi, double *dpsi)
{
    params_t q = params_from(E_NH, p, np);
    double mu = lame_mu(q), la = lame_lambda(q);
    for (int64_t s = 0; s < n; ++s) {
        hd i1 = hd_var(3, I[3 * s + 0], 0), i3 = hd_var(3, I[3 * s + 2], 2);
        hd lnJ = hd_scale(hd_log(i3), 0.5);
        hd r = hd_add(hd_sub(hd_scale(hd_addc(i1, -3.0), 0.5 * mu), hd_scale(lnJ, mu)),
                      hd_scale(hd_sq(lnJ), 0.5 * la));
        psi[s] = r.v;
        for (int k = 0; k < 3; ++k) dpsi[3 * s + k] = r.g[k];
    }
}

/* network on hyper-duals over the raw invariants: psi, dpsi/dI (3), and the
 * upper Hessian (I1I1, I1I2, I2I2, I1I3, I2I3, I3I3) per sample */
void orc_mlp_eval(const double *th, const double *norm, int64_t n, const double *I, double *out)
{
    const double *W1 = th, *b1 = W1 + MLP_H * 3, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
                 *w3 = b2 + MLP_H, *b3 = w3 + MLP_H;
    for (int64_t s = 0; s < n; ++s) {
        hd u[3], a1[MLP_H];
        for (int k = 0; k < 3; ++k)
            u[k] = hd_scale(hd_addc(hd_var(3, I[3 * s + k], k), -norm[k]), 1.0 / norm[3 + k]);
        for (int j = 0; j < MLP_H; ++j) {
            hd z = hd_const(3, b1[j]);
            for (int k = 0; k < 3; ++k) z = hd_add(z, hd_scale(u[k], W1[3 * j + k]));
            a1[j] = hd_silu(z);
        }
        hd y = hd_const(3, b3[0]);
        for (int i = 0; i < MLP_H; ++i) {
            hd z = hd_const(3, b2[i]);
            for (int j = 0; j < MLP_H; ++j) z = hd_add(z, hd_scale(a1[j], W2[MLP_H * i + j]));
            y = hd_add(y, hd_scale(hd_silu(z), w3[i]));
        }
        y = hd_addc(hd_scale(y, norm[7]), norm[6]);
        double *o = out + 10 * s;
        o[0] = y.v;
        for (int k = 0; k < 3; ++k) o[1 + k] = y.g[k];
        o[4] = y.h[0][0];
        o[5] = y.h[0][1];
        o[6] = y.h[1][1];
        o[7] = y.h[0][2];
        o[8] = y.h[1][2];
        o[9] = y.h[2][2];
    }
}

/* Sobolev loss on standardised quantities,
 *   L = mean_s (y_s - ty_s)^2 + beta mean_s sum_k (dy/du_k - tg_{s,k})^2,
 * ty = (target psi - m_psi) / s_psi, tg_k = (target dpsi/dI_k) s_k / s_psi, and its gradient
 * with respect to theta by reverse mode through the value-and-tangent
 * forward pass (written out by hand; pinned by finite differences in the
 * tests).  grad may be NULL. */
double orc_mlp_loss(const double *th, const double *norm, int64_t n, const double *I, const double *psi_t,
                    const double *g_t, double beta, double *grad)
{
    const double *W1 = th, *b1 = W1 + MLP_H * 3, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
                 *w3 = b2 + MLP_H, *b3 = w3 + MLP_H;
    double *gW1 = grad, *gb1 = grad ? gW1 + MLP_H * 3 : NULL, *gW2 = grad ? gb1 + MLP_H : NULL,
           *gb2 = grad ? gW2 + MLP_H * MLP_H : NULL, *gw3 = grad ? gb2 + MLP_H : NULL,
           *gb3 = grad ? gw3 + MLP_H : NULL;
    if (grad) memset(grad, 0, sizeof(double) * MLP_NP);
    double L = 0.0;
    double u[3], z1[MLP_H], a1[MLP_H], s1p[MLP_H], s1pp[MLP_H], t1[3][MLP_H];
    double z2[MLP_H], a2[MLP_H], s2p[MLP_H], s2pp[MLP_H], u2[3][MLP_H], t2[3][MLP_H];
    for (int64_t s = 0; s < n; ++s) {
        for (int k = 0; k < 3; ++k) u[k] = (I[3 * s + k] - norm[k]) / norm[3 + k];
        for (int j = 0; j < MLP_H; ++j) {
            z1[j] = b1[j];
            for (int k = 0; k < 3; ++k) z1[j] += W1[3 * j + k] * u[k];
            silu3(z1[j], &a1[j], &s1p[j], &s1pp[j]);
            for (int k = 0; k < 3; ++k) t1[k][j] = s1p[j] * W1[3 * j + k];
        }
        double y = b3[0], dy[3] = {0, 0, 0};
        for (int i = 0; i < MLP_H; ++i) {
            z2[i] = b2[i];
            for (int k = 0; k < 3; ++k) u2[k][i] = 0.0;
            for (int j = 0; j < MLP_H; ++j) {
                z2[i] += W2[MLP_H * i + j] * a1[j];
                for (int k = 0; k < 3; ++k) u2[k][i] += W2[MLP_H * i + j] * t1[k][j];
            }
            silu3(z2[i], &a2[i], &s2p[i], &s2pp[i]);
            y += w3[i] * a2[i];
            for (int k = 0; k < 3; ++k) {
                t2[k][i] = s2p[i] * u2[k][i];
                dy[k] += w3[i] * t2[k][i];
            }
        }
        double ty = (psi_t[s] - norm[6]) / norm[7];
        double r0 = y - ty, rk[3];
        L += r0 * r0;
        for (int k = 0; k < 3; ++k) {
            rk[k] = dy[k] - g_t[3 * s + k] * norm[3 + k] / norm[7];
            L += beta * rk[k] * rk[k];
        }
        if (!grad) continue;
        double dY = 2.0 * r0 / n, dDY[3];
        for (int k = 0; k < 3; ++k) dDY[k] = 2.0 * beta * rk[k] / n;
        gb3[0] += dY;
        double dz2[MLP_H], du2[3][MLP_H];
        for (int i = 0; i < MLP_H; ++i) {
            gw3[i] += dY * a2[i];
            for (int k = 0; k < 3; ++k) gw3[i] += dDY[k] * t2[k][i];
            /* t2_k = s'(z2) u2_k, a2 = s(z2) */
            dz2[i] = dY * w3[i] * s2p[i];
            for (int k = 0; k < 3; ++k) {
                dz2[i] += dDY[k] * w3[i] * s2pp[i] * u2[k][i];
                du2[k][i] = dDY[k] * w3[i] * s2p[i];
            }
            gb2[i] += dz2[i];
        }
        for (int i = 0; i < MLP_H; ++i)
            for (int j = 0; j < MLP_H; ++j) {
                double g = dz2[i] * a1[j];
                for (int k = 0; k < 3; ++k) g += du2[k][i] * t1[k][j];
                gW2[MLP_H * i + j] += g;
            }
        for (int j = 0; j < MLP_H; ++j) {
            double da1 = 0.0, dt1[3] = {0, 0, 0};
            for (int i = 0; i < MLP_H; ++i) {
                da1 += W2[MLP_H * i + j] * dz2[i];
                for (int k = 0; k < 3; ++k) dt1[k] += W2[MLP_H * i + j] * du2[k][i];
            }
            /* t1_k = s'(z1) W1[j][k], a1 = s(z1), z1 = W1 u + b1 */
            double dz1 = da1 * s1p[j];
            for (int k = 0; k < 3; ++k) {
                dz1 += dt1[k] * s1pp[j] * W1[3 * j + k];
                gW1[3 * j + k] += dt1[k] * s1p[j];
            }
            gb1[j] += dz1;
            for (int k = 0; k < 3; ++k) gW1[3 * j + k] += dz1 * u[k];
        }
    }
    return L / n;
}

/* learned membrane as a mesh energy: f = t A psi(I(C)), the network run on
 * hyper-dual numbers over the element's 9 DOFs (route 0) */
void orc_mlp_set(const double *theta, const double *norm)
{
    memcpy(g_mlp_theta, theta, sizeof g_mlp_theta);
    memcpy(g_mlp_norm, norm, sizeof g_mlp_norm);
}

static int mlp_hd(const hd *x, const double *Dinv, double area, params_t q, hd *out)
{
    hd I[3];
    if (nh_invariants_hd(x, Dinv, I)) return 1;
    const double *th = g_mlp_theta, *norm = g_mlp_norm;
    const double *W1 = th, *b1 = W1 + MLP_H * 3, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
                 *w3 = b2 + MLP_H, *b3 = w3 + MLP_H;
    int k = x[0].k;
    hd u[3], a1[MLP_H];
    for (int c = 0; c < 3; ++c) u[c] = hd_scale(hd_addc(I[c], -norm[c]), 1.0 / norm[3 + c]);
    for (int j = 0; j < MLP_H; ++j) {
        hd z = hd_const(k, b1[j]);
        for (int c = 0; c < 3; ++c) z = hd_add(z, hd_scale(u[c], W1[3 * j + c]));
        a1[j] = hd_silu(z);
    }
    hd y = hd_const(k, b3[0]);
    for (int i = 0; i < MLP_H; ++i) {
        hd z = hd_const(k, b2[i]);
        for (int j = 0; j < MLP_H; ++j) z = hd_add(z, hd_scale(a1[j], W2[MLP_H * i + j]));
        y = hd_add(y, hd_scale(hd_silu(z), w3[i]));
    }
    *out = hd_scale(hd_addc(hd_scale(y, norm[7]), norm[6]), q.t * area);
    return 0;
}
