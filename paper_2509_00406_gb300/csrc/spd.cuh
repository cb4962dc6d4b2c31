// spd.cuh -- per-term Hessian filtering (Sec. 7.1, after Teran et al. 2005):
// the negative eigenvalues of an element term's local Hessian are set to
// eps >= 0 before assembly.
//
// A term's local Hessian over its NV vertices is H = S^T He S, He its Hessian
// in the NE edge vectors and S = C^T (x) I the constant edge map (terms.cuh).
// With L the Cholesky factor of C^T C (so M = S S^T = (L L^T) (x) I), the rows
// of U = (L^-1 (x) I) S are orthonormal and H = U^T G U for
// G = (L (x) I)^T He (L (x) I): the nonzero spectrum of H is that of G, and
// the rest of H's spectrum is the translations' exact zeros, which clamping
// leaves alone.  An eigenvalue counts as negative below -tau max |lambda|
// (tau 1e-10 in double, 1e-5 in float).  So the filter runs on G (n = NE VD:
// 9 for a hinge, 6 for a 3D triangle, 4 for a 2D one): round-robin Jacobi in
// registers, then
//   He += sum over lambda_i < 0 of (eps - lambda_i) w_i w_i^T,
//   w_i = (L^-1 (x) I)^T v_i,
// which is U^T (clamped G) U pulled back to the edge vectors.  A term with
// no eigenvalue below -tau max |G_ii| / 2 (a shifted Cholesky test; max
// |G_ii| <= max |lambda|) is left as it is without the eigensolve.
#pragma once

#include "ad.cuh"

namespace adm {

template <typename T>
struct SpdFn;
template <>
struct SpdFn<float> {
    ADM_HD static float sqrt_(float v) { return sqrtf(v); }
    // the Jacobi rotation's ratio, reciprocal and 1/sqrt: the fast
    // intrinsics (about 2 ulp) keep c^2 + s^2 = 1 to a few ulp, which the
    // iteration tolerates; 25 % faster on the filtered shell batch than the
    // IEEE forms
#ifdef __CUDA_ARCH__
    ADM_HD static float div_(float a, float b) { return __fdividef(a, b); }
    ADM_HD static float rsqrt_(float v) { return rsqrtf(v); }
#else
    ADM_HD static float div_(float a, float b) { return a / b; }
    ADM_HD static float rsqrt_(float v) { return 1.0f / sqrtf(v); }
#endif
    ADM_HD static float eps() { return 1.1920929e-7f; }
    ADM_HD static float tau() { return 1e-5f; }
    static constexpr int kMaxSweeps = 8;
};
template <>
struct SpdFn<double> {
    ADM_HD static double sqrt_(double v) { return ::sqrt(v); }
    ADM_HD static double div_(double a, double b) { return a / b; }
    ADM_HD static double rsqrt_(double v) { return 1.0 / ::sqrt(v); }
    ADM_HD static double eps() { return 2.220446049250313e-16; }
    ADM_HD static double tau() { return 1e-10; }
    static constexpr int kMaxSweeps = 12;
};

// packed upper index of a symmetric n x n matrix, either order
ADM_HD constexpr int sym_ix(int i, int j) { return i <= j ? hix(i, j) : hix(j, i); }

// Cholesky factor of C^T C of an edge map E (NE <= 3) and its inverse, both
// lower triangular, row-major NE x NE
template <class E, typename T>
ADM_HD void edge_metric_factor(T (&L)[E::NE][E::NE], T (&Li)[E::NE][E::NE])
{
    constexpr int NE = E::NE;
#pragma unroll
    for (int i = 0; i < NE; ++i)
#pragma unroll
        for (int j = 0; j < NE; ++j) {
            L[i][j] = T(0);
            Li[i][j] = T(0);
        }
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        T d = T(0);
#pragma unroll
        for (int a = 0; a < E::NV; ++a) d += T(E::C(a, j) * E::C(a, j));
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        L[j][j] = SpdFn<T>::sqrt_(d);
#pragma unroll
        for (int i = j + 1; i < NE; ++i) {
            T m = T(0);
#pragma unroll
            for (int a = 0; a < E::NV; ++a) m += T(E::C(a, i) * E::C(a, j));
#pragma unroll
            for (int k = 0; k < j; ++k) m -= L[i][k] * L[j][k];
            L[i][j] = m / L[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) {  // forward substitution, column j of L^-1
        Li[j][j] = T(1) / L[j][j];
#pragma unroll
        for (int i = j + 1; i < NE; ++i) {
            T s = T(0);
#pragma unroll
            for (int k = j; k < i; ++k) s += L[i][k] * Li[k][j];
            Li[i][j] = -s / L[i][i];
        }
    }
}

// Round-robin pairing of n indices (n padded to even m): round r pairs
// (i, j) with i + j = 2r mod (m - 1) for i, j < m - 1, and the index i with
// 2i = 2r mod (m - 1) with m - 1.  Pairs of one round are disjoint, so their
// rotations commute; pairs with an index >= n (the pad) are skipped.
ADM_HD constexpr int rr_partner(int m, int r, int i)
{
    if (i == m - 1) {
        for (int k = 0; k < m - 1; ++k)
            if ((2 * k) % (m - 1) == (2 * r) % (m - 1)) return k;
        return -1;
    }
    if ((2 * i) % (m - 1) == (2 * r) % (m - 1)) return m - 1;
    return ((2 * r - i) % (m - 1) + (m - 1)) % (m - 1);
}
// the pairs (p < q) of every round, as a table built at compile time
template <int M>
struct RoundRobin {
    int p[M - 1][M / 2] = {}, q[M - 1][M / 2] = {};
    ADM_HD constexpr RoundRobin()
    {
        for (int r = 0; r < M - 1; ++r) {
            int cnt = 0;
            for (int i = 0; i < M; ++i) {
                const int j = rr_partner(M, r, i);
                if (i < j) {
                    p[r][cnt] = i;
                    q[r][cnt] = j;
                    ++cnt;
                }
            }
        }
    }
};

// Symmetric eigen-decomposition A = V diag(A_ii) V^T by Jacobi rotations in
// round-robin order (A packed upper, overwritten by its diagonalised form;
// V n x n, columns the eigenvectors).  Every round first takes the rotation
// angles of its disjoint pairs from the current A, then applies them, so
// the angle computations of a round are independent of one another.  Stops
// when the off-diagonal mass is below machine precision relative to the
// whole matrix, or after kMaxSweeps.
template <int N, typename T>
ADM_HD void jacobi_eig(T (&A)[N * (N + 1) / 2], T (&V)[N][N])
{
    constexpr int M = N + (N & 1), R = M - 1, P = M / 2;
    constexpr RoundRobin<M> rr;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) V[i][j] = i == j ? T(1) : T(0);
#pragma unroll 1
    for (int sweep = 0; sweep < SpdFn<T>::kMaxSweeps; ++sweep) {
        T off = T(0), all = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) {
                const T a2 = A[hix(i, j)] * A[hix(i, j)];
                all += i == j ? a2 : T(2) * a2;
                if (i != j) off += T(2) * a2;
            }
        const T e = SpdFn<T>::eps();
        if (!(off > e * e * all)) break;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T cs[P], sn[P], tn[P], ap[P];
            // angles of the round's pairs, from the current A
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int p = rr.p[r][k], q = rr.q[r][k];
                cs[k] = T(1);
                sn[k] = T(0);
                tn[k] = T(0);
                ap[k] = T(0);
                if (q >= N) continue;
                const T apq = A[hix(p, q)];
                ap[k] = apq;
                if (apq == T(0)) continue;
                const T theta = SpdFn<T>::div_(A[hix(q, q)] - A[hix(p, p)], T(2) * apq);
                const T at = theta < T(0) ? -theta : theta;
                T t = SpdFn<T>::div_(T(1), at + SpdFn<T>::sqrt_(theta * theta + T(1)));
                if (theta < T(0)) t = -t;
                const T c = SpdFn<T>::rsqrt_(t * t + T(1));
                cs[k] = c;
                sn[k] = t * c;
                tn[k] = t;
            }
            // the rotations, one pair after another
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int p = rr.p[r][k], q = rr.q[r][k];
                if (q >= N) continue;
                const T c = cs[k], s = sn[k], t = tn[k], apq = ap[k];
                A[hix(p, p)] -= t * apq;
                A[hix(q, q)] += t * apq;
                A[hix(p, q)] = T(0);
#pragma unroll
                for (int kk = 0; kk < N; ++kk) {
                    if (kk == p || kk == q) continue;
                    const T akp = A[sym_ix(kk, p)], akq = A[sym_ix(kk, q)];
                    A[sym_ix(kk, p)] = c * akp - s * akq;
                    A[sym_ix(kk, q)] = s * akp + c * akq;
                }
#pragma unroll
                for (int kk = 0; kk < N; ++kk) {
                    const T vkp = V[kk][p], vkq = V[kk][q];
                    V[kk][p] = c * vkp - s * vkq;
                    V[kk][q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

// Whether a symmetric A (packed upper) has no eigenvalue below -s: a
// Cholesky factorisation of A + s I that meets no non-positive pivot.
template <int N, typename T>
ADM_HD bool shifted_cholesky_ok(const T (&A)[N * (N + 1) / 2], T s)
{
    T Lf[N][N];      // lower factor
    bool ok = true;  // no early exit, so that the loops unroll completely
#pragma unroll
    for (int j = 0; j < N; ++j) {
        T d = A[hix(j, j)] + s;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k < j) d -= Lf[j][k] * Lf[j][k];
        ok = ok && d > T(0);
        const T ljj = SpdFn<T>::sqrt_(d > T(0) ? d : T(1)), inv = T(1) / ljj;
        Lf[j][j] = ljj;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i <= j) continue;
            T m = A[hix(j, i)];
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k < j) m -= Lf[i][k] * Lf[j][k];
            Lf[i][j] = m * inv;
        }
    }
    return ok;
}

// Filter the edge-vector Hessian He (packed upper, n = NE VD) in place.
template <class E, int VD, typename T>
ADM_HD void project_edges(T (&He)[E::NE * VD * (E::NE * VD + 1) / 2], T eps)
{
    constexpr int NE = E::NE, N = NE * VD, NP = N * (N + 1) / 2;
    T L[NE][NE], Li[NE][NE];
    edge_metric_factor<E>(L, Li);
    // G = (L (x) I)^T He (L (x) I): G_(p,r),(q,s) = sum L[p'][p] L[q'][q] He_(p',r),(q',s)
    T G[NP];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i <= j; ++i) {
            const int p = i / VD, r = i % VD, q = j / VD, s = j % VD;
            T acc = -T(0);
#pragma unroll
            for (int pp = p; pp < NE; ++pp)
#pragma unroll
                for (int qq = q; qq < NE; ++qq) acc += L[pp][p] * L[qq][q] * He[sym_ix(pp * VD + r, qq * VD + s)];
            G[hix(i, j)] = acc;
        }
    // nothing to clamp if no eigenvalue lies below -s, s = tau max |G_ii| / 2
    // (max |G_ii| <= max |lambda|): then the filter leaves He as it is
    {
        T dmax = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) dmax = fmax(dmax, fabs(G[hix(m, m)]));
        if (shifted_cholesky_ok<N>(G, T(0.5) * SpdFn<T>::tau() * dmax)) return;
    }
    T Vv[N][N];
    jacobi_eig<N>(G, Vv);
    // negative means below -tau max |lambda|: a term's structural zeros
    // (every hinge has one besides its translations) come out of round-off
    // on either side of zero and are left alone
    T lmax = T(0);
#pragma unroll
    for (int m = 0; m < N; ++m) lmax = fmax(lmax, fabs(G[hix(m, m)]));
#pragma unroll
    for (int m = 0; m < N; ++m) {
        const T lam = G[hix(m, m)];
        if (!(lam < -SpdFn<T>::tau() * lmax)) continue;
        // w = (L^-1 (x) I)^T v_m: w_(p,r) = sum_p' Li[p'][p] v_(p',r)
        T w[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int p = i / VD, r = i % VD;
            T acc = -T(0);
#pragma unroll
            for (int pp = p; pp < NE; ++pp) acc += Li[pp][p] * Vv[pp * VD + r][m];
            w[i] = acc;
        }
        const T d = eps - lam;
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) He[hix(i, j)] += d * w[i] * w[j];
    }
}

}  // namespace adm
