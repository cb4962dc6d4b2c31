// terms.cuh -- per-element energy terms written on the forward-mode engine.
//
// Every term returns the element's value f, gradient g[K] and packed upper
// Hessian H[K(K+1)/2] over its local DOFs (vertex-major, k = a * VD + d), the
// dense local derivatives of Sec. 5.1 that Eq. 2 assembles.  A term is split
// as f = psi(q(x)): q are a few polynomial invariants of the element's edge
// vectors (sparse SHDs over the K DOFs), psi a density over them (a dense SHD
// over M <= 5 seeds); compose() applies the second-order chain rule.
//
// Triangle membranes use q = (C11, C22, C12), C = F^T F the right
// Cauchy-Green tensor of the 3x2 deformation gradient F = [x1-x0, x2-x0] Dm^-1
// (Dm the rest edges in the triangle's local frame).  The symmetric Dirichlet
// term uses the same q with the 2x2 UV Jacobian J (|J|^2 = tr C,
// det(J)^2 = det C).  The hinge uses q = (e.e, e.u, e.v, u.v, det[e,u,v]) with
// e = x1 - x0, u = xa - x0, v = xb - x1, for which the signed dihedral angle
// is theta = atan2(-|e| det, (e.v)(e.u) - (e.e)(u.v)).
#pragma once

#include "ad.cuh"
#include "spd.cuh"

namespace adm {

// ------------------------------------------------------------ densities --
// StVK: t A (mu |E|^2 + lambda/2 tr(E)^2), E = (C - I)/2
template <typename T>
struct PsiStVK {
    T mu, lam, s;  // s = thickness * rest area
    template <class A, class B, class C>
    ADM_HD auto operator()(const A &c11, const B &c22, const C &c12) const
    {
        auto e11 = (c11 - T(1)) * T(0.5);
        auto e22 = (c22 - T(1)) * T(0.5);
        auto tr = e11 + e22;
        auto n2 = sq(e11) + sq(e22) + sq(c12) * T(0.5);  // 2 (c12 / 2)^2
        return (n2 * mu + sq(tr) * (T(0.5) * lam)) * s;
    }
};

// Neo-Hookean on the invariants of C3 = diag(C, 1):
// I1 = tr C + 1, I3 = det C, psi = mu/2 (I1 - 3) - mu ln J + lambda/2 (ln J)^2
template <typename T>
struct PsiNH {
    T mu, lam, s;
    template <class A, class B, class C>
    ADM_HD auto operator()(const A &c11, const B &c22, const C &c12) const
    {
        auto i3 = c11 * c22 - sq(c12);
        auto L = log(i3);  // 2 ln J
        return ((c11 + c22 - T(2)) * (T(0.5) * mu) - L * (T(0.5) * mu) + sq(L) * (T(0.125) * lam)) * s;
    }
};

// symmetric Dirichlet: A (|J|^2 + |J^-1|^2) = A tr C (1 + 1/det C)
template <typename T>
struct PsiSymDir {
    T s;  // rest area
    template <class A, class B, class C>
    ADM_HD auto operator()(const A &c11, const B &c22, const C &c12) const
    {
        auto tr = c11 + c22;
        auto det = c11 * c22 - sq(c12);
        return (tr + tr * recip(det)) * s;
    }
};

// learned membrane: the network's density tabulated per triangle in the
// invariants (I1, I2, I3) of C3 = diag(C, 1) -- value, gradient, upper
// Hessian (10 numbers) -- composed with I(C): I1 = c11 + c22 + 1,
// I3 = c11 c22 - c12^2, I2 = I3 + c11 + c22; times thickness * rest area
template <typename T>
struct PsiTable {
    const float *tab;
    T s;
    template <class A, class B, class C>
    ADM_HD auto operator()(const A &c11, const B &c22, const C &c12) const
    {
        auto i3 = c11 * c22 - sq(c12);
        auto i1 = c11 + c22 + T(1);
        auto i2 = i3 + c11 + c22;
        Dense<T, 3> p;
        p.v = (T)tab[0];
#pragma unroll
        for (int k = 0; k < 3; ++k) p.g[k] = (T)tab[1 + k];
#pragma unroll
        for (int q = 0; q < 6; ++q) p.h[q] = (T)tab[4 + q];
        return compose(p, i1, i2, i3) * s;
    }
};

// area from the Gram invariants of the edges: 1/2 sqrt(|u|^2 |w|^2 - (u.w)^2)
template <typename T>
struct PsiArea {
    template <class A, class B, class C>
    ADM_HD auto operator()(const A &uu, const B &ww, const C &uw) const
    {
        return sqrt(uu * ww - sq(uw)) * T(0.5);
    }
};

// --------------------------------------------------------------- output --
template <typename T, int K>
struct Local {
    T f;
    T g[K];
    T H[K * (K + 1) / 2];
};

template <typename T, int K, class R>
ADM_HD void store_local(const R &r, Local<T, K> &out)
{
    out.f = r.v;
#pragma unroll
    for (int i = 0; i < K; ++i) out.g[i] = gbit(R::gm, i) ? r.g[i] : T(0);
#pragma unroll
    for (int k = 0; k < K * (K + 1) / 2; ++k) out.H[k] = hbit(R::hl, R::hh, k) ? r.h[k] : T(0);
}

// ------------------------------------------------ edge-vector expansion --
// Terms are differentiated in the coordinates of NE edge vectors of their
// element (edge p = sum_a C[a][p] x_a over the NV vertices, C in {-1, 0, 1})
// and carried to the vertex DOFs by the chain rule through that constant map:
//   g_(a,d) = sum_p C[a][p] ge_(p,d),
//   H_(a,r),(b,s) = sum_(p,q) C[a][p] C[b][q] He_(p,r),(q,s).
// A triangle has 2 edge vectors (6 DOF instead of 9 for VD = 3), a hinge 3
// (9 instead of 12), so the invariants and the composition carry 21 / 45
// Hessian entries instead of 45 / 78.
// C[a][p] is packed two bits per entry at bit 2 (a NE + p): 0 -> 0, 1 -> +1, 2 -> -1
ADM_HD constexpr int edge_coef(uint64_t packed, int k) { return (int)((packed >> (2 * k)) & 1u) - (int)((packed >> (2 * k + 1)) & 1u); }
struct TriEdges {  // u = x1 - x0, w = x2 - x0: C = {{-1, -1}, {1, 0}, {0, 1}}
    static constexpr int NV = 3, NE = 2;
    ADM_HD static constexpr int C(int a, int p) { return edge_coef(0x41Au, a * NE + p); }
};
struct HingeEdges {  // e = x1 - x0, u = xa - x0, v = xb - x1: C = {{-1, -1, 0}, {1, 0, -1}, {0, 1, 0}, {0, 0, 1}}
    static constexpr int NV = 4, NE = 3;
    ADM_HD static constexpr int C(int a, int p) { return edge_coef(0x40484Au, a * NE + p); }
};
static_assert(TriEdges::C(0, 0) == -1 && TriEdges::C(0, 1) == -1 && TriEdges::C(1, 0) == 1 && TriEdges::C(1, 1) == 0 &&
              TriEdges::C(2, 0) == 0 && TriEdges::C(2, 1) == 1, "triangle edge map");
static_assert(HingeEdges::C(0, 0) == -1 && HingeEdges::C(0, 1) == -1 && HingeEdges::C(0, 2) == 0 &&
              HingeEdges::C(1, 0) == 1 && HingeEdges::C(1, 1) == 0 && HingeEdges::C(1, 2) == -1 &&
              HingeEdges::C(2, 0) == 0 && HingeEdges::C(2, 1) == 1 && HingeEdges::C(2, 2) == 0 &&
              HingeEdges::C(3, 0) == 0 && HingeEdges::C(3, 1) == 0 && HingeEdges::C(3, 2) == 1, "hinge edge map");

struct SpringEdges {  // d = x0 - x1: C = {{1}, {-1}}
    static constexpr int NV = 2, NE = 1;
    ADM_HD static constexpr int C(int a, int p) { return edge_coef(0x9u, a * NE + p); }
};
static_assert(SpringEdges::C(0, 0) == 1 && SpringEdges::C(1, 0) == -1, "spring edge map");

template <class E, int VD, typename T>
ADM_HD void expand_edges(const Local<T, E::NE * VD> &le, Local<T, E::NV * VD> &out)
{
    constexpr int NE = E::NE, K = E::NV * VD;
    out.f = le.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int a = i / VD, d = i % VD;
        T acc = -T(0);
#pragma unroll
        for (int p = 0; p < NE; ++p) {
            if (E::C(a, p) == 0) continue;
            acc = E::C(a, p) > 0 ? acc + le.g[p * VD + d] : acc - le.g[p * VD + d];
        }
        out.g[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int i = 0; i <= j; ++i) {
            const int a = i / VD, r = i % VD, b = j / VD, s = j % VD;
            T acc = -T(0);
#pragma unroll
            for (int p = 0; p < NE; ++p)
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    const int c = E::C(a, p) * E::C(b, q);
                    if (c == 0) continue;
                    const int ii = p * VD + r, jj = q * VD + s;
                    const T h = le.H[ii <= jj ? hix(ii, jj) : hix(jj, ii)];
                    acc = c > 0 ? acc + h : acc - h;
                }
            out.H[hix(i, j)] = acc;
        }
}

// A term's derivatives kept in its edge-vector coordinates.  The vertex-DOF
// gradient and Hessian entries are formed on demand (local_g, local_H) by the
// sums expand_edges does, in the same order, so a consumer that adds them
// into accumulators one at a time never holds the expanded Hessian.
template <class E, int VD, typename T>
struct EdgeLocal {
    using Edges = E;
    static constexpr int vd = VD;
    Local<T, E::NE * VD> e;
};
template <class Out>
struct IsEdgeLocal : std::false_type {};
template <class E, int VD, typename T>
struct IsEdgeLocal<EdgeLocal<E, VD, T>> : std::true_type {};

// hand a term's edge-coordinate result to its output: kept as it is, or
// expanded to the vertex DOFs
template <class E, int VD, typename T, class Out>
ADM_HD void emit_local(const Local<T, E::NE * VD> &le, Out &out)
{
    if constexpr (IsEdgeLocal<Out>::value) {
        static_assert(std::is_same_v<typename Out::Edges, E> && Out::vd == VD, "edge map of the term");
        out.e = le;
    } else {
        expand_edges<E, VD>(le, out);
    }
}

template <typename T, int K>
ADM_HD T local_f(const Local<T, K> &L) { return L.f; }
template <typename T, int K>
ADM_HD T local_g(const Local<T, K> &L, int i) { return L.g[i]; }
template <typename T, int K>
ADM_HD T local_H(const Local<T, K> &L, int i, int j) { return L.H[i <= j ? hix(i, j) : hix(j, i)]; }

template <class E, int VD, typename T>
ADM_HD T local_f(const EdgeLocal<E, VD, T> &L) { return L.e.f; }

template <class E, int VD, typename T>
ADM_HD T local_g(const EdgeLocal<E, VD, T> &L, int i)
{
    const int a = i / VD, d = i % VD;
    T acc = -T(0);
#pragma unroll
    for (int p = 0; p < E::NE; ++p) {
        if (E::C(a, p) == 0) continue;
        acc = E::C(a, p) > 0 ? acc + L.e.g[p * VD + d] : acc - L.e.g[p * VD + d];
    }
    return acc;
}

template <class E, int VD, typename T>
ADM_HD T local_H(const EdgeLocal<E, VD, T> &L, int i0, int j0)
{
    const int i = i0 <= j0 ? i0 : j0, j = i0 <= j0 ? j0 : i0;  // the upper entry, as expand_edges forms it
    const int a = i / VD, r = i % VD, b = j / VD, s = j % VD;
    T acc = -T(0);
#pragma unroll
    for (int p = 0; p < E::NE; ++p)
#pragma unroll
        for (int q = 0; q < E::NE; ++q) {
            const int c = E::C(a, p) * E::C(b, q);
            if (c == 0) continue;
            const int ii = p * VD + r, jj = q * VD + s;
            const T h = L.e.H[ii <= jj ? hix(ii, jj) : hix(jj, ii)];
            acc = c > 0 ? acc + h : acc - h;
        }
    return acc;
}

// ------------------------------------------------------ triangle, VD = 3 --
// C = F^T F of F = [x1-x0, x2-x0] Dinv;  Dinv row-major (d00, d01, d10, d11).
// Differentiated in the edge vectors u = x1 - x0, w = x2 - x0.
template <typename T, class Psi, bool PROJ = false, class Out>
ADM_HD void membrane_local(const T (&x)[9], const T (&D)[4], const Psi &psi, Out &out, T eps = T(0))
{
    auto u0 = seed<T, 6, 0>(x[3] - x[0]);
    auto u1 = seed<T, 6, 1>(x[4] - x[1]);
    auto u2 = seed<T, 6, 2>(x[5] - x[2]);
    auto w0 = seed<T, 6, 3>(x[6] - x[0]);
    auto w1 = seed<T, 6, 4>(x[7] - x[1]);
    auto w2 = seed<T, 6, 5>(x[8] - x[2]);
    auto a0 = u0 * D[0] + w0 * D[2];               // first column of F
    auto a1 = u1 * D[0] + w1 * D[2];
    auto a2 = u2 * D[0] + w2 * D[2];
    auto b0 = u0 * D[1] + w0 * D[3];               // second column of F
    auto b1 = u1 * D[1] + w1 * D[3];
    auto b2 = u2 * D[1] + w2 * D[3];
    auto c11 = sq(a0) + sq(a1) + sq(a2);
    auto c22 = sq(b0) + sq(b1) + sq(b2);
    auto c12 = a0 * b0 + a1 * b1 + a2 * b2;
    auto p = psi(seed<T, 3, 0>(c11.v), seed<T, 3, 1>(c22.v), seed<T, 3, 2>(c12.v));
    Local<T, 6> le;
    store_local(compose(p, c11, c22, c12), le);
    if constexpr (PROJ) project_edges<TriEdges, 3>(le.H, eps);
    emit_local<TriEdges, 3>(le, out);
}

// area term (test energy of Sec. 7.6), in the edge vectors u, w
template <typename T, bool PROJ = false, class Out>
ADM_HD void area_local(const T (&x)[9], Out &out, T eps = T(0))
{
    auto u0 = seed<T, 6, 0>(x[3] - x[0]);
    auto u1 = seed<T, 6, 1>(x[4] - x[1]);
    auto u2 = seed<T, 6, 2>(x[5] - x[2]);
    auto w0 = seed<T, 6, 3>(x[6] - x[0]);
    auto w1 = seed<T, 6, 4>(x[7] - x[1]);
    auto w2 = seed<T, 6, 5>(x[8] - x[2]);
    auto uu = sq(u0) + sq(u1) + sq(u2);
    auto ww = sq(w0) + sq(w1) + sq(w2);
    auto uw = u0 * w0 + u1 * w1 + u2 * w2;
    auto p = PsiArea<T>{}(seed<T, 3, 0>(uu.v), seed<T, 3, 1>(ww.v), seed<T, 3, 2>(uw.v));
    Local<T, 6> le;
    store_local(compose(p, uu, ww, uw), le);
    if constexpr (PROJ) project_edges<TriEdges, 3>(le.H, eps);
    emit_local<TriEdges, 3>(le, out);
}

// ------------------------------------------------------ triangle, VD = 2 --
// C = J^T J of the UV Jacobian J = [b-a, c-a] Dinv, differentiated in the
// edge vectors b - a, c - a; returns det J (value)
template <typename T, class Psi, bool PROJ = false, class Out>
ADM_HD T uv_local(const T (&x)[6], const T (&D)[4], const Psi &psi, Out &out, T eps = T(0))
{
    auto u0 = seed<T, 4, 0>(x[2] - x[0]);  // b - a
    auto u1 = seed<T, 4, 1>(x[3] - x[1]);
    auto w0 = seed<T, 4, 2>(x[4] - x[0]);  // c - a
    auto w1 = seed<T, 4, 3>(x[5] - x[1]);
    auto j00 = u0 * D[0] + w0 * D[2];
    auto j10 = u1 * D[0] + w1 * D[2];
    auto j01 = u0 * D[1] + w0 * D[3];
    auto j11 = u1 * D[1] + w1 * D[3];
    auto c11 = sq(j00) + sq(j10);
    auto c22 = sq(j01) + sq(j11);
    auto c12 = j00 * j01 + j10 * j11;
    auto p = psi(seed<T, 3, 0>(c11.v), seed<T, 3, 1>(c22.v), seed<T, 3, 2>(c12.v));
    Local<T, 4> le;
    store_local(compose(p, c11, c22, c12), le);
    if constexpr (PROJ) project_edges<TriEdges, 2>(le.H, eps);
    emit_local<TriEdges, 2>(le, out);
    return j00.v * j11.v - j01.v * j10.v;
}

// ----------------------------------------------------------------- hinge --
// hinge (x0, x1, xa, xb), face A = (x0, x1, xa), face B = (x1, x0, xb);
// psi = w (theta - thetabar)^2, differentiated in the edge vectors e, u, v.
// Returns false for a degenerate hinge.
template <typename T, bool PROJ = false, class Out>
ADM_HD bool hinge_local(const T (&x)[12], T thetabar, T w, Out &out, T eps = T(0))
{
    auto e0 = seed<T, 9, 0>(x[3] - x[0]);  // e = x1 - x0
    auto e1 = seed<T, 9, 1>(x[4] - x[1]);
    auto e2 = seed<T, 9, 2>(x[5] - x[2]);
    auto u0 = seed<T, 9, 3>(x[6] - x[0]);  // u = xa - x0
    auto u1 = seed<T, 9, 4>(x[7] - x[1]);
    auto u2 = seed<T, 9, 5>(x[8] - x[2]);
    auto v0 = seed<T, 9, 6>(x[9] - x[3]);  // v = xb - x1
    auto v1 = seed<T, 9, 7>(x[10] - x[4]);
    auto v2 = seed<T, 9, 8>(x[11] - x[5]);
    auto ee = sq(e0) + sq(e1) + sq(e2);
    auto eu = e0 * u0 + e1 * u1 + e2 * u2;
    auto ev = e0 * v0 + e1 * v1 + e2 * v2;
    auto uv = u0 * v0 + u1 * v1 + u2 * v2;
    auto det = e0 * (u1 * v2 - u2 * v1) + e1 * (u2 * v0 - u0 * v2) + e2 * (u0 * v1 - u1 * v0);
    auto EE = seed<T, 5, 0>(ee.v);
    auto EU = seed<T, 5, 1>(eu.v);
    auto EV = seed<T, 5, 2>(ev.v);
    auto UV = seed<T, 5, 3>(uv.v);
    auto DD = seed<T, 5, 4>(det.v);
    auto ys = -(sqrt(EE) * DD);
    auto xc = EV * EU - EE * UV;
    if (!(xc.v != T(0) || ys.v != T(0))) return false;
    auto th = atan2(ys, xc);
    auto p = sq(th - thetabar) * w;
    Local<T, 9> le;
    store_local(compose(p, ee, eu, ev, uv, det), le);
    if constexpr (PROJ) project_edges<HingeEdges, 3>(le.H, eps);
    emit_local<HingeEdges, 3>(le, out);
    return true;
}

// ------------------------------------------------- mass-spring (Sec. 7.1) --
// spring of edge (x0, x1), squared rest length l2, times h^2:
// kh2 l2/2 (|d|^2 / l2 - 1)^2 = kh2 / (2 l2) (|d|^2 - l2)^2, d = x0 - x1,
// differentiated in d
template <typename T, bool PROJ = false, class Out>
ADM_HD void spring_local(const T (&x)[6], T l2, T kh2, Out &out, T eps = T(0))
{
    auto d0 = seed<T, 3, 0>(x[0] - x[3]);
    auto d1 = seed<T, 3, 1>(x[1] - x[4]);
    auto d2 = seed<T, 3, 2>(x[2] - x[5]);
    auto q = sq(d0) + sq(d1) + sq(d2);
    auto Q = seed<T, 1, 0>(q.v);
    auto p = sq(Q - l2) * (kh2 / (T(2) * l2));
    Local<T, 3> le;
    store_local(compose(p, q), le);
    if constexpr (PROJ) project_edges<SpringEdges, 3>(le.H, eps);
    emit_local<SpringEdges, 3>(le, out);
}

// vertex-vertex contact barrier (Sec. 7.7): c dhat (s - 1) ln s for
// s = |d| / dhat < 1 (else 0), d = x0 - x1, c = kappa/2 A_c h^2; differentiated
// in d.  Returns false outside the activation distance (out zeroed).
template <typename T, bool PROJ = false>
ADM_HD bool contact_local(const T (&x)[6], T c, T dhat, Local<T, 6> &out, T eps = T(0))
{
    const T r0 = x[0] - x[3], r1 = x[1] - x[4], r2 = x[2] - x[5];
    const T q0 = r0 * r0 + r1 * r1 + r2 * r2;
    if (!(q0 < dhat * dhat) || !(q0 > T(0))) {
        out.f = T(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) out.g[i] = T(0);
#pragma unroll
        for (int k = 0; k < 21; ++k) out.H[k] = T(0);
        return false;
    }
    auto d0 = seed<T, 3, 0>(r0);
    auto d1 = seed<T, 3, 1>(r1);
    auto d2 = seed<T, 3, 2>(r2);
    auto q = sq(d0) + sq(d1) + sq(d2);
    auto Q = seed<T, 1, 0>(q.v);
    auto sv = sqrt(Q) * (T(1) / dhat);
    auto p = (sv - T(1)) * log(sv) * (c * dhat);
    Local<T, 3> le;
    store_local(compose(p, q), le);
    if constexpr (PROJ) project_edges<SpringEdges, 3>(le.H, eps);
    expand_edges<SpringEdges, 3>(le, out);
    return true;
}

// vertex-face contact (Sec. 7.7) on (p, a, b, c), differentiated in
// r = p - a, e1 = b - a, e2 = c - a: C = {{1, 0, 0}, {-1, -1, -1}, {0, 1, 0}, {0, 0, 1}}
struct VFEdges {
    static constexpr int NV = 4, NE = 3;
    ADM_HD static constexpr int C(int a, int p) { return edge_coef(0x404A81u, a * NE + p); }
};
static_assert(VFEdges::C(0, 0) == 1 && VFEdges::C(0, 1) == 0 && VFEdges::C(0, 2) == 0 && VFEdges::C(1, 0) == -1 &&
                  VFEdges::C(1, 1) == -1 && VFEdges::C(1, 2) == -1 && VFEdges::C(2, 0) == 0 &&
                  VFEdges::C(2, 1) == 1 && VFEdges::C(2, 2) == 0 && VFEdges::C(3, 0) == 0 &&
                  VFEdges::C(3, 1) == 0 && VFEdges::C(3, 2) == 1,
              "vertex-face edge map");

// part of the triangle nearest to p: 0, 1, 2 the corners a, b, c; 3, 4, 5
// the edges ab, ac, bc; 6 the interior.  Signs of the projections of p onto
// the edge directions from each corner (the corners' and edges' Voronoi
// regions in the triangle's plane), in the precision of the term.
template <typename T>
ADM_HD int vf_region(const T (&r)[3], const T (&e1)[3], const T (&e2)[3])
{
    auto dot = [](const T *u, const T *w) { return u[0] * w[0] + u[1] * w[1] + u[2] * w[2]; };
    const T d1 = dot(e1, r), d2 = dot(e2, r);
    if (d1 <= T(0) && d2 <= T(0)) return 0;
    const T rb[3] = {r[0] - e1[0], r[1] - e1[1], r[2] - e1[2]};
    const T d3 = dot(e1, rb), d4 = dot(e2, rb);
    if (d3 >= T(0) && d4 <= d3) return 1;
    if (d1 * d4 - d3 * d2 <= T(0) && d1 >= T(0) && d3 <= T(0)) return 3;
    const T rc[3] = {r[0] - e2[0], r[1] - e2[1], r[2] - e2[2]};
    const T d5 = dot(e1, rc), d6 = dot(e2, rc);
    if (d6 >= T(0) && d5 <= d6) return 2;
    if (d5 * d2 - d1 * d6 <= T(0) && d2 >= T(0) && d6 <= T(0)) return 4;
    if (d3 * d6 - d5 * d4 <= T(0) && d4 >= d3 && d5 >= d6) return 5;
    return 6;
}

// squared distance from a point at w (relative to the edge start) to the
// line of direction t: |w|^2 - (w.t)^2 / |t|^2
template <class W0, class W1, class W2, class D0, class D1, class D2>
ADM_HD auto line_sq(const W0 &w0, const W1 &w1, const W2 &w2, const D0 &t0, const D1 &t1, const D2 &t2)
{
    return sq(w0) + sq(w1) + sq(w2) - sq(w0 * t0 + w1 * t1 + w2 * t2) / (sq(t0) + sq(t1) + sq(t2));
}

// barrier c dhat (s - 1) ln s of s = sqrt(q) / dhat, composed with q(x);
// false (nothing stored) when q is outside (0, dhat^2)
template <typename T, class Q>
ADM_HD bool barrier_of_sq(const Q &q, T c, T dhat, Local<T, 9> &le)
{
    if (!(q.v < dhat * dhat) || !(q.v > T(0))) return false;
    auto Q1 = seed<T, 1, 0>(q.v);
    auto sv = sqrt(Q1) * (T(1) / dhat);
    auto p = (sv - T(1)) * log(sv) * (c * dhat);
    store_local(compose(p, q), le);
    return true;
}

// vertex-face contact barrier: c dhat (s - 1) ln s, s = d / dhat < 1, d the
// distance from p to triangle (a, b, c), c = kappa/2 A_c h^2; the squared
// distance written for the region nearest to p (corner: |p - v|^2; edge:
// distance to its line; interior: ((p - a).n)^2 / |n|^2, n = e1 x e2).
// x = (p, a, b, c), 3 coordinates each.  Returns false outside dhat (out zeroed).
template <typename T, bool PROJ = false>
ADM_HD bool vf_local(const T (&x)[12], T c, T dhat, Local<T, 12> &out, T eps = T(0))
{
    T r[3], e1[3], e2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        r[d] = x[d] - x[3 + d];
        e1[d] = x[6 + d] - x[3 + d];
        e2[d] = x[9 + d] - x[3 + d];
    }
    const int reg = vf_region(r, e1, e2);
    auto R0 = seed<T, 9, 0>(r[0]);
    auto R1 = seed<T, 9, 1>(r[1]);
    auto R2 = seed<T, 9, 2>(r[2]);
    auto U0 = seed<T, 9, 3>(e1[0]);
    auto U1 = seed<T, 9, 4>(e1[1]);
    auto U2 = seed<T, 9, 5>(e1[2]);
    auto W0 = seed<T, 9, 6>(e2[0]);
    auto W1 = seed<T, 9, 7>(e2[1]);
    auto W2 = seed<T, 9, 8>(e2[2]);
    Local<T, 9> le;
    bool active;
    switch (reg) {
    case 0: active = barrier_of_sq(sq(R0) + sq(R1) + sq(R2), c, dhat, le); break;
    case 1: active = barrier_of_sq(sq(R0 - U0) + sq(R1 - U1) + sq(R2 - U2), c, dhat, le); break;
    case 2: active = barrier_of_sq(sq(R0 - W0) + sq(R1 - W1) + sq(R2 - W2), c, dhat, le); break;
    case 3: active = barrier_of_sq(line_sq(R0, R1, R2, U0, U1, U2), c, dhat, le); break;
    case 4: active = barrier_of_sq(line_sq(R0, R1, R2, W0, W1, W2), c, dhat, le); break;
    case 5: active = barrier_of_sq(line_sq(R0 - U0, R1 - U1, R2 - U2, W0 - U0, W1 - U1, W2 - U2), c, dhat, le); break;
    default: {
        auto n0 = U1 * W2 - U2 * W1;
        auto n1 = U2 * W0 - U0 * W2;
        auto n2 = U0 * W1 - U1 * W0;
        active = barrier_of_sq(sq(n0 * R0 + n1 * R1 + n2 * R2) / (sq(n0) + sq(n1) + sq(n2)), c, dhat, le);
    }
    }
    if (!active) {
        out.f = T(0);
#pragma unroll
        for (int i = 0; i < 12; ++i) out.g[i] = T(0);
#pragma unroll
        for (int k = 0; k < 78; ++k) out.H[k] = T(0);
        return false;
    }
    if constexpr (PROJ) project_edges<VFEdges, 3>(le.H, eps);
    expand_edges<VFEdges, 3>(le, out);
    return true;
}

// per-vertex inertia and gravity: m/2 |x - xhat|^2 - h2 m g.x (Hessian m I,
// semidefinite, so filtering never changes it)
template <typename T>
ADM_HD void vertex_local(const T (&x)[3], const T (&xh)[3], T m, T h2, const T (&g)[3], Local<T, 3> &out)
{
    auto X0 = seed<T, 3, 0>(x[0]);
    auto X1 = seed<T, 3, 1>(x[1]);
    auto X2 = seed<T, 3, 2>(x[2]);
    auto f = (sq(X0 - xh[0]) + sq(X1 - xh[1]) + sq(X2 - xh[2])) * (T(0.5) * m) -
             (X0 * g[0] + X1 * g[1] + X2 * g[2]) * (h2 * m);
    store_local(f, out);
}

// --------------------------------------------- ARAP-style residual (Eq. 3) --
// r = sqrt(A) vec_rowmajor(J - R(J)), R the closest rotation: with
// p = J00 + J11, q = J10 - J01, n = |(p, q)|, R = [[p, -q], [q, p]] / n.
// Out: r[4], Jr[4][6] over the local DOFs (vertex-major).
template <typename T>
ADM_HD bool arap_local(const T (&x)[6], const T (&D)[4], T sqrt_area, T (&r)[4], T (&Jr)[4][6])
{
    auto X0 = dseed<T, 6, 0>(x[0]);
    auto X1 = dseed<T, 6, 1>(x[1]);
    auto X2 = dseed<T, 6, 2>(x[2]);
    auto X3 = dseed<T, 6, 3>(x[3]);
    auto X4 = dseed<T, 6, 4>(x[4]);
    auto X5 = dseed<T, 6, 5>(x[5]);
    auto u0 = X2 - X0;
    auto u1 = X3 - X1;
    auto w0 = X4 - X0;
    auto w1 = X5 - X1;
    auto j00 = u0 * D[0] + w0 * D[2];
    auto j10 = u1 * D[0] + w1 * D[2];
    auto j01 = u0 * D[1] + w0 * D[3];
    auto j11 = u1 * D[1] + w1 * D[3];
    auto p = j00 + j11;
    auto q = j10 - j01;
    T n2 = p.v * p.v + q.v * q.v;
    if (!(n2 > T(0))) return false;
    T in = T(1) / Fn<T>::sqrt_(n2);
    T in3 = in * in * in;
    // c = p/n, s = q/n:  dc = (q^2 dp - p q dq)/n^3, ds = (p^2 dq - p q dp)/n^3
    auto c = dchain2(p, q, p.v * in, q.v * q.v * in3, -p.v * q.v * in3);
    auto s = dchain2(p, q, q.v * in, -p.v * q.v * in3, p.v * p.v * in3);
    auto r0 = (j00 - c) * sqrt_area;
    auto r1 = (j01 + s) * sqrt_area;
    auto r2 = (j10 - s) * sqrt_area;
    auto r3 = (j11 - c) * sqrt_area;
    r[0] = r0.v;
    r[1] = r1.v;
    r[2] = r2.v;
    r[3] = r3.v;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Jr[0][i] = gbit(decltype(r0)::gm, i) ? r0.g[i] : T(0);
        Jr[1][i] = gbit(decltype(r1)::gm, i) ? r1.g[i] : T(0);
        Jr[2][i] = gbit(decltype(r2)::gm, i) ? r2.g[i] : T(0);
        Jr[3][i] = gbit(decltype(r3)::gm, i) ? r3.g[i] : T(0);
    }
    return true;
}

}  // namespace adm
