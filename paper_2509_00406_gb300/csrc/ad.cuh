// ad.cuh -- forward-mode AD in registers for per-element mesh terms.
//
// Sec. 5.1 / Sec. 6.2 of the paper lift the local variables of one element
// into an active type carrying the value, the k-gradient and the k x k
// Hessian, fixed in size at compile time.  On GB300 the dense form of that
// type is ALU-bound (a k = 12 product is ~350 FMA), so this engine keeps the
// same semantics but makes the *sparsity* of every derivative part of the
// type:
//
//   SHD<T, N, G, HL, HH>   value v, gradient g[N], packed upper Hessian
//                          h[N(N+1)/2]; bit i of G says g[i] may be nonzero,
//                          bit k of the 128-bit mask (HL, HH) says h[k] may
//                          be nonzero.  Every operator computes the result
//                          masks at compile time and emits arithmetic only
//                          for entries that can be nonzero; after full
//                          unrolling the compiler keeps only those entries in
//                          registers.  Seeds have a single gradient bit.
//
//   compose(psi, q0..q_{M-1})   second-order chain rule
//                          d2 f = sum_a psi_a d2 q_a + sum_ab psi_ab dq_a dq_b^T
//                          for f = psi(q(x)): a term is written as a density
//                          psi over M <= 5 invariants (itself differentiated
//                          by a dense SHD over M seeds) composed with sparse
//                          invariants q(x) of the element's DOFs.
//
//   D1<T, N, G>            first-order dual (value + gradient) for Jacobians
//                          of vector-valued terms (Eq. 3).
//
// All loops are fully unrolled with compile-time trip counts; conditions on
// the masks fold to constants.  Accumulators start at -0.0 so that the first
// addition folds away (x + -0.0 == x exactly).
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#if defined(__CUDACC__)
#define ADM_HD __host__ __device__ __forceinline__
#else
#define ADM_HD inline
#endif

namespace adm {

// ---------------------------------------------------------------- masks --
ADM_HD constexpr int hix(int i, int j) { return j * (j + 1) / 2 + i; }  // i <= j

ADM_HD constexpr bool gbit(uint64_t g, int i) { return ((g >> i) & 1ull) != 0; }
ADM_HD constexpr bool hbit(uint64_t lo, uint64_t hi, int k)
{
    return k < 64 ? (((lo >> k) & 1ull) != 0) : (((hi >> (k - 64)) & 1ull) != 0);
}

// bits of the packed pairs (i <= j) with (ga_i & gb_j) | (ga_j & gb_i)
template <int N>
ADM_HD constexpr uint64_t outer_mask(uint64_t ga, uint64_t gb, bool high)
{
    uint64_t m = 0;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i <= j; ++i) {
            int k = hix(i, j);
            bool on = (gbit(ga, i) && gbit(gb, j)) || (gbit(ga, j) && gbit(gb, i));
            if (!on) continue;
            if (!high && k < 64) m |= (1ull << k);
            if (high && k >= 64) m |= (1ull << (k - 64));
        }
    return m;
}

template <int N>
ADM_HD constexpr uint64_t full_g() { return N >= 64 ? ~0ull : ((1ull << N) - 1ull); }

template <int N>
ADM_HD constexpr uint64_t full_h(bool high)
{
    return outer_mask<N>(full_g<N>(), full_g<N>(), high);
}

// ----------------------------------------------------------------- SHD ---
template <typename T, int N, uint64_t G, uint64_t HL, uint64_t HH>
struct SHD {
    static constexpr int n = N;
    static constexpr int nh = N * (N + 1) / 2;
    static constexpr uint64_t gm = G, hl = HL, hh = HH;
    using scalar = T;
    T v;
    T g[N];
    T h[nh];
    ADM_HD static constexpr bool G_(int i) { return gbit(G, i); }
    ADM_HD static constexpr bool H_(int k) { return hbit(HL, HH, k); }
};

template <typename T, int N>
using Const = SHD<T, N, 0, 0, 0>;

template <typename T, int N>
using Dense = SHD<T, N, full_g<N>(), full_h<N>(false), full_h<N>(true)>;

// seed variable I with value x: gradient e_I, zero Hessian
template <typename T, int N, int I>
ADM_HD SHD<T, N, (1ull << I), 0, 0> seed(T x)
{
    SHD<T, N, (1ull << I), 0, 0> r;
    r.v = x;
    r.g[I] = T(1);
    return r;
}

template <typename T, int N>
ADM_HD Const<T, N> cst(T x)
{
    Const<T, N> r;
    r.v = x;
    return r;
}

// ------------------------------------------------------ linear operators --
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1, uint64_t G2, uint64_t L2,
          uint64_t H2>
ADM_HD SHD<T, N, G1 | G2, L1 | L2, H1 | H2> operator+(const SHD<T, N, G1, L1, H1> &a,
                                                     const SHD<T, N, G2, L2, H2> &b)
{
    SHD<T, N, G1 | G2, L1 | L2, H1 | H2> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (gbit(G1, i) && gbit(G2, i)) r.g[i] = a.g[i] + b.g[i];
        else if (gbit(G1, i)) r.g[i] = a.g[i];
        else if (gbit(G2, i)) r.g[i] = b.g[i];
    }
#pragma unroll
    for (int k = 0; k < N * (N + 1) / 2; ++k) {
        if (hbit(L1, H1, k) && hbit(L2, H2, k)) r.h[k] = a.h[k] + b.h[k];
        else if (hbit(L1, H1, k)) r.h[k] = a.h[k];
        else if (hbit(L2, H2, k)) r.h[k] = b.h[k];
    }
    return r;
}

template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1>
ADM_HD SHD<T, N, G1, L1, H1> operator-(const SHD<T, N, G1, L1, H1> &a)
{
    SHD<T, N, G1, L1, H1> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (gbit(G1, i)) r.g[i] = -a.g[i];
#pragma unroll
    for (int k = 0; k < N * (N + 1) / 2; ++k)
        if (hbit(L1, H1, k)) r.h[k] = -a.h[k];
    return r;
}

template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1, uint64_t G2, uint64_t L2,
          uint64_t H2>
ADM_HD SHD<T, N, G1 | G2, L1 | L2, H1 | H2> operator-(const SHD<T, N, G1, L1, H1> &a,
                                                     const SHD<T, N, G2, L2, H2> &b)
{
    SHD<T, N, G1 | G2, L1 | L2, H1 | H2> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (gbit(G1, i) && gbit(G2, i)) r.g[i] = a.g[i] - b.g[i];
        else if (gbit(G1, i)) r.g[i] = a.g[i];
        else if (gbit(G2, i)) r.g[i] = -b.g[i];
    }
#pragma unroll
    for (int k = 0; k < N * (N + 1) / 2; ++k) {
        if (hbit(L1, H1, k) && hbit(L2, H2, k)) r.h[k] = a.h[k] - b.h[k];
        else if (hbit(L1, H1, k)) r.h[k] = a.h[k];
        else if (hbit(L2, H2, k)) r.h[k] = -b.h[k];
    }
    return r;
}

// scalar * SHD, SHD * scalar, SHD + scalar
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1>
ADM_HD SHD<T, N, G1, L1, H1> operator*(const SHD<T, N, G1, L1, H1> &a, T s)
{
    SHD<T, N, G1, L1, H1> r;
    r.v = a.v * s;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (gbit(G1, i)) r.g[i] = a.g[i] * s;
#pragma unroll
    for (int k = 0; k < N * (N + 1) / 2; ++k)
        if (hbit(L1, H1, k)) r.h[k] = a.h[k] * s;
    return r;
}
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1>
ADM_HD SHD<T, N, G1, L1, H1> operator*(T s, const SHD<T, N, G1, L1, H1> &a)
{
    return a * s;
}
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1>
ADM_HD SHD<T, N, G1, L1, H1> operator+(const SHD<T, N, G1, L1, H1> &a, T s)
{
    SHD<T, N, G1, L1, H1> r = a;
    r.v = a.v + s;
    return r;
}
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1>
ADM_HD SHD<T, N, G1, L1, H1> operator-(const SHD<T, N, G1, L1, H1> &a, T s)
{
    SHD<T, N, G1, L1, H1> r = a;
    r.v = a.v - s;
    return r;
}

// --------------------------------------------------------------- product --
template <int N, uint64_t G1, uint64_t L1, uint64_t H1, uint64_t G2, uint64_t L2, uint64_t H2>
struct MulMask {
    static constexpr uint64_t G = G1 | G2;
    static constexpr uint64_t L = L1 | L2 | outer_mask<N>(G1, G2, false);
    static constexpr uint64_t H = H1 | H2 | outer_mask<N>(G1, G2, true);
};

// (ab)'' = a'' b + a b'' + a' b'^T + b' a'^T
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1, uint64_t G2, uint64_t L2,
          uint64_t H2>
ADM_HD SHD<T, N, MulMask<N, G1, L1, H1, G2, L2, H2>::G, MulMask<N, G1, L1, H1, G2, L2, H2>::L,
           MulMask<N, G1, L1, H1, G2, L2, H2>::H>
operator*(const SHD<T, N, G1, L1, H1> &a, const SHD<T, N, G2, L2, H2> &b)
{
    using M = MulMask<N, G1, L1, H1, G2, L2, H2>;
    SHD<T, N, M::G, M::L, M::H> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (!gbit(M::G, i)) continue;
        T acc = -T(0);
        if (gbit(G1, i)) acc += a.g[i] * b.v;
        if (gbit(G2, i)) acc += a.v * b.g[i];
        r.g[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int i = 0; i <= j; ++i) {
            const int k = hix(i, j);
            if (!hbit(M::L, M::H, k)) continue;
            T acc = -T(0);
            if (hbit(L1, H1, k)) acc += a.h[k] * b.v;
            if (hbit(L2, H2, k)) acc += a.v * b.h[k];
            if (i == j) {
                if (gbit(G1, i) && gbit(G2, i)) acc += T(2) * (a.g[i] * b.g[i]);
            } else {
                if (gbit(G1, i) && gbit(G2, j)) acc += a.g[i] * b.g[j];
                if (gbit(G1, j) && gbit(G2, i)) acc += a.g[j] * b.g[i];
            }
            r.h[k] = acc;
        }
    }
    return r;
}

// ---------------------------------------------------------- chain rules --
// r = f(a): r' = f1 a', r'' = f1 a'' + f2 a' a'^T
template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1>
ADM_HD SHD<T, N, G1, L1 | outer_mask<N>(G1, G1, false), H1 | outer_mask<N>(G1, G1, true)>
chain1(const SHD<T, N, G1, L1, H1> &a, T f0, T f1, T f2)
{
    constexpr uint64_t L = L1 | outer_mask<N>(G1, G1, false);
    constexpr uint64_t H = H1 | outer_mask<N>(G1, G1, true);
    SHD<T, N, G1, L, H> r;
    r.v = f0;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (gbit(G1, i)) r.g[i] = f1 * a.g[i];
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int i = 0; i <= j; ++i) {
            const int k = hix(i, j);
            if (!hbit(L, H, k)) continue;
            T acc = -T(0);
            if (hbit(L1, H1, k)) acc += f1 * a.h[k];
            if (gbit(G1, i) && gbit(G1, j)) acc += f2 * (a.g[i] * a.g[j]);
            r.h[k] = acc;
        }
    }
    return r;
}

// r = f(a, b) with partials fa, fb, faa, fab, fbb
template <int N, uint64_t G1, uint64_t L1, uint64_t H1, uint64_t G2, uint64_t L2, uint64_t H2>
struct Chain2Mask {
    static constexpr uint64_t G = G1 | G2;
    static constexpr uint64_t L = L1 | L2 | outer_mask<N>(G, G, false);
    static constexpr uint64_t H = H1 | H2 | outer_mask<N>(G, G, true);
};

template <typename T, int N, uint64_t G1, uint64_t L1, uint64_t H1, uint64_t G2, uint64_t L2,
          uint64_t H2>
ADM_HD SHD<T, N, Chain2Mask<N, G1, L1, H1, G2, L2, H2>::G, Chain2Mask<N, G1, L1, H1, G2, L2, H2>::L,
           Chain2Mask<N, G1, L1, H1, G2, L2, H2>::H>
chain2(const SHD<T, N, G1, L1, H1> &a, const SHD<T, N, G2, L2, H2> &b, T f0, T fa, T fb, T faa,
       T fab, T fbb)
{
    using M = Chain2Mask<N, G1, L1, H1, G2, L2, H2>;
    SHD<T, N, M::G, M::L, M::H> r;
    r.v = f0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (!gbit(M::G, i)) continue;
        T acc = -T(0);
        if (gbit(G1, i)) acc += fa * a.g[i];
        if (gbit(G2, i)) acc += fb * b.g[i];
        r.g[i] = acc;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int i = 0; i <= j; ++i) {
            const int k = hix(i, j);
            if (!hbit(M::L, M::H, k)) continue;
            T acc = -T(0);
            if (hbit(L1, H1, k)) acc += fa * a.h[k];
            if (hbit(L2, H2, k)) acc += fb * b.h[k];
            if (gbit(G1, i) && gbit(G1, j)) acc += faa * (a.g[i] * a.g[j]);
            if (gbit(G2, i) && gbit(G2, j)) acc += fbb * (b.g[i] * b.g[j]);
            T cross = -T(0);
            if (gbit(G1, i) && gbit(G2, j)) cross += a.g[i] * b.g[j];
            if (gbit(G2, i) && gbit(G1, j)) cross += b.g[i] * a.g[j];
            if ((gbit(G1, i) && gbit(G2, j)) || (gbit(G2, i) && gbit(G1, j))) acc += fab * cross;
            r.h[k] = acc;
        }
    }
    return r;
}

// ------------------------------------------------------- elementary maps --
// active operands only (plain scalars keep the C math functions)
template <class A>
concept Active = requires { typename A::scalar; };

template <typename T> struct Fn;
// FP32 on the device: reciprocal by the fast divide intrinsic and square
// root as x rsqrt(x) (about 2 ulp each, against the correctly rounded forms'
// multi-instruction sequences); arguments are positive and normal where the
// terms call them (squared lengths, r^2 of atan2)
template <> struct Fn<float> {
#ifdef __CUDA_ARCH__
    ADM_HD static float sqrt_(float x) { return x * rsqrtf(x); }
    ADM_HD static float rcp_(float x) { return __fdividef(1.0f, x); }
#else
    ADM_HD static float sqrt_(float x) { return ::sqrtf(x); }
    ADM_HD static float rcp_(float x) { return 1.0f / x; }
#endif
    ADM_HD static float log_(float x) { return ::logf(x); }
    ADM_HD static float atan2_(float y, float x) { return ::atan2f(y, x); }
};
template <> struct Fn<double> {
    ADM_HD static double sqrt_(double x) { return ::sqrt(x); }
    ADM_HD static double log_(double x) { return ::log(x); }
    ADM_HD static double atan2_(double y, double x) { return ::atan2(y, x); }
    ADM_HD static double rcp_(double x) { return 1.0 / x; }
};

template <Active A>
ADM_HD auto sqrt(const A &a)
{
    using T = typename A::scalar;
    T s = Fn<T>::sqrt_(a.v);
    T is = Fn<T>::rcp_(s);
    return chain1(a, s, T(0.5) * is, T(-0.25) * is * Fn<T>::rcp_(a.v));
}

template <Active A>
ADM_HD auto log(const A &a)
{
    using T = typename A::scalar;
    T ia = Fn<T>::rcp_(a.v);
    return chain1(a, Fn<T>::log_(a.v), ia, -ia * ia);
}

template <Active A>
ADM_HD auto recip(const A &a)
{
    using T = typename A::scalar;
    T ia = Fn<T>::rcp_(a.v);
    return chain1(a, ia, -ia * ia, T(2) * ia * ia * ia);
}

template <Active A>
ADM_HD auto sq(const A &a)
{
    using T = typename A::scalar;
    return chain1(a, a.v * a.v, T(2) * a.v, T(2));
}

template <Active A, Active B>
ADM_HD auto operator/(const A &a, const B &b)
{
    return a * recip(b);
}

// theta = atan2(y, x); d/dy = x/r2, d/dx = -y/r2, d2/dy2 = -2xy/r4,
// d2/dx2 = 2xy/r4, d2/dydx = (y^2 - x^2)/r4
template <Active Y, Active X>
ADM_HD auto atan2(const Y &y, const X &x)
{
    using T = typename Y::scalar;
    T r2 = x.v * x.v + y.v * y.v;
    T ir2 = Fn<T>::rcp_(r2);
    T ir4 = ir2 * ir2;
    T xy2 = T(2) * x.v * y.v;
    return chain2(y, x, Fn<T>::atan2_(y.v, x.v), x.v * ir2, -y.v * ir2, -xy2 * ir4,
                  (y.v * y.v - x.v * x.v) * ir4, xy2 * ir4);
}

// ------------------------------------------------------------- compose ---
template <int I, int E, class F>
ADM_HD void sfor(F &&f)
{
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, E>(static_cast<F &&>(f));
    }
}

template <class... Q>
struct PackMask;
template <class Q0, class... Q>
struct PackMask<Q0, Q...> {
    static constexpr uint64_t G = (Q0::gm | ... | Q::gm);
    static constexpr uint64_t L = (Q0::hl | ... | Q::hl);
    static constexpr uint64_t H = (Q0::hh | ... | Q::hh);
};

template <int I, class Q0, class... Q>
ADM_HD const auto &pick(const Q0 &q0, const Q &...q)
{
    if constexpr (I == 0) return q0;
    else return pick<I - 1>(q...);
}

// f = psi(q_0(x), ..., q_{M-1}(x)) with psi an SHD over M inner seeds
// (value, gradient psi_a, Hessian psi_ab) and q_a SHDs over the N outer DOFs.
template <typename T, int M, uint64_t PG, uint64_t PL, uint64_t PH, class Q0, class... Q>
ADM_HD auto compose(const SHD<T, M, PG, PL, PH> &psi, const Q0 &q0, const Q &...qs)
{
    static_assert(1 + sizeof...(Q) == M, "one invariant per inner seed");
    constexpr int N = Q0::n;
    using PM = PackMask<Q0, Q...>;
    constexpr uint64_t G = PM::G;
    constexpr uint64_t L = PM::L | outer_mask<N>(G, G, false);
    constexpr uint64_t H = PM::H | outer_mask<N>(G, G, true);
    SHD<T, N, G, L, H> r;
    r.v = psi.v;
    // gradient: sum_a psi_a dq_a
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (!gbit(G, i)) continue;
        T acc = -T(0);
        sfor<0, M>([&](auto A) {
            constexpr int a = decltype(A)::value;
            const auto &qa = pick<a>(q0, qs...);
            using QA = std::decay_t<decltype(qa)>;
            if (gbit(PG, a) && gbit(QA::gm, i)) acc += psi.g[a] * qa.g[i];
        });
        r.g[i] = acc;
    }
    // Hessian: sum_a psi_a d2q_a + sum_b K[b][i] dq_b^T, row by row with
    // K[b][i] = sum_a psi_ab dq_a[i] formed for row i only (M values live
    // instead of M N)
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T K[M];
        sfor<0, M>([&](auto B) {
            constexpr int b = decltype(B)::value;
            T acc = -T(0);
            sfor<0, M>([&](auto A) {
                constexpr int a = decltype(A)::value;
                const auto &qa = pick<a>(q0, qs...);
                using QA = std::decay_t<decltype(qa)>;
                constexpr int k = a <= b ? hix(a, b) : hix(b, a);
                if (gbit(G, i) && hbit(PL, PH, k) && gbit(QA::gm, i)) acc += psi.h[k] * qa.g[i];
            });
            K[b] = acc;
        });
#pragma unroll
        for (int j = i; j < N; ++j) {
            const int k = hix(i, j);
            if (!hbit(L, H, k)) continue;
            T acc = -T(0);
            sfor<0, M>([&](auto A) {
                constexpr int a = decltype(A)::value;
                const auto &qa = pick<a>(q0, qs...);
                using QA = std::decay_t<decltype(qa)>;
                if (gbit(PG, a) && hbit(QA::hl, QA::hh, k)) acc += psi.g[a] * qa.h[k];
                if (gbit(G, i) && gbit(QA::gm, j)) acc += K[a] * qa.g[j];
            });
            r.h[k] = acc;
        }
    }
    return r;
}

// ------------------------------------------------------- first order D1 --
template <typename T, int N, uint64_t G>
struct D1 {
    static constexpr int n = N;
    static constexpr uint64_t gm = G;
    using scalar = T;
    T v;
    T g[N];
};

template <typename T, int N, int I>
ADM_HD D1<T, N, (1ull << I)> dseed(T x)
{
    D1<T, N, (1ull << I)> r;
    r.v = x;
    r.g[I] = T(1);
    return r;
}

template <typename T, int N, uint64_t G1, uint64_t G2>
ADM_HD D1<T, N, G1 | G2> operator+(const D1<T, N, G1> &a, const D1<T, N, G2> &b)
{
    D1<T, N, G1 | G2> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (gbit(G1, i) && gbit(G2, i)) r.g[i] = a.g[i] + b.g[i];
        else if (gbit(G1, i)) r.g[i] = a.g[i];
        else if (gbit(G2, i)) r.g[i] = b.g[i];
    }
    return r;
}

template <typename T, int N, uint64_t G1, uint64_t G2>
ADM_HD D1<T, N, G1 | G2> operator-(const D1<T, N, G1> &a, const D1<T, N, G2> &b)
{
    D1<T, N, G1 | G2> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (gbit(G1, i) && gbit(G2, i)) r.g[i] = a.g[i] - b.g[i];
        else if (gbit(G1, i)) r.g[i] = a.g[i];
        else if (gbit(G2, i)) r.g[i] = -b.g[i];
    }
    return r;
}

template <typename T, int N, uint64_t G1>
ADM_HD D1<T, N, G1> operator*(const D1<T, N, G1> &a, T s)
{
    D1<T, N, G1> r;
    r.v = a.v * s;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (gbit(G1, i)) r.g[i] = a.g[i] * s;
    return r;
}

template <typename T, int N, uint64_t G1, uint64_t G2>
ADM_HD D1<T, N, G1 | G2> operator*(const D1<T, N, G1> &a, const D1<T, N, G2> &b)
{
    D1<T, N, G1 | G2> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (gbit(G1, i) && gbit(G2, i)) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
        else if (gbit(G1, i)) r.g[i] = a.g[i] * b.v;
        else if (gbit(G2, i)) r.g[i] = a.v * b.g[i];
    }
    return r;
}

// r = f(a, b) with first partials
template <typename T, int N, uint64_t G1, uint64_t G2>
ADM_HD D1<T, N, G1 | G2> dchain2(const D1<T, N, G1> &a, const D1<T, N, G2> &b, T f0, T fa, T fb)
{
    D1<T, N, G1 | G2> r;
    r.v = f0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (gbit(G1, i) && gbit(G2, i)) r.g[i] = fa * a.g[i] + fb * b.g[i];
        else if (gbit(G1, i)) r.g[i] = fa * a.g[i];
        else if (gbit(G2, i)) r.g[i] = fb * b.g[i];
    }
    return r;
}

}  // namespace adm
