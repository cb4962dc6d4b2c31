// device_common.cuh -- definitions shared by the kernel translation units of
// libadm (one per assembler and precision, so that they compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "terms.cuh"

namespace adm {

constexpr int kThreads = 128;      // per-element kernels
constexpr int kRedThreads = 256;   // reductions
// tiled kernel: FP32 tiles run 512 threads at two blocks per SM (64
// registers, 32 warps per SM); FP64 and the Hessian-filtering variants keep
// 256 threads and the full register file
template <typename T, bool PROJ>
constexpr int tile_threads() { return (sizeof(T) == 4 && !PROJ) ? 512 : 256; }

template <typename T>
struct TermConsts {
    T mu, lam, thick, kbh2;
    T eps;  // Hessian filtering: value negative local eigenvalues are raised to
    T kh2, h2, rho, g[3];  // mass-spring: k h^2, h^2, areal density, gravity
};

// deterministic block sum of one double per thread (fixed tree order)
template <int THREADS>
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < THREADS / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

// ------------------------------------------------- bulk (TMA) copies --
// One thread: initialise the mbarrier for one arrival, arm it with the byte
// count and start a bulk copy global -> shared that completes it.  dst, src
// and bytes must be multiples of 16 (bytes below 2^20).
__device__ __forceinline__ void bulk_load_start(uint64_t *bar, void *dst, const void *src, uint32_t bytes)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// Wait for phase 0 of the mbarrier; gives up after about a second (2^20
// waits of at most ~1 us each) and returns false.
__device__ __forceinline__ bool bulk_load_wait(uint64_t *bar)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(1000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ----------------------------------------------------- term evaluation --
template <int ENERGY>
struct TriTraits {
    static constexpr int VD = ENERGY == ADM_SYMDIR2D ? 2 : 3;
    static constexpr int K = 3 * VD;
};

// local f, g, H of one triangle term; false outside the energy's domain
// (PROJ: with the local Hessian filtered, spd.cuh)
template <typename T, int ENERGY, bool PROJ = false, class Out>
__device__ __forceinline__ bool tri_term(const T (&x)[TriTraits<ENERGY>::K], const T (&D)[4], T area,
                                         const TermConsts<T> &c, Out &L, const float *tab = nullptr)
{
    bool ok = true;
    if constexpr (ENERGY == ADM_SYMDIR2D) {
        T det = uv_local<T, PsiSymDir<T>, PROJ>(x, D, PsiSymDir<T>{area}, L, c.eps);
        ok = det > T(0);
    } else if constexpr (ENERGY == ADM_STVK_MEMBRANE || ENERGY == ADM_SHELL) {
        membrane_local<T, PsiStVK<T>, PROJ>(x, D, PsiStVK<T>{c.mu, c.lam, c.thick * area}, L, c.eps);
    } else if constexpr (ENERGY == ADM_NH_MEMBRANE) {
        membrane_local<T, PsiNH<T>, PROJ>(x, D, PsiNH<T>{c.mu, c.lam, c.thick * area}, L, c.eps);
    } else if constexpr (ENERGY == ADM_AREA) {
        area_local<T, PROJ>(x, L, c.eps);
    } else if constexpr (ENERGY == ADM_MLP_MEMBRANE) {
        membrane_local<T, PsiTable<T>, PROJ>(x, D, PsiTable<T>{tab, c.thick * area}, L, c.eps);
    }
    return ok && isfinite(local_f(L));
}

inline bool has_tris(int energy)
{
    return energy == ADM_SYMDIR2D || energy == ADM_STVK_MEMBRANE || energy == ADM_SHELL ||
           energy == ADM_NH_MEMBRANE || energy == ADM_AREA;
}
inline bool has_hinges(int energy) { return energy == ADM_HINGE_BENDING || energy == ADM_SHELL; }

template <typename T>
inline TermConsts<T> consts(const adm_ctx *h, int energy)
{
    EnergyParams p;
    auto it = h->params.find(energy);
    if (it != h->params.end()) p = it->second;
    TermConsts<T> c;
    c.mu = (T)p.mu();
    c.lam = (T)p.lambda();
    c.thick = (T)p.t;
    c.kbh2 = (T)(p.kbend() * p.h * p.h);
    c.eps = (T)h->proj_eps;
    c.kh2 = (T)(p.k * p.dt * p.dt);
    c.h2 = (T)(p.dt * p.dt);
    c.rho = (T)p.rho;
    for (int d = 0; d < 3; ++d) c.g[d] = (T)p.g[d];
    return c;
}


// per-assembler evaluations (explicitly instantiated for float and double)
template <typename T>
adm_status eval_atomic(adm_ctx *h, const EvalArgs &a);
template <typename T>
adm_status eval_tiled(adm_ctx *h, const EvalArgs &a);

// FP64 per-mesh energy (from element-block or tile partials) and gradient
// norm, enqueued after an assembler (reduce.cu)
adm_status launch_reduce(adm_ctx *h, const EvalArgs &a, const int32_t *tri_off, const int32_t *hinge_off,
                         int32_t hinge_base, StageTimer &tm);

}  // namespace adm
