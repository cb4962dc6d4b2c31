// kernels.cu -- sm_103a kernels of libadm and their launchers.
//
// Per element (one thread): gather the stencil's DOFs, run the term on the
// forward-mode engine (registers only, Sec. 5.1 / Sec. 6.2), then assemble
// g += S^T g_j and H += S^T H_j S (Eq. 2).  This file holds the per-element
// scatter assembler (global atomic additions through the precomputed slot
// map, the scheme of Sec. 5.5) and the deterministic FP64 reductions of the
// energy (Eq. 1) and of the gradient norm.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "terms.cuh"

namespace adm {

enum Mode { MODE_VALUE = 0, MODE_GRAD = 1, MODE_HESS = 2 };

template <typename T>
struct TermConsts {
    T mu, lam, thick, kbh2;
};

template <typename T>
struct ElemArgs {
    const int32_t *verts;   // nv per element
    const T *rest;          // SoA fields of n elements
    int64_t n;
    const int32_t *slots;   // nv * nv per element
    const int32_t *blk_begin, *blk_end;
    const T *x;
    T *grad;
    T *bsr;
    double *epart;          // one partial per block
    int *status;
    TermConsts<T> c;
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

template <typename T, int VD, int NV, int K>
__device__ __forceinline__ void scatter_atomic(const ElemArgs<T> &A, int64_t e, const int32_t (&v)[NV],
                                               const Local<T, K> &L, int mode)
{
    if (mode >= MODE_GRAD && A.grad) {
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
            for (int d = 0; d < VD; ++d) atomicAdd(A.grad + (int64_t)v[a] * VD + d, L.g[a * VD + d]);
    }
    if (mode >= MODE_HESS) {
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                const int32_t blk = A.slots[e * NV * NV + a * NV + b];
                T *out = A.bsr + (int64_t)blk * VD * VD;
#pragma unroll
                for (int r = 0; r < VD; ++r)
#pragma unroll
                    for (int s = 0; s < VD; ++s) {
                        const int i = a * VD + r, j = b * VD + s;
                        atomicAdd(out + r * VD + s, L.H[i <= j ? hix(i, j) : hix(j, i)]);
                    }
            }
    }
}

// ------------------------------------------------------------ triangles --
template <typename T, int ENERGY, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS) k_tri_atomic(ElemArgs<T> A)
{
    constexpr int VD = ENERGY == ADM_SYMDIR2D ? 2 : 3;
    constexpr int K = 3 * VD;
    const int64_t e = (int64_t)A.blk_begin[blockIdx.x] + threadIdx.x;
    double fe = 0.0;
    if (e < A.blk_end[blockIdx.x]) {
        int32_t v[3];
        T x[K];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] = A.verts[3 * e + a];
#pragma unroll
            for (int d = 0; d < VD; ++d) x[a * VD + d] = A.x[(int64_t)v[a] * VD + d];
        }
        T D[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = A.rest[k * A.n + e];
        const T area = A.rest[4 * A.n + e];
        Local<T, K> L;
        bool ok = true;
        if constexpr (ENERGY == ADM_SYMDIR2D) {
            T det = uv_local(x, D, PsiSymDir<T>{area}, L);
            ok = det > T(0);
        } else if constexpr (ENERGY == ADM_STVK_MEMBRANE || ENERGY == ADM_SHELL) {
            membrane_local(x, D, PsiStVK<T>{A.c.mu, A.c.lam, A.c.thick * area}, L);
        } else if constexpr (ENERGY == ADM_NH_MEMBRANE) {
            membrane_local(x, D, PsiNH<T>{A.c.mu, A.c.lam, A.c.thick * area}, L);
        } else if constexpr (ENERGY == ADM_AREA) {
            area_local(x, L);
        }
        ok = ok && isfinite(L.f);
        if (!ok) {
            atomicOr(A.status, ST_DOMAIN);
        } else {
            fe = (double)L.f;
            scatter_atomic<T, VD, 3, K>(A, e, v, L, MODE);
        }
    }
    double s = block_sum<THREADS>(fe);
    if (threadIdx.x == 0) A.epart[blockIdx.x] = s;
}

// --------------------------------------------------------------- hinges --
template <typename T, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS) k_hinge_atomic(ElemArgs<T> A)
{
    const int64_t e = (int64_t)A.blk_begin[blockIdx.x] + threadIdx.x;
    double fe = 0.0;
    if (e < A.blk_end[blockIdx.x]) {
        int32_t v[4];
        T x[12];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[a] = A.verts[4 * e + a];
#pragma unroll
            for (int d = 0; d < 3; ++d) x[a * 3 + d] = A.x[(int64_t)v[a] * 3 + d];
        }
        const T thetabar = A.rest[e];
        const T w = A.c.kbh2 * A.rest[A.n + e];
        Local<T, 12> L;
        bool ok = hinge_local(x, thetabar, w, L) && isfinite(L.f);
        if (!ok) {
            atomicOr(A.status, ST_DOMAIN);
        } else {
            fe = (double)L.f;
            scatter_atomic<T, 3, 4, 12>(A, e, v, L, MODE);
        }
    }
    double s = block_sum<THREADS>(fe);
    if (threadIdx.x == 0) A.epart[blockIdx.x] = s;
}

// ------------------------------------------------------------ reductions --
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_sumsq(const T *g, const int32_t *cb, const int32_t *ce,
                                                   double *gpart)
{
    double s = 0.0;
    for (int64_t i = cb[blockIdx.x] + threadIdx.x; i < ce[blockIdx.x]; i += THREADS) {
        double v = (double)g[i];
        s += v * v;
    }
    s = block_sum<THREADS>(s);
    if (threadIdx.x == 0) gpart[blockIdx.x] = s;
}

// per mesh: energy = sum of its element-block partials (triangle blocks, then
// hinge blocks), gnorm = sqrt(sum of its chunk partials); total = sum over
// meshes.  One block, fixed order.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_finalize(int n_mesh, const double *epart,
                                                      const int32_t *tri_off, const int32_t *hinge_off,
                                                      int32_t hinge_base, const double *gpart,
                                                      const int32_t *chunk_off, double *e_mesh,
                                                      double *gn_mesh, double *e_total)
{
    double tot = 0.0;
    for (int m = threadIdx.x; m < n_mesh; m += THREADS) {
        double e = 0.0;
        if (tri_off)
            for (int b = tri_off[m]; b < tri_off[m + 1]; ++b) e += epart[b];
        if (hinge_off)
            for (int b = hinge_off[m]; b < hinge_off[m + 1]; ++b) e += epart[hinge_base + b];
        if (e_mesh) e_mesh[m] = e;
        tot += e;
        if (gn_mesh) {
            double s = 0.0;
            for (int c = chunk_off[m]; c < chunk_off[m + 1]; ++c) s += gpart[c];
            gn_mesh[m] = ::sqrt(s);
        }
    }
    tot = block_sum<THREADS>(tot);
    if (threadIdx.x == 0 && e_total) *e_total = tot;
}

// ------------------------------------------------------ ARAP Jacobian ---
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_arap_jacobian(const int32_t *F, const T *rest, int64_t nT,
                                                           const T *x, const int32_t *slots, T *r,
                                                           T *jv, T *jtj, int *status)
{
    const int64_t t = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (t >= nT) return;
    int32_t v[3];
    T xl[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = F[3 * t + a];
        xl[2 * a] = x[2 * (int64_t)v[a]];
        xl[2 * a + 1] = x[2 * (int64_t)v[a] + 1];
    }
    T D[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) D[k] = rest[k * nT + t];
    const T sa = Fn<T>::sqrt_(rest[4 * nT + t]);
    T res[4], Jr[4][6];
    if (!arap_local(xl, D, sa, res, Jr)) {
        atomicOr(status, ST_DOMAIN);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            res[i] = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) Jr[i][c] = T(0);
        }
    }
    // columns of a row: local vertices sorted by global id, then coordinate
    int o0 = 0, o1 = 1, o2 = 2, tmp;
    if (v[o1] < v[o0]) { tmp = o0; o0 = o1; o1 = tmp; }
    if (v[o2] < v[o1]) { tmp = o1; o1 = o2; o2 = tmp; }
    if (v[o1] < v[o0]) { tmp = o0; o0 = o1; o1 = tmp; }
    const int ord[3] = {o0, o1, o2};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        r[4 * t + i] = res[i];
        if (jv) {
#pragma unroll
            for (int oi = 0; oi < 3; ++oi) {
                jv[24 * t + 6 * i + 2 * oi] = Jr[i][2 * ord[oi]];
                jv[24 * t + 6 * i + 2 * oi + 1] = Jr[i][2 * ord[oi] + 1];
            }
        }
    }
    if (!jtj) return;
    // J_t^T J_t: 6 x 6 over the local DOFs, assembled into the 2 x 2 blocks
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T *out = jtj + (int64_t)slots[9 * t + 3 * a + b] * 4;
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    T s = T(0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) s += Jr[i][2 * a + p] * Jr[i][2 * b + q];
                    atomicAdd(out + 2 * p + q, s);
                }
        }
}

// ------------------------------------------------------------ launchers --
static bool has_tris(int energy)
{
    return energy == ADM_SYMDIR2D || energy == ADM_STVK_MEMBRANE || energy == ADM_SHELL ||
           energy == ADM_NH_MEMBRANE || energy == ADM_AREA;
}
static bool has_hinges(int energy) { return energy == ADM_HINGE_BENDING || energy == ADM_SHELL; }

template <typename T>
static TermConsts<T> consts(const adm_ctx *h, int energy)
{
    EnergyParams p;
    auto it = h->params.find(energy);
    if (it != h->params.end()) p = it->second;
    TermConsts<T> c;
    c.mu = (T)p.mu();
    c.lam = (T)p.lambda();
    c.thick = (T)p.t;
    c.kbh2 = (T)(p.kbend() * p.h * p.h);
    return c;
}

template <typename T, int THREADS>
static void launch_tri(int energy, int mode, dim3 grid, cudaStream_t s, const ElemArgs<T> &A)
{
#define ADM_TRI(EN, MO) k_tri_atomic<T, EN, MO, THREADS><<<grid, THREADS, 0, s>>>(A)
#define ADM_TRI_MODES(EN)                                   \
    do {                                                     \
        if (mode == MODE_VALUE) ADM_TRI(EN, MODE_VALUE);     \
        else if (mode == MODE_GRAD) ADM_TRI(EN, MODE_GRAD);  \
        else ADM_TRI(EN, MODE_HESS);                         \
    } while (0)
    switch (energy) {
    case ADM_SYMDIR2D: ADM_TRI_MODES(ADM_SYMDIR2D); break;
    case ADM_STVK_MEMBRANE:
    case ADM_SHELL: ADM_TRI_MODES(ADM_STVK_MEMBRANE); break;
    case ADM_NH_MEMBRANE: ADM_TRI_MODES(ADM_NH_MEMBRANE); break;
    case ADM_AREA: ADM_TRI_MODES(ADM_AREA); break;
    default: break;
    }
#undef ADM_TRI_MODES
#undef ADM_TRI
}

template <typename T, int THREADS>
static void launch_hinge(int mode, dim3 grid, cudaStream_t s, const ElemArgs<T> &A)
{
    if (mode == MODE_VALUE) k_hinge_atomic<T, MODE_VALUE, THREADS><<<grid, THREADS, 0, s>>>(A);
    else if (mode == MODE_GRAD) k_hinge_atomic<T, MODE_GRAD, THREADS><<<grid, THREADS, 0, s>>>(A);
    else k_hinge_atomic<T, MODE_HESS, THREADS><<<grid, THREADS, 0, s>>>(A);
}

constexpr int kThreads = 128;
constexpr int kRedThreads = 256;

StageTimer::StageTimer(adm_ctx *h_, cudaStream_t s_) : h(h_), s(s_), slot(-1)
{
    if (h->prof_ring <= 0) return;
    slot = h->prof_next;
    h->prof_next = (h->prof_next + 1) % h->prof_ring;
    h->prof_count = std::min(h->prof_count + 1, h->prof_ring);
    for (int k = 0; k < ADM_N_STAGES; ++k) h->prof_ran[slot * ADM_N_STAGES + k] = 0;
}
void StageTimer::begin(int stage)
{
    if (slot < 0) return;
    cudaEventRecord(h->prof_ev[(slot * ADM_N_STAGES + stage) * 2 + 0], s);
}
void StageTimer::end(int stage)
{
    if (slot < 0) return;
    cudaEventRecord(h->prof_ev[(slot * ADM_N_STAGES + stage) * 2 + 1], s);
    h->prof_ran[slot * ADM_N_STAGES + stage] = 1;
}

template <typename T>
static adm_status eval_typed(adm_ctx *h, const EvalArgs &a)
{
    const HostMesh &m = h->m;
    const int vd = m.vdim;
    const int pk = has_hinges(a.energy) ? PAT_SHELL : PAT_TRI;
    const Pattern &P = h->pat[pk];
    const int mode = a.bsr ? MODE_HESS : (a.grad ? MODE_GRAD : MODE_VALUE);
    cudaStream_t s = a.stream;
    StageTimer tm(h, s);
    tm.begin(ADM_STAGE_ZERO);
    if (cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return ADM_ERR_CUDA;
    if (a.grad && cudaMemsetAsync(a.grad, 0, sizeof(T) * m.nV * vd, s) != cudaSuccess)
        return ADM_ERR_CUDA;
    if (a.bsr && cudaMemsetAsync(a.bsr, 0, sizeof(T) * P.nnzb * vd * vd, s) != cudaSuccess)
        return ADM_ERR_CUDA;
    tm.end(ADM_STAGE_ZERO);
    const int prec = a.prec;
    const TermConsts<T> c = consts<T>(h, a.energy);
    const bool tri = has_tris(a.energy), hin = has_hinges(a.energy);
    if (tri) {
        ElemArgs<T> A;
        A.verts = h->d_F;
        A.rest = (const T *)h->d_tri_rest[prec];
        A.n = m.nT;
        A.slots = P.d_tri_slots;
        A.blk_begin = h->tri_blocks.d_begin;
        A.blk_end = h->tri_blocks.d_end;
        A.x = (const T *)a.x;
        A.grad = (T *)a.grad;
        A.bsr = (T *)a.bsr;
        A.epart = h->d_epart;
        A.status = h->d_status;
        A.c = c;
        tm.begin(ADM_STAGE_TRIANGLES);
        launch_tri<T, kThreads>(a.energy, mode, dim3(h->tri_blocks.n_blocks), s, A);
        tm.end(ADM_STAGE_TRIANGLES);
    }
    if (hin) {
        ElemArgs<T> A;
        A.verts = h->d_H;
        A.rest = (const T *)h->d_hinge_rest[prec];
        A.n = m.nH();
        A.slots = P.d_hinge_slots;
        A.blk_begin = h->hinge_blocks.d_begin;
        A.blk_end = h->hinge_blocks.d_end;
        A.x = (const T *)a.x;
        A.grad = (T *)a.grad;
        A.bsr = (T *)a.bsr;
        A.epart = h->d_epart + (tri ? h->tri_blocks.n_blocks : 0);
        A.status = h->d_status;
        A.c = c;
        if (h->hinge_blocks.n_blocks > 0) {
            tm.begin(ADM_STAGE_HINGES);
            launch_hinge<T, kThreads>(mode, dim3(h->hinge_blocks.n_blocks), s, A);
            tm.end(ADM_STAGE_HINGES);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return ADM_ERR_CUDA;
    if (a.gnorm_per_mesh) {
        tm.begin(ADM_STAGE_GNORM);
        k_sumsq<T, kRedThreads><<<h->chunks.n_chunks, kRedThreads, 0, s>>>(
            (const T *)a.grad, h->chunks.d_begin, h->chunks.d_end, h->d_gpart);
        tm.end(ADM_STAGE_GNORM);
    }
    tm.begin(ADM_STAGE_FINALIZE);
    k_finalize<1024><<<1, 1024, 0, s>>>(
        m.n_mesh, h->d_epart, tri ? h->tri_blocks.d_mesh_block_off : nullptr,
        hin ? h->hinge_blocks.d_mesh_block_off : nullptr, tri ? h->tri_blocks.n_blocks : 0,
        h->d_gpart, h->chunks.d_mesh_chunk_off, a.energy_per_mesh, a.gnorm_per_mesh,
        a.energy_total);
    tm.end(ADM_STAGE_FINALIZE);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status launch_eval(adm_ctx *h, const EvalArgs &a)
{
    if (a.prec == ADM_FP32) return eval_typed<float>(h, a);
    return eval_typed<double>(h, a);
}

template <typename T>
static adm_status jac_typed(adm_ctx *h, const void *x, void *r, void *jv, void *jtj, cudaStream_t s)
{
    const HostMesh &m = h->m;
    const Pattern &P = h->pat[PAT_TRI];
    if (cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return ADM_ERR_CUDA;
    if (jtj && cudaMemsetAsync(jtj, 0, sizeof(T) * P.nnzb * 4, s) != cudaSuccess) return ADM_ERR_CUDA;
    const int prec = std::is_same<T, float>::value ? ADM_FP32 : ADM_FP64;
    const int64_t nb = (m.nT + kThreads - 1) / kThreads;
    k_arap_jacobian<T, kThreads><<<(unsigned)nb, kThreads, 0, s>>>(
        h->d_F, (const T *)h->d_tri_rest[prec], m.nT, (const T *)x, P.d_tri_slots, (T *)r, (T *)jv,
        (T *)jtj, h->d_status);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status launch_jacobian(adm_ctx *h, int prec, const void *x, void *r, void *jv, void *jtj,
                           cudaStream_t stream)
{
    if (prec == ADM_FP32) return jac_typed<float>(h, x, r, jv, jtj, stream);
    return jac_typed<double>(h, x, r, jv, jtj, stream);
}

}  // namespace adm
