// atomic_impl.cuh -- per-element kernels with the paper's assembly scheme:
// one thread per element, local derivatives by forward-mode AD in registers
// (Sec. 5.1, Sec. 6.2), global atomic scatter through the precomputed slot
// map into zeroed outputs (Sec. 5.5).  Kept as the reference assembler.
#pragma once

#include "device_common.cuh"

namespace adm {

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
        const bool ok = tri_term<T, ENERGY>(x, D, area, A.c, L);
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

template <typename T>
adm_status eval_atomic(adm_ctx *h, const EvalArgs &a)
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
    return launch_reduce(h, a, tri ? h->tri_blocks.d_mesh_block_off : nullptr,
                         hin ? h->hinge_blocks.d_mesh_block_off : nullptr, tri ? h->tri_blocks.n_blocks : 0, tm);
}

}  // namespace adm
