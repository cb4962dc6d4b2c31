// ring.cu -- per-vertex one-ring terms.  A term over the closed one-ring
// (v, n_0, .., n_{k-1}) of every vertex: the uniform-Laplacian (umbrella)
// smoothing energy w/2 |x_v - (1/k) sum_j x_{n_j}|^2.  Its local derivatives
// come from forward mode over the ring's positions, one coordinate at a time
// (the energy is a sum over coordinates, so cross-coordinate second
// derivatives vanish), with the ring padded to kMaxValence neighbours.  The
// rings have different sizes, so this term runs one thread per vertex and
// scatters into the two-ring block pattern through a precomputed slot map
// with atomic additions (the paper's scheme, Sec. 5.5), instead of the tiles.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace adm {

namespace {

constexpr int kRingThreads = 128;
constexpr int kRingN = kMaxValence + 1;  // seeds: the vertex and up to kMaxValence neighbours

// sum over seeds J..kRingN-1 of w_j x_j as one active value (compile-time recursion:
// every term has its own derivative mask, so the sum's type grows with it)
template <int J, typename T>
__device__ __forceinline__ auto ring_sum(const T (&xs)[kRingN], const T (&ws)[kRingN])
{
    if constexpr (J == kRingN - 1) return seed<T, kRingN, J>(xs[J]) * ws[J];
    else return seed<T, kRingN, J>(xs[J]) * ws[J] + ring_sum<J + 1>(xs, ws);
}

template <typename T>
struct RingArgs {
    int64_t nV;
    const int32_t *ring_off, *ring, *slots, *slot_off;
    const int32_t *blk_begin, *blk_end;
    const T *x, *v;
    T *grad, *bsr, *hv;
    double *epart;
    T w;
};

template <typename T, int VD, int MODE>
__global__ void __launch_bounds__(kRingThreads) k_ring(RingArgs<T> A)
{
    const int32_t b0 = A.blk_begin[blockIdx.x], b1 = A.blk_end[blockIdx.x];
    const int64_t vtx = (int64_t)b0 + threadIdx.x;
    double fe = 0.0;
    if (vtx < b1) {
        const int32_t r0 = A.ring_off[vtx], k = A.ring_off[vtx + 1] - r0;
        int32_t vid[kRingN];
        vid[0] = (int32_t)vtx;
#pragma unroll
        for (int j = 1; j < kRingN; ++j) vid[j] = j <= k ? A.ring[r0 + j - 1] : (int32_t)vtx;
        const T inv = k > 0 ? T(1) / T(k) : T(0);
        const int32_t *sl = A.slots + A.slot_off[vtx];  // (k + 1)^2, row-major
#pragma unroll 1
        for (int d = 0; d < VD; ++d) {
            // L_d = x_v - (1/k) sum_j x_{n_j}, padded seeds weighted 0
            T xs[kRingN], ws[kRingN];
#pragma unroll
            for (int j = 0; j < kRingN; ++j) {
                xs[j] = A.x[(int64_t)vid[j] * VD + d];
                ws[j] = (j >= 1 && j <= k) ? inv : T(0);
            }
            const auto L = seed<T, kRingN, 0>(xs[0]) - ring_sum<1>(xs, ws);
            const auto E = sq(L) * (T(0.5) * A.w);
            fe += (double)E.v;
            if (MODE >= MODE_GRAD && A.grad)
#pragma unroll
                for (int a = 0; a < kRingN; ++a)
                    if (a <= k) atomicAdd(A.grad + (int64_t)vid[a] * VD + d, E.g[a]);
            if (MODE == MODE_HESS) {
#pragma unroll
                for (int a = 0; a < kRingN; ++a)
#pragma unroll
                    for (int b = 0; b < kRingN; ++b)
                        if (a <= k && b <= k)
                            atomicAdd(A.bsr + (int64_t)sl[a * (k + 1) + b] * (VD * VD) + d * VD + d,
                                      E.h[a <= b ? hix(a, b) : hix(b, a)]);
            } else if (MODE == MODE_HVP) {
#pragma unroll
                for (int a = 0; a < kRingN; ++a) {
                    if (a > k) continue;
                    T y = -T(0);
#pragma unroll
                    for (int b = 0; b < kRingN; ++b)
                        if (b <= k) y += E.h[a <= b ? hix(a, b) : hix(b, a)] * A.v[(int64_t)vid[b] * VD + d];
                    atomicAdd(A.hv + (int64_t)vid[a] * VD + d, y);
                }
            }
        }
    }
    const double s = block_sum<kRingThreads>(fe);
    if (threadIdx.x == 0) A.epart[blockIdx.x] = s;
}

template <typename T, int VD>
void launch(int mode, int nb, cudaStream_t s, const RingArgs<T> &A)
{
    if (mode == MODE_VALUE) k_ring<T, VD, MODE_VALUE><<<nb, kRingThreads, 0, s>>>(A);
    else if (mode == MODE_GRAD) k_ring<T, VD, MODE_GRAD><<<nb, kRingThreads, 0, s>>>(A);
    else if (mode == MODE_HESS) k_ring<T, VD, MODE_HESS><<<nb, kRingThreads, 0, s>>>(A);
    else k_ring<T, VD, MODE_HVP><<<nb, kRingThreads, 0, s>>>(A);
}

template <typename T>
adm_status eval_ring_t(adm_ctx *h, const EvalArgs &a)
{
    const HostMesh &m = h->m;
    const Pattern &P = h->pat[PAT_RING];
    const int vd = m.vdim;
    const int mode = a.hv ? MODE_HVP : (a.bsr ? MODE_HESS : (a.grad ? MODE_GRAD : MODE_VALUE));
    cudaStream_t s = a.stream;
    StageTimer tm(h, s);
    tm.begin(ADM_STAGE_ZERO);
    if (cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return ADM_ERR_CUDA;
    if (a.grad && cudaMemsetAsync(a.grad, 0, sizeof(T) * m.nV * vd, s) != cudaSuccess) return ADM_ERR_CUDA;
    if (a.bsr && cudaMemsetAsync(a.bsr, 0, sizeof(T) * P.nnzb * vd * vd, s) != cudaSuccess) return ADM_ERR_CUDA;
    if (a.hv && cudaMemsetAsync(a.hv, 0, sizeof(T) * m.nV * vd, s) != cudaSuccess) return ADM_ERR_CUDA;
    tm.end(ADM_STAGE_ZERO);
    RingArgs<T> A;
    A.nV = m.nV;
    A.ring_off = P.d_ring_off;
    A.ring = P.d_ring;
    A.slots = P.d_ring_slots;
    A.slot_off = P.d_ring_slot_off;
    A.blk_begin = h->vert_blocks.d_begin;
    A.blk_end = h->vert_blocks.d_end;
    A.x = (const T *)a.x;
    A.v = (const T *)a.v;
    A.grad = (T *)a.grad;
    A.bsr = (T *)a.bsr;
    A.hv = (T *)a.hv;
    A.epart = h->d_epart;
    EnergyParams p;
    auto it = h->params.find(ADM_UMBRELLA);
    if (it != h->params.end()) p = it->second;
    A.w = (T)p.w;
    tm.begin(ADM_STAGE_TRIANGLES);  // the per-element kernel stage
    if (vd == 3) launch<T, 3>(mode, h->vert_blocks.n_blocks, s, A);
    else launch<T, 2>(mode, h->vert_blocks.n_blocks, s, A);
    tm.end(ADM_STAGE_TRIANGLES);
    if (cudaGetLastError() != cudaSuccess) return ADM_ERR_CUDA;
    return launch_reduce(h, a, h->vert_blocks.d_mesh_block_off, nullptr, 0, tm);
}

}  // namespace

adm_status eval_ring(adm_ctx *h, const EvalArgs &a)
{
    if (h->vert_blocks.threads != kRingThreads) return ADM_ERR_UNSUPPORTED;
    return a.prec == ADM_FP32 ? eval_ring_t<float>(h, a) : eval_ring_t<double>(h, a);
}

}  // namespace adm
