// reduce.cu -- FP64 reductions (Eq. 1 energy per mesh, gradient norm), the
// stage timer, the evaluation dispatch and the least-squares Jacobian kernel.
#include "device_common.cuh"

namespace adm {

// ------------------------------------------------------------ reductions --
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_sumsq(const T *g, const int32_t *cb, const int32_t *ce,
                                                   double *gpart)
{
    double s = 0.0;
    const int64_t e = ce[blockIdx.x];
    int64_t i = cb[blockIdx.x] + threadIdx.x;
    if constexpr (sizeof(T) == 4) {
        // FP32 entries: squares, and sums of four of them, in FP32 (relative
        // error below 2^-22 per group of four), groups accumulated in FP64.
        // The FP64 pipe of this GPU runs at a small fraction of the FP32
        // rate; it now does one add per four entries instead of a convert
        // and a fused multiply-add per entry.
        // unrolled so that several rounds of loads are in flight; the
        // summation order (one running sum per thread) is unchanged
#pragma unroll 4
        for (; i + 3 * THREADS < e; i += 4 * THREADS) {
            const float v0 = g[i], v1 = g[i + THREADS], v2 = g[i + 2 * THREADS], v3 = g[i + 3 * THREADS];
            s += (double)((v0 * v0 + v1 * v1) + (v2 * v2 + v3 * v3));
        }
    }
#pragma unroll 4
    for (; i < e; i += THREADS) {
        const double v = (double)g[i];
        s += v * v;
    }
    s = block_sum<THREADS>(s);
    if (threadIdx.x == 0) gpart[blockIdx.x] = s;
}

// per mesh, one warp: energy = sum of its element-block partials (triangle
// blocks, then hinge blocks), gnorm = sqrt(sum of its chunk partials).  The
// lanes stride over the partials and a fixed shuffle tree adds them, so the
// result does not depend on scheduling.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in lane 0
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_mesh_sums(int n_mesh, const double *epart, const int32_t *tri_off,
                                                       const int32_t *hinge_off, int32_t hinge_base,
                                                       const double *gpart, const int32_t *chunk_off,
                                                       double *e_mesh, double *gn_mesh)
{
    const int m = blockIdx.x * (THREADS / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (m >= n_mesh) return;
    double e = 0.0;
    if (tri_off)
        for (int b = tri_off[m] + lane; b < tri_off[m + 1]; b += 32) e += epart[b];
    if (hinge_off)
        for (int b = hinge_off[m] + lane; b < hinge_off[m + 1]; b += 32) e += epart[hinge_base + b];
    e = warp_sum(e);
    if (lane == 0 && e_mesh) e_mesh[m] = e;
    if (gn_mesh) {
        double q = 0.0;
        for (int c = chunk_off[m] + lane; c < chunk_off[m + 1]; c += 32) q += gpart[c];
        q = warp_sum(q);
        if (lane == 0) gn_mesh[m] = ::sqrt(q);
    }
}

// total = sum of the per-mesh energies, fixed order (one block)
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_total(int n_mesh, const double *e_mesh, double *e_total)
{
    double tot = 0.0;
    for (int m = threadIdx.x; m < n_mesh; m += THREADS) tot += e_mesh[m];
    tot = block_sum<THREADS>(tot);
    if (threadIdx.x == 0) *e_total = tot;
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

adm_status launch_reduce(adm_ctx *h, const EvalArgs &a, const int32_t *tri_off, const int32_t *hinge_off,
                         int32_t hinge_base, StageTimer &tm)
{
    const HostMesh &m = h->m;
    cudaStream_t s = a.stream;
    if (a.gnorm_per_mesh) {
        tm.begin(ADM_STAGE_GNORM);
        if (a.prec == ADM_FP32)
            k_sumsq<float, kRedThreads><<<h->chunks.n_chunks, kRedThreads, 0, s>>>(
                (const float *)a.grad, h->chunks.d_begin, h->chunks.d_end, h->d_gpart);
        else
            k_sumsq<double, kRedThreads><<<h->chunks.n_chunks, kRedThreads, 0, s>>>(
                (const double *)a.grad, h->chunks.d_begin, h->chunks.d_end, h->d_gpart);
        tm.end(ADM_STAGE_GNORM);
    }
    tm.begin(ADM_STAGE_FINALIZE);
    double *e_mesh = a.energy_per_mesh ? a.energy_per_mesh : (a.energy_total ? h->d_emesh : nullptr);
    if (e_mesh || a.gnorm_per_mesh) {
        constexpr int kSumThreads = 256;
        const int nb = (m.n_mesh + kSumThreads / 32 - 1) / (kSumThreads / 32);
        k_mesh_sums<kSumThreads><<<nb, kSumThreads, 0, s>>>(m.n_mesh, h->d_epart, tri_off, hinge_off, hinge_base,
                                                            h->d_gpart, h->chunks.d_mesh_chunk_off, e_mesh,
                                                            a.gnorm_per_mesh);
    }
    if (a.energy_total) k_total<1024><<<1, 1024, 0, s>>>(m.n_mesh, e_mesh, a.energy_total);
    tm.end(ADM_STAGE_FINALIZE);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

// ------------------------------------------------- bounded-wait check --
// One thread waits, through the bounded wait the tiled kernel uses for its
// metadata copy, on a shared-memory barrier that expects two arrivals and
// gets one: the phase never completes, so the wait must give up.
static __device__ int g_wait_result;

__global__ void k_wait_check()
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
    g_wait_result = bulk_load_wait(&bar) ? 0 : ST_TIMEOUT;
}

adm_status bounded_wait_check(cudaStream_t s)
{
    k_wait_check<<<1, 1, 0, s>>>();
    int r = -1;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&r, g_wait_result, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ADM_ERR_CUDA;
    return r == ST_TIMEOUT ? ADM_ERR_TIMEOUT : ADM_ERR_CUDA;  // a completed wait would be a defect
}

adm_status launch_eval(adm_ctx *h, const EvalArgs &a)
{
    // the matrix-free product and Hessian filtering are implemented by the tiled kernel only
    const bool tiled = a.energy != ADM_UMBRELLA && (h->assembler == 0 || a.hv || (h->proj && a.bsr) ||
                                                    a.energy == ADM_MASS_SPRING || h->inter.n_terms() > 0);
    if (a.n_split > 0 && !tiled)  // x arriving in ranges: only the tiled pass consumes them one by one
        for (int k = 0; k < a.n_split; ++k)
            if (cudaStreamWaitEvent(a.stream, a.split_ready[k], 0) != cudaSuccess) return ADM_ERR_CUDA;
    if (a.energy == ADM_UMBRELLA) return eval_ring(h, a);
    if (tiled) return a.prec == ADM_FP32 ? eval_tiled<float>(h, a) : eval_tiled<double>(h, a);
    return a.prec == ADM_FP32 ? eval_atomic<float>(h, a) : eval_atomic<double>(h, a);
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
