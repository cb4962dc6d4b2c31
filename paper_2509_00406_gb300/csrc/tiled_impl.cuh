// tiled_impl.cuh -- the tiled assembler: one block per tile of triangles and
// hinges, shared-memory staging and accumulation, row-contiguous BSR stores.
#pragma once

#include "device_common.cuh"

namespace adm {

// ----------------------------------------------------------- tiled pass --
// One block per tile: stage the footprint positions in shared memory, run
// every triangle and hinge term of the tile, accumulate gradient rows,
// diagonal blocks (upper 6) and pair blocks (9, oriented lower -> higher
// local id) with shared-memory atomics, then write every footprint row of the
// BSR with row-contiguous stores (plain for blocks only this tile touches,
// global atomic adds into pre-zeroed shared blocks).
// shared-memory strides of the accumulators, in elements: a vertex's diagonal
// block keeps its VD (VD + 1) / 2 upper entries, a pair block its VD^2, each
// padded to an odd stride (7 for 3x3 diagonals, 5 for 2x2 pairs) so that the
// same entry of different vertices or pairs maps the slot index mod 32
// one-to-one onto the 32 banks
template <int VD>
struct AccStride {
    static constexpr int D = VD == 3 ? 7 : 3;
    static constexpr int P = VD == 3 ? 9 : 5;
};

template <typename T>
struct TiledArgs {
    const int32_t *hdr;
    const uint16_t *tri_loc, *hinge_loc;
    const int32_t *foot;
    const unsigned char *meta;        // per tile: row starts, row code offsets, codes (16-byte aligned)
    const int64_t *meta_off;          // n_tiles + 1
    const T *tri_rest, *hinge_rest;   // SoA in tile order
    int64_t nT, nH;                   // SoA strides
    const T *x;
    T *grad, *bsr;
    const T *v;                       // matrix-free mode: direction
    T *hv;                            // matrix-free mode: H v
    double *epart;
    int *status;
    TermConsts<T> c;
    const float *mlp_table;           // learned membrane: 10 per triangle, tile order
    // mass-spring: per tile {edge begin, count, vertex begin, count}; per edge
    // 2 local ids + pair slot and squared rest length; per vertex its local id
    // and a third of the rest area around it; the inertial target (like x)
    const int32_t *cloth_hdr;
    const uint16_t *edge_loc, *vert_loc;
    const T *edge_l2, *vert_area3, *xhat;
};

// the element's gradient and Hessian blocks added into the footprint
// accumulators (LT: a Local in vertex DOFs or an EdgeLocal, whose entries are
// formed as they are added)
template <typename T, int VD, int NV, int NP, class LT>
__device__ __forceinline__ void tile_accumulate(const LT &L, const uint16_t (&lid)[NV], const uint16_t (&slot)[NP],
                                                const int (&pr)[NP][2], T *gacc, T *dacc, T *pacc, int mode)
{
    constexpr int NDS = AccStride<VD>::D, NPS = AccStride<VD>::P;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int d = 0; d < VD; ++d) atomicAdd(gacc + lid[a] * VD + d, local_g(L, a * VD + d));
    if (mode != MODE_HESS) return;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int s = 0; s < VD; ++s)
#pragma unroll
            for (int r = 0; r <= s; ++r)
                atomicAdd(dacc + lid[a] * NDS + hix(r, s), local_H(L, a * VD + r, a * VD + s));
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int a = pr[p][0], b = pr[p][1];
        const bool fwd = lid[a] < lid[b];
        T *dst = pacc + slot[p] * NPS;
#pragma unroll
        for (int r = 0; r < VD; ++r)
#pragma unroll
            for (int s = 0; s < VD; ++s)
                atomicAdd(dst + r * VD + s, fwd ? local_H(L, a * VD + r, b * VD + s) : local_H(L, b * VD + r, a * VD + s));
    }
}

// matrix-free mode: the element's local Hessian applied to its gathered
// part of v, added with its gradient into the footprint accumulators
template <typename T, int VD, int NV, int K>
__device__ __forceinline__ void tile_hvp(const Local<T, K> &L, const uint16_t (&lid)[NV], const T *vs, T *gacc,
                                         T *hacc)
{
    T vl[K];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int d = 0; d < VD; ++d) vl[a * VD + d] = vs[lid[a] * VD + d];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        T y = -T(0);
#pragma unroll
        for (int j = 0; j < K; ++j) y += local_H(L, i, j) * vl[j];
        atomicAdd(hacc + lid[i / VD] * VD + i % VD, y);
        atomicAdd(gacc + lid[i / VD] * VD + i % VD, L.g[i]);
    }
}

// the same in edge-vector coordinates: v_e = C^T v (per edge the signed sum
// of its vertices' v), y_e = H_e v_e, y = C y_e
template <typename T, int VD, int NV, class E>
__device__ __forceinline__ void tile_hvp(const EdgeLocal<E, VD, T> &L, const uint16_t (&lid)[NV], const T *vs,
                                         T *gacc, T *hacc)
{
    static_assert(E::NV == NV, "vertices of the edge map");
    constexpr int NE = E::NE, KE = NE * VD;
    T ve[KE], ye[KE];
#pragma unroll
    for (int p = 0; p < NE; ++p)
#pragma unroll
        for (int d = 0; d < VD; ++d) {
            T acc = -T(0);
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                if (E::C(a, p) == 0) continue;
                const T va = vs[lid[a] * VD + d];
                acc = E::C(a, p) > 0 ? acc + va : acc - va;
            }
            ve[p * VD + d] = acc;
        }
#pragma unroll
    for (int i = 0; i < KE; ++i) {
        T y = -T(0);
#pragma unroll
        for (int j = 0; j < KE; ++j) y += L.e.H[i <= j ? hix(i, j) : hix(j, i)] * ve[j];
        ye[i] = y;
    }
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int d = 0; d < VD; ++d) {
            T acc = -T(0);
#pragma unroll
            for (int p = 0; p < NE; ++p) {
                if (E::C(a, p) == 0) continue;
                acc = E::C(a, p) > 0 ? acc + ye[p * VD + d] : acc - ye[p * VD + d];
            }
            atomicAdd(hacc + lid[a] * VD + d, acc);
            atomicAdd(gacc + lid[a] * VD + d, local_g(L, a * VD + d));
        }
}

// FP32 tiles are register-capped at two resident blocks per SM (64 registers
// for 512 threads); FP64, and the Hessian-filtering variant (PROJ: an
// in-register eigensolve per element), keep one block of 256 threads and the
// full register file
template <typename T, int ENERGY, bool TRIS, bool HINGES, int MODE, int THREADS, bool PROJ = false>
__global__ void __launch_bounds__(THREADS, (sizeof(T) == 4 && !PROJ) ? 2 : 1) k_tiled(TiledArgs<T> A)
{
    constexpr int VD = TriTraits<ENERGY>::VD;
    constexpr int K = 3 * VD;
    constexpr int NB = VD * VD;
    constexpr int NDS = AccStride<VD>::D, NPS = AccStride<VD>::P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t meta_bar;
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int t = blockIdx.x;
    const int32_t *hd = A.hdr + 8 * t;
    const int32_t tri_begin = hd[0], n_tri = hd[1], hinge_begin = hd[2], n_hinge = hd[3];
    const int32_t foot_begin = hd[4], nf = hd[5], np = hd[6];
    T *xs = sm;
    T *gacc = xs + VD * nf;
    T *dacc = gacc + VD * nf;
    T *pacc = dacc + NDS * nf;
    T *vs = gacc + VD * nf;    // matrix-free mode: v of the footprint ...
    T *hacc = vs + VD * nf;    // ... and the H v accumulators (in place of dacc, pacc)
    // the tile's row metadata follows the accumulators; one thread starts
    // its bulk copy now, and it lands while the elements are evaluated
    const size_t acc_bytes = sizeof(T) * (size_t)((2 * VD + NDS) * nf + NPS * np);
    unsigned char *meta_s = smem_raw + ((acc_bytes + 15) & ~size_t(15));
    const int32_t *ms_row = reinterpret_cast<const int32_t *>(meta_s);
    const uint16_t *ms_coff = reinterpret_cast<const uint16_t *>(meta_s + 4 * nf);
    const uint16_t *ms_codes = ms_coff + nf + 1;
    if (MODE >= MODE_GRAD && threadIdx.x == 0) {
        const int64_t m0 = A.meta_off[t];
        bulk_load_start(&meta_bar, meta_s, A.meta + m0, (uint32_t)(A.meta_off[t + 1] - m0));
    }
    for (int i = threadIdx.x; i < nf; i += THREADS) {
        const int64_t v = A.foot[foot_begin + i];
#pragma unroll
        for (int d = 0; d < VD; ++d) xs[VD * i + d] = A.x[v * VD + d];
        if (MODE == MODE_HVP) {
#pragma unroll
            for (int d = 0; d < VD; ++d) {
                vs[VD * i + d] = A.v[v * VD + d];
                gacc[VD * i + d] = T(0);
                hacc[VD * i + d] = T(0);
            }
        }
    }
    if (MODE != MODE_HVP)
        for (int i = threadIdx.x; i < (VD + NDS) * nf + NPS * np; i += THREADS) gacc[i] = T(0);
    __syncthreads();
    double fe = 0.0;
    if constexpr (TRIS) {
        static constexpr int TP[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int i = threadIdx.x; i < n_tri; i += THREADS) {
            const int64_t e = (int64_t)tri_begin + i;
            uint16_t lid[3], slot[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lid[a] = A.tri_loc[6 * e + a];
                slot[a] = A.tri_loc[6 * e + 3 + a];
            }
            T x[K];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int d = 0; d < VD; ++d) x[a * VD + d] = xs[lid[a] * VD + d];
            T D[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) D[k] = A.tri_rest[k * A.nT + e];
            const T area = A.tri_rest[4 * A.nT + e];
            EdgeLocal<TriEdges, VD, T> L;
            if (!tri_term<T, ENERGY, PROJ>(x, D, area, A.c, L, A.mlp_table ? A.mlp_table + 10 * e : nullptr)) {
                atomicOr(A.status, ST_DOMAIN);
                continue;
            }
            fe += (double)local_f(L);
            if (MODE == MODE_HVP) tile_hvp<T, VD, 3>(L, lid, vs, gacc, hacc);
            else if (MODE >= MODE_GRAD) tile_accumulate<T, VD, 3, 3>(L, lid, slot, TP, gacc, dacc, pacc, MODE);
        }
    }
    if constexpr (HINGES) {
        static constexpr int HP[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
        for (int i = threadIdx.x; i < n_hinge; i += THREADS) {
            const int64_t e = (int64_t)hinge_begin + i;
            uint16_t lid[4], slot[6];
#pragma unroll
            for (int a = 0; a < 4; ++a) lid[a] = A.hinge_loc[10 * e + a];
#pragma unroll
            for (int p = 0; p < 6; ++p) slot[p] = A.hinge_loc[10 * e + 4 + p];
            T x[12];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int d = 0; d < 3; ++d) x[a * 3 + d] = xs[lid[a] * 3 + d];
            const T thetabar = A.hinge_rest[e];
            const T w = A.c.kbh2 * A.hinge_rest[A.nH + e];
            EdgeLocal<HingeEdges, 3, T> L;
            if (!(hinge_local<T, PROJ>(x, thetabar, w, L, A.c.eps) && isfinite(local_f(L)))) {
                atomicOr(A.status, ST_DOMAIN);
                continue;
            }
            fe += (double)local_f(L);
            if (MODE == MODE_HVP) tile_hvp<T, 3, 4>(L, lid, vs, gacc, hacc);
            else if (MODE >= MODE_GRAD) tile_accumulate<T, 3, 4, 6>(L, lid, slot, HP, gacc, dacc, pacc, MODE);
        }
    }
    if constexpr (ENERGY == ADM_MASS_SPRING) {
        static constexpr int EP[1][2] = {{0, 1}};
        const int32_t *ch = A.cloth_hdr + 4 * t;
        const int32_t edge_begin = ch[0], n_edge = ch[1], vert_begin = ch[2], n_vert = ch[3];
        for (int i = threadIdx.x; i < n_edge; i += THREADS) {
            const int64_t e = (int64_t)edge_begin + i;
            const uint16_t lid[2] = {A.edge_loc[3 * e], A.edge_loc[3 * e + 1]};
            const uint16_t slot[1] = {A.edge_loc[3 * e + 2]};
            T x[6];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int d = 0; d < 3; ++d) x[a * 3 + d] = xs[lid[a] * 3 + d];
            EdgeLocal<SpringEdges, 3, T> L;
            spring_local<T, PROJ>(x, A.edge_l2[e], A.c.kh2, L, A.c.eps);
            if (!isfinite(local_f(L))) {
                atomicOr(A.status, ST_DOMAIN);
                continue;
            }
            fe += (double)local_f(L);
            if (MODE == MODE_HVP) tile_hvp<T, 3, 2>(L, lid, vs, gacc, hacc);
            else if (MODE >= MODE_GRAD) tile_accumulate<T, 3, 2, 1>(L, lid, slot, EP, gacc, dacc, pacc, MODE);
        }
        for (int i = threadIdx.x; i < n_vert; i += THREADS) {
            const int64_t e = (int64_t)vert_begin + i;
            const uint16_t lid[1] = {A.vert_loc[e]};
            const int64_t v = A.foot[foot_begin + lid[0]];
            T x[3], xh[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                x[d] = xs[lid[0] * 3 + d];
                xh[d] = A.xhat[v * 3 + d];
            }
            Local<T, 3> L;
            vertex_local(x, xh, A.c.rho * A.vert_area3[e], A.c.h2, A.c.g, L);
            fe += (double)L.f;
            if (MODE == MODE_HVP) {
                tile_hvp<T, 3, 1, 3>(L, lid, vs, gacc, hacc);
            } else if (MODE >= MODE_GRAD) {
#pragma unroll
                for (int d = 0; d < 3; ++d) atomicAdd(gacc + lid[0] * 3 + d, L.g[d]);
                if (MODE == MODE_HESS)
#pragma unroll
                    for (int d = 0; d < 3; ++d) atomicAdd(dacc + lid[0] * NDS + hix(d, d), L.H[hix(d, d)]);
            }
        }
    }
    __syncthreads();
    bool meta_ok = true;
    if (MODE >= MODE_GRAD && !bulk_load_wait(&meta_bar)) {
        atomicOr(A.status, ST_TIMEOUT);
        meta_ok = false;
        bulk_load_wait(&meta_bar);  // give the copy into this block's shared memory time to land
    }
    if (MODE >= MODE_GRAD && A.grad && meta_ok) {
        for (int i = threadIdx.x; i < nf; i += THREADS) {
            const int32_t rs = ms_row[i];
            const int64_t v = A.foot[foot_begin + i];
#pragma unroll
            for (int d = 0; d < VD; ++d) {
                const T val = gacc[VD * i + d];
                if (rs < 0) atomicAdd(A.grad + v * VD + d, val);
                else A.grad[v * VD + d] = val;
            }
        }
    }
    if (MODE == MODE_HVP && meta_ok) {  // H v rows: shared exactly where gradient rows are
        for (int i = threadIdx.x; i < nf; i += THREADS) {
            const int32_t rs = ms_row[i];
            const int64_t v = A.foot[foot_begin + i];
#pragma unroll
            for (int d = 0; d < VD; ++d) {
                const T val = hacc[VD * i + d];
                if (rs < 0) atomicAdd(A.hv + v * VD + d, val);
                else A.hv[v * VD + d] = val;
            }
        }
    }
    if (MODE == MODE_HESS && meta_ok) {
        // one warp per footprint row: the row's blocks are contiguous in the
        // BSR and its codes say, per block, where the tile's sum is (none,
        // the vertex's diagonal, a pair block or its transpose) and whether
        // other tiles add into the same block.  A warp iteration writes BPI
        // consecutive blocks; lane = sub * NB + k takes entry k of block sub,
        // so the lane's offsets into the three source layouts are fixed.
        constexpr int BPI = 32 / NB;
        constexpr uint64_t DTAB = VD == 3 ? 0x543421310ull : 0x2110ull;  // (r,s) -> packed upper
        constexpr uint64_t TTAB = VD == 3 ? 0x852741630ull : 0x3120ull;  // (r,s) -> (s,r)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int sub = lane / NB, k = lane - sub * NB;
        const bool active = sub < BPI;
        const int off_d = (int)((DTAB >> (4 * k)) & 0xf), off_t = (int)((TTAB >> (4 * k)) & 0xf);
        for (int r = warp; r < nf; r += THREADS / 32) {
            const int64_t rs = ms_row[r] & 0x7fffffff;
            const int c0 = ms_coff[r], nb = ms_coff[r + 1] - c0;
            T *out = A.bsr + rs * NB + lane;
            if (!active) continue;
            for (int e = sub; e < nb; e += BPI) {
                const uint32_t code = ms_codes[c0 + e];
                const uint32_t kind = code >> 14;
                if (kind == 0) continue;
                const int slot = (int)(code & 0x1fffu);
                const T *src = kind == 1 ? dacc + r * NDS + off_d : pacc + slot * NPS + (kind == 2 ? k : off_t);
                const T val = *src;
                T *dst = out + (e - sub) * NB;
                if (code & 0x2000u) atomicAdd(dst, val);
                else *dst = val;
            }
        }
    }
    const double sum = block_sum<THREADS>(fe);
    if (threadIdx.x == 0) A.epart[t] = sum;
}

// zero the blocks and gradient (and H v) rows that several tiles add into
template <typename T, int VD>
__global__ void k_zero_shared(const int32_t *blocks, int64_t nb, const int32_t *verts, int64_t nv, T *bsr,
                              T *grad, T *hv)
{
    constexpr int NB = VD * VD;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bsr)
        for (int64_t i = i0; i < nb * NB; i += stride) bsr[(int64_t)blocks[i / NB] * NB + i % NB] = T(0);
    if (grad)
        for (int64_t i = i0; i < nv * VD; i += stride) grad[(int64_t)verts[i / VD] * VD + i % VD] = T(0);
    if (hv)
        for (int64_t i = i0; i < nv * VD; i += stride) hv[(int64_t)verts[i / VD] * VD + i % VD] = T(0);
}

// Launch of one (precision, mode, filtering) variant for any energy.  Each
// variant is instantiated in its own translation unit (tiled_inst.cu) so
// that they compile in parallel.
template <typename T, int MODE, bool PROJ>
void launch_tiled_mode(int energy, int n_tiles, size_t smem, cudaStream_t s, const TiledArgs<T> &A)
{
    constexpr int TT = tile_threads<T, PROJ>();
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<n_tiles, TT, smem, s>>>(A);
    };
    switch (energy) {
    case ADM_SYMDIR2D: go(k_tiled<T, ADM_SYMDIR2D, true, false, MODE, TT, PROJ>); break;
    case ADM_STVK_MEMBRANE: go(k_tiled<T, ADM_STVK_MEMBRANE, true, false, MODE, TT, PROJ>); break;
    case ADM_NH_MEMBRANE: go(k_tiled<T, ADM_NH_MEMBRANE, true, false, MODE, TT, PROJ>); break;
    case ADM_AREA: go(k_tiled<T, ADM_AREA, true, false, MODE, TT, PROJ>); break;
    case ADM_MLP_MEMBRANE:
        if constexpr (sizeof(T) == 4) go(k_tiled<T, ADM_MLP_MEMBRANE, true, false, MODE, TT, PROJ>);
        break;
    case ADM_SHELL: go(k_tiled<T, ADM_SHELL, true, true, MODE, TT, PROJ>); break;
    case ADM_HINGE_BENDING: go(k_tiled<T, ADM_STVK_MEMBRANE, false, true, MODE, TT, PROJ>); break;
    case ADM_MASS_SPRING: go(k_tiled<T, ADM_MASS_SPRING, false, false, MODE, TT, PROJ>); break;
    default: break;
    }
}

#define ADM_TILED_VARIANTS(X, T)                                                                          \
    X(T, MODE_VALUE, false) X(T, MODE_GRAD, false) X(T, MODE_HESS, false) X(T, MODE_HESS, true)           \
    X(T, MODE_HVP, false) X(T, MODE_HVP, true)
#define ADM_TILED_EXTERN(T, M, P)                                                                          \
    extern template void launch_tiled_mode<T, M, P>(int, int, size_t, cudaStream_t, const TiledArgs<T> &);
#define ADM_TILED_INST(T, M, P) \
    template void launch_tiled_mode<T, M, P>(int, int, size_t, cudaStream_t, const TiledArgs<T> &);

template <typename T>
static void launch_tiled(int energy, int mode, bool proj, int n_tiles, size_t smem, cudaStream_t s,
                         const TiledArgs<T> &A)
{
    if (mode == MODE_VALUE) launch_tiled_mode<T, MODE_VALUE, false>(energy, n_tiles, smem, s, A);
    else if (mode == MODE_GRAD) launch_tiled_mode<T, MODE_GRAD, false>(energy, n_tiles, smem, s, A);
    else if (mode == MODE_HESS && !proj) launch_tiled_mode<T, MODE_HESS, false>(energy, n_tiles, smem, s, A);
    else if (mode == MODE_HESS) launch_tiled_mode<T, MODE_HESS, true>(energy, n_tiles, smem, s, A);
    else if (!proj) launch_tiled_mode<T, MODE_HVP, false>(energy, n_tiles, smem, s, A);
    else launch_tiled_mode<T, MODE_HVP, true>(energy, n_tiles, smem, s, A);
}

template <typename T>
adm_status eval_tiled(adm_ctx *h, const EvalArgs &a)
{
    const HostMesh &m = h->m;
    const int vd = m.vdim;
    const bool hin = has_hinges(a.energy);
    const TileSet &ts = h->tiles[hin ? PAT_SHELL : PAT_TRI];
    const int mode = a.hv ? MODE_HVP : (a.bsr ? MODE_HESS : (a.grad ? MODE_GRAD : MODE_VALUE));
    const size_t smem = (size_t)ts.smem_bytes[vd == 3][sizeof(T) == 4 ? ADM_FP32 : ADM_FP64];
    if (smem > 227 * 1024) return ADM_ERR_UNSUPPORTED;
    cudaStream_t s = a.stream;
    StageTimer tm(h, s);
    const bool pairs = h->inter.kind == (hin ? PAT_SHELL : PAT_TRI) && h->inter.n_terms() > 0;
    if (cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return ADM_ERR_CUDA;
    const bool with_bsr = a.bsr != nullptr, with_rows = a.grad || a.hv;
    // zero the shared outputs listed in [zb0, zb1) and [zv0, zv1)
    auto zero_range = [&](int64_t zb0, int64_t zb1, int64_t zv0, int64_t zv1, cudaStream_t zs) {
        const int64_t nzb = with_bsr ? zb1 - zb0 : 0, nzv = with_rows ? zv1 - zv0 : 0;
        if (nzb + nzv == 0) return;
        const int64_t work = std::max(nzb * vd * vd, nzv * vd);
        const int blocks = (int)std::min<int64_t>((work + 255) / 256, 152 * 8);
        if (vd == 3)
            k_zero_shared<T, 3><<<blocks, 256, 0, zs>>>(ts.d_zero_blocks + zb0, nzb, ts.d_zero_verts + zv0, nzv,
                                                         (T *)a.bsr, (T *)a.grad, (T *)a.hv);
        else
            k_zero_shared<T, 2><<<blocks, 256, 0, zs>>>(ts.d_zero_blocks + zb0, nzb, ts.d_zero_verts + zv0, nzv,
                                                         (T *)a.bsr, (T *)a.grad, (T *)a.hv);
    };
    const bool split = a.n_split > 0 && a.split_mesh && a.split_ready && !pairs && a.energy != ADM_MLP_MEMBRANE &&
                       h->split_stream[0] && h->split_stream[1] && h->split_start &&
                       (int)h->split_done.size() >= a.n_split;
    if (a.n_split > 0 && !split)  // x arriving in ranges, consumed whole here: wait for all of them
        for (int k = 0; k < a.n_split; ++k)
            if (cudaStreamWaitEvent(s, a.split_ready[k], 0) != cudaSuccess) return ADM_ERR_CUDA;
    if (!split) {
        tm.begin(ADM_STAGE_ZERO);
        zero_range(0, (int64_t)ts.zero_blocks.size(), 0, (int64_t)ts.zero_verts.size(), s);
        tm.end(ADM_STAGE_ZERO);
    }
    TiledArgs<T> A;
    A.hdr = ts.d_hdr;
    A.tri_loc = ts.d_tri_loc;
    A.hinge_loc = ts.d_hinge_loc;
    A.foot = ts.d_foot;
    A.meta = ts.d_meta;
    A.meta_off = ts.d_meta_off;
    A.tri_rest = (const T *)ts.d_tri_rest[a.prec];
    A.hinge_rest = (const T *)ts.d_hinge_rest[a.prec];
    A.nT = m.nT;
    A.nH = hin ? m.nH() : 0;
    A.x = (const T *)a.x;
    A.grad = (T *)a.grad;
    A.bsr = (T *)a.bsr;
    A.v = (const T *)a.v;
    A.hv = (T *)a.hv;
    A.epart = h->d_epart;
    A.status = h->d_status;
    A.c = consts<T>(h, a.energy);
    A.mlp_table = nullptr;
    A.cloth_hdr = ts.d_cloth_hdr;
    A.edge_loc = ts.d_edge_loc;
    A.vert_loc = ts.d_vert_loc;
    A.edge_l2 = (const T *)ts.d_edge_l2[a.prec];
    A.vert_area3 = (const T *)ts.d_vert_area3[a.prec];
    A.xhat = (const T *)h->d_xhat[a.prec];
    if (a.energy == ADM_MASS_SPRING && (!ts.cloth_built || !A.xhat)) return ADM_ERR_UNSUPPORTED;
    if (a.energy == ADM_MLP_MEMBRANE) {
        if (sizeof(T) != 4 || !h->d_mlp_theta || !ts.d_tri_perm) return ADM_ERR_UNSUPPORTED;
        tm.begin(ADM_STAGE_MLP);
        adm_status st = mlp_triangle_table(h->d_mlp_theta, h->d_mlp_norm, m.nT, ts.d_tri_perm, h->d_F,
                                           (const float *)ts.d_tri_rest[ADM_FP32], (const float *)a.x,
                                           h->d_mlp_table, s);
        tm.end(ADM_STAGE_MLP);
        if (st != ADM_OK) return st;
        A.mlp_table = h->d_mlp_table;
    }
    // tiles [t0, t1): the kernel indexes its per-tile arrays by block, so a
    // range is a launch over offset pointers
    auto tiled_range = [&](int32_t t0, int32_t t1, cudaStream_t ks) {
        if (t1 <= t0) return;
        TiledArgs<T> B = A;
        B.hdr += 8 * (int64_t)t0;
        B.meta_off += t0;
        B.epart += t0;
        if (B.cloth_hdr) B.cloth_hdr += 4 * (int64_t)t0;
        launch_tiled<T>(a.energy, mode, h->proj != 0, t1 - t0, smem, ks, B);
    };
    tm.begin(ADM_STAGE_TILED);
    if (!split) {
        tiled_range(0, ts.n_tiles, s);
    } else {
        // per mesh range, on two streams in turn: wait for its x, zero its
        // shared outputs (they lie in its own rows) and run its tiles.  The
        // copies of later ranges overlap the kernels of earlier ones, and a
        // range's launch overlaps the tail of the one before; the pass's
        // stream resumes when every range is done.
        const Pattern &P = h->pat[hin ? PAT_SHELL : PAT_TRI];
        auto lb = [](const std::vector<int32_t> &v, int64_t key) {
            return (int64_t)(std::lower_bound(v.begin(), v.end(), (int32_t)key) - v.begin());
        };
        if (cudaEventRecord(h->split_start, s) != cudaSuccess) return ADM_ERR_CUDA;
        for (int k = 0; k < a.n_split; ++k) {
            cudaStream_t ks = h->split_stream[k & 1];
            const int32_t m0 = a.split_mesh[k], m1 = a.split_mesh[k + 1];
            const int64_t v0 = m.v_off[m0], v1 = m.v_off[m1];
            if (cudaStreamWaitEvent(ks, h->split_start, 0) != cudaSuccess ||
                cudaStreamWaitEvent(ks, a.split_ready[k], 0) != cudaSuccess)
                return ADM_ERR_CUDA;
            zero_range(lb(ts.zero_blocks, P.row_ptr[v0]), lb(ts.zero_blocks, P.row_ptr[v1]), lb(ts.zero_verts, v0),
                       lb(ts.zero_verts, v1), ks);
            tiled_range(ts.mesh_tile_off[m0], ts.mesh_tile_off[m1], ks);
            if (cudaEventRecord(h->split_done[k], ks) != cudaSuccess) return ADM_ERR_CUDA;
        }
        for (int k = 0; k < a.n_split; ++k)
            if (cudaStreamWaitEvent(s, h->split_done[k], 0) != cudaSuccess) return ADM_ERR_CUDA;
    }
    tm.end(ADM_STAGE_TILED);
    if (cudaGetLastError() != cudaSuccess) return ADM_ERR_CUDA;
    if (pairs) {
        tm.begin(ADM_STAGE_PAIRS);
        adm_status st = interactions_eval(h, a, mode);
        tm.end(ADM_STAGE_PAIRS);
        if (st != ADM_OK) return st;
    }
    adm_status st = launch_reduce(h, a, ts.d_mesh_tile_off, nullptr, 0, tm);
    if (st != ADM_OK || !pairs) return st;
    return interactions_energy(h, a);
}

}  // namespace adm
