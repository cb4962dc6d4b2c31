// tiled_impl.cuh -- the staged-gather assembler: a persistent grid whose
// blocks take tiles of units (a triangle and its attached hinges or springs)
// from a queue, evaluate them with per-element forward mode, stage every
// contribution in shared memory sorted by the output it adds to, and write
// each BSR entry, gradient and H v entry as the fixed-order sum of one
// contiguous segment.  No float atomics anywhere, and no tile waits for
// another: an output that several tiles produce is stored by the
// lowest-index one, the others store their parts in partial slots, and a
// fix-up kernel adds the slots in tile order, so two passes on the same
// input give bit-identical results.
#pragma once

#include <climits>
#include <type_traits>

#include "device_common.cuh"

namespace adm {

template <typename T>
struct TiledArgs {
    const int32_t *hdr;               // kHdr per tile
    const uint16_t *unit;             // 8 per unit
    const uint16_t *unit_dst;         // 6 per unit
    const uint16_t *slot_dst;         // 4 per slot
    const int32_t *foot;
    const unsigned char *meta;        // per tile blob (16-byte aligned)
    const int64_t *meta_off;          // n_tiles + 1
    const T *tri_rest;                // SoA 5 x nU, unit order (rotated triangles)
    const T *slot_rest;               // SoA 2 x nS
    const T *vterm_rest;              // cloth vertex terms
    int64_t nU, nS;
    const T *x;
    T *grad, *bsr;
    const T *v;                       // matrix-free mode: direction
    T *hv;                            // matrix-free mode: H v
    int32_t *next;                    // work queue position of this launch
    T *vpart, *ppart;                 // partial slots of shared outputs: Chunk<MODE_HESS, VD>::V, VD^2 each
    int32_t tile_begin, tile_end;     // this launch's tiles
    int32_t nf_cap;                   // largest footprint of the tile set (rows of the x region)
    double *epart;                    // per tile
    int *status;
    TermConsts<T> c;
    const float *mlp_table;           // learned membrane: 10 per unit
    const T *xhat;                    // cloth inertial target
    const T *loc_tri, *loc_slot;      // filtered passes: the terms' filtered results (SoA)
};

// floats of a vertex and of a pair chunk
template <int MODE, int VD>
struct Chunk {
    static constexpr int V = MODE == MODE_HESS ? VD + VD * (VD + 1) / 2 : (MODE == MODE_HVP ? 2 * VD : (MODE == MODE_GRAD ? VD : 0));
    static constexpr int P = MODE == MODE_HESS ? VD * VD : 0;
};

template <typename U>
__device__ __forceinline__ U sel3(int k, U a, U b, U c) { return k == 0 ? a : (k == 1 ? b : c); }

// ------------------------------------------------------- chunk writers --
// vertex a of an element's local result into a vertex chunk: gradient, then
// (Hessian mode) the upper entries of its diagonal block; ADD adds into what
// the chunk holds (the unit's own chunk), otherwise stores
template <int MODE, int VD, int A, bool ADD, typename T, class LT>
__device__ __forceinline__ void put_vertex(const LT &L, T *ch)
{
#pragma unroll
    for (int d = 0; d < VD; ++d) {
        const T g = local_g(L, A * VD + d);
        if (ADD) ch[d] += g;
        else ch[d] = g;
    }
    if constexpr (MODE == MODE_HESS) {
#pragma unroll
        for (int s = 0; s < VD; ++s)
#pragma unroll
            for (int r = 0; r <= s; ++r) {
                const T h = local_H(L, A * VD + r, A * VD + s);
                if (ADD) ch[VD + hix(r, s)] += h;
                else ch[VD + hix(r, s)] = h;
            }
    }
}

// the block of element vertices (A, B) into a pair chunk, oriented from the
// lower to the higher footprint index (tr: B's is the lower)
template <int VD, int A, int B, bool ADD, typename T, class LT>
__device__ __forceinline__ void put_pair(const LT &L, T *ch, bool tr)
{
    T v[VD][VD];
#pragma unroll
    for (int r = 0; r < VD; ++r)
#pragma unroll
        for (int s = 0; s < VD; ++s) v[r][s] = local_H(L, A * VD + r, B * VD + s);
#pragma unroll
    for (int r = 0; r < VD; ++r)
#pragma unroll
        for (int s = 0; s < VD; ++s) {
            const T val = tr ? v[s][r] : v[r][s];
            if (ADD) ch[r * VD + s] += val;
            else ch[r * VD + s] = val;
        }
}

// matrix-free mode: y = H_e v_e of an element in edge coordinates
// (v_e = C^T v, y = C y_e), gradient and y per vertex into vertex chunks
template <int VD, class E, typename T>
__device__ __forceinline__ void hvp_edge(const EdgeLocal<E, VD, T> &L, const T (&vl)[E::NV * VD], T (&y)[E::NV * VD])
{
    constexpr int NE = E::NE, NV = E::NV, KE = NE * VD;
    T ve[KE], ye[KE];
#pragma unroll
    for (int p = 0; p < NE; ++p)
#pragma unroll
        for (int d = 0; d < VD; ++d) {
            T acc = -T(0);
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                if (E::C(a, p) == 0) continue;
                acc = E::C(a, p) > 0 ? acc + vl[a * VD + d] : acc - vl[a * VD + d];
            }
            ve[p * VD + d] = acc;
        }
#pragma unroll
    for (int i = 0; i < KE; ++i) {
        T acc = -T(0);
#pragma unroll
        for (int j = 0; j < KE; ++j) acc += L.e.H[i <= j ? hix(i, j) : hix(j, i)] * ve[j];
        ye[i] = acc;
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
            y[a * VD + d] = acc;
        }
}

template <int VD, int A, bool ADD, typename T, class LT>
__device__ __forceinline__ void put_vertex_hvp(const LT &L, const T *y, T *ch)
{
#pragma unroll
    for (int d = 0; d < VD; ++d) {
        const T g = local_g(L, A * VD + d), hy = y[A * VD + d];
        if (ADD) {
            ch[d] += g;
            ch[VD + d] += hy;
        } else {
            ch[d] = g;
            ch[VD + d] = hy;
        }
    }
}

// the element's contributions for vertices (A) / pairs (A, B) into chunks
// given by pointer arrays; a whole element at once
template <int MODE, int VD, int NV, bool ADD, typename T, class LT>
__device__ __forceinline__ void put_vertices(const LT &L, T *const (&vch)[NV], const T *y)
{
    sfor<0, NV>([&](auto Ai) {
        constexpr int A = decltype(Ai)::value;
        if constexpr (MODE == MODE_HVP) put_vertex_hvp<VD, A, ADD>(L, y, vch[A]);
        else put_vertex<MODE, VD, A, ADD>(L, vch[A]);
    });
}

// ------------------------------------------------------- row stores --
// store N consecutive reals from registers to global memory whose start is
// aligned to one real: in aligned pairs where the run allows (a 3x3 FP32
// block at 36 b bytes takes one single and four pair stores instead of
// nine single ones, whichever parity b has)
template <int N, typename T>
__device__ __forceinline__ void store_run(T *dst, const T *v)
{
    using V2 = std::conditional_t<sizeof(T) == 4, float2, double2>;
    if constexpr (N == 1) {
        dst[0] = v[0];
    } else if constexpr (N > 1) {
        const bool odd = ((reinterpret_cast<uintptr_t>(dst) / sizeof(T)) & 1u) != 0;
        if constexpr (N % 2 == 1) {
            // odd start: the first real alone, then pairs; even start: pairs,
            // then the last real alone
            dst[odd ? 0 : N - 1] = odd ? v[0] : v[N - 1];
            V2 *p = reinterpret_cast<V2 *>(dst + (odd ? 1 : 0));
#pragma unroll
            for (int j = 0; j < (N - 1) / 2; ++j) {
                V2 w;
                w.x = odd ? v[2 * j + 1] : v[2 * j];
                w.y = odd ? v[2 * j + 2] : v[2 * j + 1];
                p[j] = w;
            }
        } else if (!odd) {
            V2 *p = reinterpret_cast<V2 *>(dst);
#pragma unroll
            for (int j = 0; j < N / 2; ++j) {
                V2 w;
                w.x = v[2 * j];
                w.y = v[2 * j + 1];
                p[j] = w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) dst[j] = v[j];
        }
    }
}

// one real global -> shared without passing through registers (cp.async);
// the copies of a thread are complete after cp_async_wait_all
template <typename T>
__device__ __forceinline__ void cp_async_real(T *dst, const T *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// L2 prefetch (bulk, one thread) of the 16-byte aligned part of
// [p, p + bytes): the start is rounded up and the end down, so nothing
// outside the range is touched
__device__ __forceinline__ void l2_prefetch(const void *p, int64_t bytes)
{
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + (uintptr_t)bytes) & ~uintptr_t(15);
    if (bytes > 0 && e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// ------------------------------------------------------------ waits --
__device__ __forceinline__ void bar_init(uint64_t *bar)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one thread: arm the barrier with the byte count and start the bulk copy
// (dst, src, bytes multiples of 16); generic-proxy reads of dst by the
// previous tile are ordered before the async-proxy writes
__device__ __forceinline__ void bulk_copy_start(uint64_t *bar, void *dst, const void *src, uint32_t bytes)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// wait for the barrier phase of the given parity; gives up after about a
// second (2^20 waits of at most ~1 us) and returns false
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(parity), "r"(1000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------ filtered terms --
// Filtered passes: each term's filtered edge-coordinate result (energy,
// gradient, packed Hessian), one thread per term, into structure-of-arrays
// buffers that k_tiled then reads in place of evaluating the terms.  The
// filter's eigensolve is the expensive part; here it runs one term per
// thread with no shared memory and no barriers.  A term outside the
// energy's domain stores a NaN energy, which k_tiled reports.
template <typename T>
struct LocalArgs {
    int64_t nU, nS;
    const int32_t *tri_verts;         // 3 per unit
    const int4 *slot_verts;           // per slot: t_k, t_k+1, t_k+2, extra (-1: none)
    const T *tri_rest, *slot_rest;    // SoA, as k_tiled reads them
    const T *x;
    const float *mlp_table;           // learned membrane: 10 per unit
    T *loc_tri, *loc_slot;
    TermConsts<T> c;
};

// store / load one Local of K edge coordinates at index i of a
// structure-of-arrays buffer of n entries
template <int K, typename T>
__device__ __forceinline__ void store_local_soa(const Local<T, K> &e, T *buf, int64_t i, int64_t n, bool ok)
{
    buf[i] = ok ? e.f : T(NAN);
#pragma unroll
    for (int k = 0; k < K; ++k) buf[(1 + k) * n + i] = e.g[k];
#pragma unroll
    for (int k = 0; k < K * (K + 1) / 2; ++k) buf[(1 + K + k) * n + i] = e.H[k];
}
template <int K, typename T>
__device__ __forceinline__ void load_local_soa(Local<T, K> &e, const T *buf, int64_t i, int64_t n)
{
    e.f = buf[i];
#pragma unroll
    for (int k = 0; k < K; ++k) e.g[k] = buf[(1 + k) * n + i];
#pragma unroll
    for (int k = 0; k < K * (K + 1) / 2; ++k) e.H[k] = buf[(1 + K + k) * n + i];
}

template <typename T, int ENERGY>
__global__ void __launch_bounds__(128) k_filtered_tris(LocalArgs<T> A)
{
    constexpr int VD = TriTraits<ENERGY>::VD;
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= A.nU) return;
    T x[3 * VD];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int64_t v = A.tri_verts[3 * u + q];
#pragma unroll
        for (int d = 0; d < VD; ++d) x[q * VD + d] = A.x[v * VD + d];
    }
    T D[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) D[k] = A.tri_rest[k * A.nU + u];
    const T area = A.tri_rest[4 * A.nU + u];
    EdgeLocal<TriEdges, VD, T> L;
    const bool ok = tri_term<T, ENERGY, true>(x, D, area, A.c, L, A.mlp_table ? A.mlp_table + 10 * u : nullptr);
    store_local_soa(L.e, A.loc_tri, u, A.nU, ok);
}

// slots: hinges (ENERGY != ADM_MASS_SPRING) or springs.  Blocks of 256,
// two per SM: the 9x9 eigensolve then runs at 128 registers with part of
// its eigenvectors spilled to L1-resident local memory, 16 warps per SM;
// unbounded it takes 240 registers and runs 8 warps, 17 % slower on the
// shell batch
template <typename T, int ENERGY>
__global__ void __launch_bounds__(256, 2) k_filtered_slots(LocalArgs<T> A)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.nS) return;
    const int4 v = A.slot_verts[s];
    const int32_t vv[4] = {v.x, v.y, v.z, v.w};
    if constexpr (ENERGY == ADM_MASS_SPRING) {
        T x[6];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int d = 0; d < 3; ++d) x[q * 3 + d] = A.x[(int64_t)vv[q] * 3 + d];
        EdgeLocal<SpringEdges, 3, T> L;
        spring_local<T, true>(x, A.slot_rest[s], A.c.kh2, L, A.c.eps);
        store_local_soa(L.e, A.loc_slot, s, A.nS, isfinite(local_f(L)));
    } else {
        if (v.w < 0) return;  // no hinge on this slot's edge
        T x[12];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int d = 0; d < 3; ++d) x[q * 3 + d] = A.x[(int64_t)vv[q] * 3 + d];
        const T thetabar = A.slot_rest[s];
        const T w = A.c.kbh2 * A.slot_rest[A.nS + s];
        EdgeLocal<HingeEdges, 3, T> L;
        const bool ok = hinge_local<T, true>(x, thetabar, w, L, A.c.eps) && isfinite(local_f(L));
        store_local_soa(L.e, A.loc_slot, s, A.nS, ok);
    }
}

// ------------------------------------------------------------- kernel --
// resident blocks per SM the register budget is sized for: FP32 tiles run
// 512 threads per SM at 128 registers (two blocks of 256 or four of 128);
// FP64 tiles one block of 256 with the full register file.  Filtered tiles
// read their terms' filtered results (k_filtered_tris, k_filtered_slots), so
// they have the budget of plain ones.
template <typename T, bool PROJ, int THREADS>
constexpr int tile_min_blocks() { return sizeof(T) == 4 ? 512 / THREADS : 1; }

template <typename T, int ENERGY, bool TRIS, bool HINGES, int MODE, int THREADS, bool PROJ>
__global__ void __launch_bounds__(THREADS, (tile_min_blocks<T, PROJ, THREADS>())) k_tiled(TiledArgs<T> A)
{
    constexpr int VD = TriTraits<ENERGY>::VD;
    constexpr int CV = Chunk<MODE, VD>::V, CP = Chunk<MODE, VD>::P;
    constexpr bool CLOTH = ENERGY == ADM_MASS_SPRING;
    constexpr int NW = THREADS / 32;
    constexpr int KR = (kMaxFootRows + THREADS - 1) / THREADS;  // footprint rows a thread stages
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t meta_bar;
    __shared__ int s_next;
    __shared__ double s_red[NW];
    // header and metadata span of the current tile and of the next one
    // (double buffered by tile parity), written by the control thread
    __shared__ int32_t s_hdr[2][kHdr];
    __shared__ int64_t s_moff[2][2];
    const int tid = threadIdx.x;
    // the control thread: the block's last thread, whose warp has no unit
    // to evaluate unless the tile fills the block
    constexpr int CTL = THREADS - 1;
    // x (and v) of the footprint sit in a region of fixed size, below every
    // tile's chunks, so the next tile's rows land there while the current
    // tile's chunks are summed
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *vsm = reinterpret_cast<T *>(smem_raw + tile_layout(A.nf_cap, 0, 0, 0, MODE, VD, (int)sizeof(T)).off_vs);
    // x (and v) rows of a tile into the fixed region: cp.async, no registers;
    // completed by cp_async_wait_all before the barrier that opens the tile
    auto stage_rows = [&](const int32_t *hd, const int32_t (&fv)[KR]) {
        const int nf = hd[kHdrNF];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int i = tid + k * THREADS;
            if (i >= nf) break;
            const int64_t v = fv[k];
#pragma unroll
            for (int d = 0; d < VD; ++d) cp_async_real(xs + VD * i + d, A.x + v * VD + d);
            if constexpr (MODE == MODE_HVP)
#pragma unroll
                for (int d = 0; d < VD; ++d) cp_async_real(vsm + VD * i + d, A.v + v * VD + d);
        }
    };
    auto foot_rows = [&](const int32_t *hd, int32_t (&fv)[KR]) {
        const int fb = hd[kHdrFoot], nf = hd[kHdrNF];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int i = tid + k * THREADS;
            fv[k] = i < nf ? A.foot[fb + i] : 0;
        }
    };
    // control thread: the header and metadata span of tile t into buffer b,
    // and an L2 prefetch of what the tile's evaluation and staging read
    auto fetch_tile = [&](int t, int b) {
        const int32_t *g = A.hdr + kHdr * (int64_t)t;
#pragma unroll
        for (int k = 0; k < kHdr; ++k) s_hdr[b][k] = g[k];
        const int64_t m0 = A.meta_off[t], m1 = A.meta_off[t + 1];
        s_moff[b][0] = m0;
        s_moff[b][1] = m1;
        const int64_t u0 = g[kHdrUnit], nu = g[kHdrNUnit], sl0 = g[kHdrSlot], ns = g[kHdrNSlot];
        l2_prefetch(A.unit + 8 * u0, nu * 16);
        l2_prefetch(A.unit_dst + 6 * u0, nu * 12);
        if constexpr (TRIS && !PROJ) {
            if (A.mlp_table) l2_prefetch(A.mlp_table + 10 * u0, nu * 40);
#pragma unroll
            for (int k = 0; k < 5; ++k) l2_prefetch(A.tri_rest + k * A.nU + u0, nu * (int64_t)sizeof(T));
        }
        if constexpr (HINGES || CLOTH) {
            l2_prefetch(A.slot_dst + 4 * sl0, ns * 8);
            if constexpr (!PROJ) {
                l2_prefetch(A.slot_rest + sl0, ns * (int64_t)sizeof(T));
                if constexpr (HINGES) l2_prefetch(A.slot_rest + A.nS + sl0, ns * (int64_t)sizeof(T));
            }
        }
        l2_prefetch(A.foot + g[kHdrFoot], (int64_t)g[kHdrNF] * 4);
        if constexpr (MODE >= MODE_GRAD) l2_prefetch(A.meta + m0, m1 - m0);
    };
    if (tid == CTL) {
        if (MODE >= MODE_GRAD) bar_init(&meta_bar);
        const int t0 = A.tile_begin + atomicAdd(A.next, 1);
        s_next = t0;
        if (t0 < A.tile_end) fetch_tile(t0, 0);
    }
    __syncthreads();
    uint32_t phase = 0;
    int p = 0;  // header buffer of the current tile
    // every queue position taken is bounded by the tile count + 1; a block
    // that takes that many without the queue running dry reports a timeout
    const int32_t cap = A.tile_end - A.tile_begin + 1;
    int32_t taken = 1;
    int t = s_next;
    if (t < A.tile_end) {
        int32_t fv[KR];
        foot_rows(s_hdr[0], fv);
        stage_rows(s_hdr[0], fv);
        cp_async_wait_all();
    }
    while (t < A.tile_end) {
        // x of tile t is staged; the previous tile's chunks, blob and
        // partial energies are no longer read
        __syncthreads();
        const int32_t *hd = s_hdr[p];
        const int32_t u0 = hd[kHdrUnit], nu = hd[kHdrNUnit], slot0 = hd[kHdrSlot];
        const int32_t fb = hd[kHdrFoot], nf = hd[kHdrNF];
        const int64_t m0 = s_moff[p][0];
        const int32_t meta_bytes = (int32_t)(s_moff[p][1] - m0);
        const TileLayout lay = tile_layout(A.nf_cap, hd[kHdrNVC], hd[kHdrNPC], meta_bytes, MODE, VD, (int)sizeof(T));
        T *sv = reinterpret_cast<T *>(smem_raw + lay.off_sv);
        T *sp = reinterpret_cast<T *>(smem_raw + lay.off_sp);
        unsigned char *blob = smem_raw + lay.off_blob;
        if (tid == CTL) {
            if (MODE >= MODE_GRAD) bulk_copy_start(&meta_bar, blob, A.meta + m0, (uint32_t)meta_bytes);
            const int tn = taken < cap ? A.tile_begin + atomicAdd(A.next, 1) : INT_MAX;
            s_next = tn;
            if (tn < A.tile_end) fetch_tile(tn, p ^ 1);
        }

        // ---- units: evaluate, stage contributions in their chunks
        double fe = 0.0;
        for (int ul = tid; ul < nu; ul += THREADS) {
            const int64_t u = (int64_t)u0 + ul;
            const uint4 rec = *reinterpret_cast<const uint4 *>(A.unit + 8 * u);
            const int l[3] = {(int)(rec.x & 0xffffu), (int)(rec.x >> 16), (int)(rec.y & 0xffffu)};
            const int ex[3] = {(int)(rec.y >> 16), (int)(rec.z & 0xffffu), (int)(rec.z >> 16)};
            const int flags = (int)(rec.w & 0xffffu), ufirst = (int)(rec.w >> 16);
            const int nslot = flags & 3, rot = (flags >> 5) & 3;
            const uint16_t *ud = A.unit_dst + 6 * u;
            T *vch[3] = {nullptr, nullptr, nullptr}, *pch[3] = {nullptr, nullptr, nullptr};
            if constexpr (MODE >= MODE_GRAD) {
#pragma unroll
                for (int q = 0; q < 3; ++q) vch[q] = sv + CV * (int)ud[q];
                if constexpr (CP > 0)
#pragma unroll
                    for (int q = 0; q < 3; ++q) pch[q] = sp + CP * (int)ud[3 + q];
            }
            const bool tr01 = l[0] > l[1], tr02 = l[0] > l[2], tr12 = l[1] > l[2];
            T yv[3 * VD];  // matrix-free: the element's H v per vertex
            // -- the triangle term (stores every unit chunk first), or zeros
            bool wrote = false;
            if constexpr (TRIS) {
                T x[3 * VD];
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int d = 0; d < VD; ++d) x[q * VD + d] = xs[l[q] * VD + d];
                T D[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) D[k] = A.tri_rest[k * A.nU + u];
                const T area = A.tri_rest[4 * A.nU + u];
                EdgeLocal<TriEdges, VD, T> L;
                bool ok;
                if constexpr (PROJ) {  // the filtered result of k_filtered_tris
                    load_local_soa(L.e, A.loc_tri, u, A.nU);
                    ok = isfinite(L.e.f);
                } else {
                    ok = tri_term<T, ENERGY, false>(x, D, area, A.c, L, A.mlp_table ? A.mlp_table + 10 * u : nullptr);
                }
                if (ok) {
                    fe += (double)local_f(L);
                    if constexpr (MODE >= MODE_GRAD) {
                        if constexpr (MODE == MODE_HVP) {
                            T vl[3 * VD];
#pragma unroll
                            for (int q = 0; q < 3; ++q)
#pragma unroll
                                for (int d = 0; d < VD; ++d) vl[q * VD + d] = vsm[l[q] * VD + d];
                            hvp_edge<VD>(L, vl, yv);
                        }
                        put_vertices<MODE, VD, 3, false>(L, vch, yv);
                        if constexpr (CP > 0) {
                            put_pair<VD, 0, 1, false>(L, pch[0], tr01);
                            put_pair<VD, 0, 2, false>(L, pch[1], tr02);
                            put_pair<VD, 1, 2, false>(L, pch[2], tr12);
                        }
                    }
                    wrote = true;
                } else {
                    atomicOr(A.status, ST_DOMAIN);
                }
            }
            if (MODE >= MODE_GRAD && !wrote) {
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int k = 0; k < CV; ++k) vch[q][k] = T(0);
                if constexpr (CP > 0)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int k = 0; k < CP; ++k) pch[q][k] = T(0);
            }
            // -- hinges of the attached edges: slot s (edge k) is evaluated as
            // the hinge (t_k, t_k+1, t_k+2, extra)
            if constexpr (HINGES) {
                for (int s = 0; s < nslot; ++s) {
                    const int xe = sel3(s, ex[0], ex[1], ex[2]);
                    if (xe == 0xffff) continue;
                    // the slot's edge (t_k, t_k+1), k = rot + s mod 3
                    const int k0 = rot + s >= 3 ? rot + s - 3 : rot + s;
                    const int s1 = k0 == 2 ? 0 : k0 + 1, s2 = k0 == 0 ? 2 : k0 - 1;
                    const int hl[4] = {sel3(k0, l[0], l[1], l[2]), sel3(s1, l[0], l[1], l[2]),
                                       sel3(s2, l[0], l[1], l[2]), xe};
                    T x[12];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int d = 0; d < 3; ++d) x[q * 3 + d] = xs[hl[q] * 3 + d];
                    const int64_t sg = (int64_t)slot0 + ufirst + s;
                    const T thetabar = A.slot_rest[sg];
                    const T w = A.c.kbh2 * A.slot_rest[A.nS + sg];
                    EdgeLocal<HingeEdges, 3, T> L;
                    bool ok;
                    if constexpr (PROJ) {  // the filtered result of k_filtered_slots
                        load_local_soa(L.e, A.loc_slot, sg, A.nS);
                        ok = isfinite(L.e.f);
                    } else {
                        ok = hinge_local<T, false>(x, thetabar, w, L, A.c.eps) && isfinite(local_f(L));
                    }
                    if (!ok) {
                        atomicOr(A.status, ST_DOMAIN);
                        if constexpr (MODE >= MODE_GRAD) {  // its own chunks still need values
                            const uint16_t *sd = A.slot_dst + 4 * sg;
#pragma unroll
                            for (int k = 0; k < CV; ++k) sv[CV * (int)sd[0] + k] = T(0);
                            if constexpr (CP > 0)
#pragma unroll
                                for (int q = 0; q < 3; ++q)
#pragma unroll
                                    for (int k = 0; k < CP; ++k) sp[CP * (int)sd[1 + q] + k] = T(0);
                        }
                        continue;
                    }
                    fe += (double)local_f(L);
                    if constexpr (MODE >= MODE_GRAD) {
                        const uint16_t *sd = A.slot_dst + 4 * sg;
                        T *hv4[4] = {sel3(k0, vch[0], vch[1], vch[2]), sel3(s1, vch[0], vch[1], vch[2]),
                                     sel3(s2, vch[0], vch[1], vch[2]), sv + CV * (int)sd[0]};
                        T hy[12];
                        if constexpr (MODE == MODE_HVP) {
                            T vl[12];
#pragma unroll
                            for (int q = 0; q < 4; ++q)
#pragma unroll
                                for (int d = 0; d < 3; ++d) vl[q * 3 + d] = vsm[hl[q] * 3 + d];
                            hvp_edge<3>(L, vl, hy);
                        }
                        // unit vertices add, the extra vertex stores
                        T *const vadd[3] = {hv4[0], hv4[1], hv4[2]};
                        put_vertices<MODE, 3, 3, true>(L, vadd, hy);
                        if constexpr (MODE == MODE_HVP) put_vertex_hvp<3, 3, false>(L, hy, hv4[3]);
                        else put_vertex<MODE, 3, 3, false>(L, hv4[3]);
                        if constexpr (CP > 0) {
                            // unit pairs (tri vertices p, q: role p + q - 1)
                            const int p01 = k0 + s1 - 1, p02 = k0 + s2 - 1, p12 = s1 + s2 - 1;
                            put_pair<3, 0, 1, true>(L, sel3(p01, pch[0], pch[1], pch[2]), hl[0] > hl[1]);
                            put_pair<3, 0, 2, true>(L, sel3(p02, pch[0], pch[1], pch[2]), hl[0] > hl[2]);
                            put_pair<3, 1, 2, true>(L, sel3(p12, pch[0], pch[1], pch[2]), hl[1] > hl[2]);
                            // pairs with the extra vertex: chunk holds (lower, higher)
                            put_pair<3, 0, 3, false>(L, sp + CP * (int)sd[1], hl[0] > xe);
                            put_pair<3, 1, 3, false>(L, sp + CP * (int)sd[2], hl[1] > xe);
                            put_pair<3, 2, 3, false>(L, sp + CP * (int)sd[3], hl[2] > xe);
                        }
                    }
                }
            }
            // -- cloth: springs on the attached edges, vertex terms
            if constexpr (CLOTH) {
                for (int s = 0; s < nslot; ++s) {
                    const int k0 = rot + s >= 3 ? rot + s - 3 : rot + s;
                    const int s1 = k0 == 2 ? 0 : k0 + 1;
                    const int sl[2] = {sel3(k0, l[0], l[1], l[2]), sel3(s1, l[0], l[1], l[2])};
                    T x[6];
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int d = 0; d < 3; ++d) x[q * 3 + d] = xs[sl[q] * 3 + d];
                    const int64_t sg = (int64_t)slot0 + ufirst + s;
                    EdgeLocal<SpringEdges, 3, T> L;
                    if constexpr (PROJ) load_local_soa(L.e, A.loc_slot, sg, A.nS);
                    else spring_local<T, false>(x, A.slot_rest[sg], A.c.kh2, L, A.c.eps);
                    if (!isfinite(local_f(L))) {
                        atomicOr(A.status, ST_DOMAIN);
                        continue;
                    }
                    fe += (double)local_f(L);
                    if constexpr (MODE >= MODE_GRAD) {
                        T hy[6];
                        if constexpr (MODE == MODE_HVP) {
                            T vl[6];
#pragma unroll
                            for (int q = 0; q < 2; ++q)
#pragma unroll
                                for (int d = 0; d < 3; ++d) vl[q * 3 + d] = vsm[sl[q] * 3 + d];
                            hvp_edge<3>(L, vl, hy);
                        }
                        T *const va[2] = {sel3(k0, vch[0], vch[1], vch[2]), sel3(s1, vch[0], vch[1], vch[2])};
                        put_vertices<MODE, 3, 2, true>(L, va, hy);
                        if constexpr (CP > 0) put_pair<3, 0, 1, true>(L, sel3(k0 + s1 - 1, pch[0], pch[1], pch[2]), sl[0] > sl[1]);
                    }
                }
                const int vmask = flags >> 2;
                int vt = hd[kHdrVTerm] + ex[0];  // the unit's first vertex term (cloth units carry no hinge extras)
                for (int q = 0; q < 3; ++q) {
                    if (!((vmask >> q) & 1)) continue;
                    const int lq = l[q];
                    const int64_t vg = A.foot[fb + lq];
                    T x[3], xh[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        x[d] = xs[lq * 3 + d];
                        xh[d] = A.xhat[vg * 3 + d];
                    }
                    Local<T, 3> L;
                    vertex_local(x, xh, A.c.rho * A.vterm_rest[vt], A.c.h2, A.c.g, L);
                    ++vt;
                    fe += (double)L.f;
                    if constexpr (MODE >= MODE_GRAD) {
                        T *ch = sel3(q, vch[0], vch[1], vch[2]);
#pragma unroll
                        for (int d = 0; d < 3; ++d) ch[d] += L.g[d];
                        if constexpr (MODE == MODE_HVP) {
#pragma unroll
                            for (int d = 0; d < 3; ++d) ch[3 + d] += L.H[hix(d, d)] * vsm[lq * 3 + d];
                        }
                        if constexpr (MODE == MODE_HESS) {
#pragma unroll
                            for (int d = 0; d < 3; ++d) ch[3 + hix(d, d)] += L.H[hix(d, d)];
                        }
                    }
                }
            }
        }
        // per-warp energy partials, summed in warp order after the barrier
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fe += __shfl_down_sync(0xffffffffu, fe, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = fe;
        // chunks complete, the next tile known, x of this tile no longer read
        __syncthreads();
        const int tn = s_next;
        ++taken;
        int32_t fvn[KR];
        if (tn < A.tile_end) foot_rows(s_hdr[p ^ 1], fvn);  // the loads land while the vertex pass runs

        // ---- gather: every output entry is the sum of its segment
        bool meta_ok = true;
        if (MODE >= MODE_GRAD) {
            if (!bar_wait(&meta_bar, phase & 1u)) {
                atomicOr(A.status, ST_TIMEOUT);
                meta_ok = false;
                bar_wait(&meta_bar, phase & 1u);  // give the copy into this block's shared memory time to land
            }
            ++phase;
        }
        const int32_t *rows = reinterpret_cast<const int32_t *>(blob);
        const uint32_t *codes = reinterpret_cast<const uint32_t *>(blob + hd[kHdrCodeOff]);
        const int32_t *ptab = reinterpret_cast<const int32_t *>(blob + hd[kHdrPartOff]);
        if (MODE >= MODE_GRAD && meta_ok) {
            // vertex pass: one lane per footprint row sums the row's vertex
            // chunks (gradient and diagonal upper entries, or gradient and
            // H v) in registers and writes its gradient (H v) row and
            // diagonal block, or its partial slot
            constexpr int CVH = Chunk<MODE_HESS, VD>::V;
            for (int r = tid; r < nf; r += THREADS) {
                const int4 rw = *reinterpret_cast<const int4 *>(rows + kRowWords * r);
                const int nv = (int)((uint32_t)rw.y >> 24), vs0 = rw.z & 0xffff;
                T acc[CV > 0 ? CV : 1];
#pragma unroll
                for (int e = 0; e < CV; ++e) acc[e] = -T(0);
                const T *src = sv + CV * vs0;
                // two chunks per iteration: their loads are in flight together
                // (the sums keep the chunk order)
#pragma unroll 2
                for (int q = 0; q < nv; ++q)
#pragma unroll
                    for (int e = 0; e < CV; ++e) acc[e] += src[CV * q + e];
                if ((rw.w >> 15) & 1) {  // a later producer of a shared row
                    store_run<CV>(A.vpart + (int64_t)ptab[rw.w >> 16] * CVH, acc);
                    continue;
                }
                const int64_t vg = A.foot[fb + r];
                if (A.grad) store_run<VD>(A.grad + vg * VD, acc);
                if constexpr (MODE == MODE_HVP) store_run<VD>(A.hv + vg * VD, acc + VD);
                if constexpr (MODE == MODE_HESS) {
                    T blk[VD * VD];
#pragma unroll
                    for (int i = 0; i < VD; ++i)
#pragma unroll
                        for (int j = 0; j < VD; ++j) blk[i * VD + j] = acc[VD + (i <= j ? hix(i, j) : hix(j, i))];
                    store_run<VD * VD>(A.bsr + ((int64_t)rw.x + (rw.w & 0x7fff)) * (VD * VD), blk);
                }
            }
        }
        // x (and v) of the next tile into the fixed region; eval of this tile
        // is over, and the region lies below this tile's chunks and blob
        if (tn < A.tile_end) stage_rows(s_hdr[p ^ 1], fvn);
        if (MODE == MODE_HESS && meta_ok) {
            // pair pass: one lane per pair segment; the lane sums the
            // segment in chunk order once, then writes block A = (lo, hi)
            // and its transpose, block B = (hi, lo), each to the BSR or to
            // its partial slot
            constexpr int NB = VD * VD;
            const int npair = hd[kHdrNCode];
            const uint2 *pc = reinterpret_cast<const uint2 *>(codes);
            for (int j = tid; j < npair; j += THREADS) {
                const uint2 c = pc[j];
                const int start = (int)(c.x & 0x1fffu), cnt = (int)((c.x >> 13) & 15u);
                T acc[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k) acc[k] = -T(0);
                const T *src = sp + CP * start;
#pragma unroll 2
                for (int q = 0; q < cnt; ++q)
#pragma unroll
                    for (int k = 0; k < NB; ++k) acc[k] += src[CP * q + k];
                const uint32_t da = ((c.x >> 19) & 511u) << 9 | (c.y & 511u);
                const uint32_t db = ((c.y >> 9) & 511u) << 9 | ((c.y >> 18) & 511u);
                T *oa = (c.x >> 17) & 1u ? A.ppart + (int64_t)ptab[da] * NB
                                         : A.bsr + ((int64_t)rows[kRowWords * (da >> 9)] + (da & 511u)) * NB;
                T *ob = (c.x >> 18) & 1u ? A.ppart + (int64_t)ptab[db] * NB
                                         : A.bsr + ((int64_t)rows[kRowWords * (db >> 9)] + (db & 511u)) * NB;
                T tr[NB];
#pragma unroll
                for (int i = 0; i < VD; ++i)
#pragma unroll
                    for (int k = 0; k < VD; ++k) tr[i * VD + k] = acc[k * VD + i];
                store_run<NB>(oa, acc);
                store_run<NB>(ob, tr);
            }
        }
        if (tid == 0) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) sum += s_red[w];
            A.epart[t] = sum;
        }
        cp_async_wait_all();
        t = tn;
        p ^= 1;
    }
    if (t == INT_MAX && tid == 0) atomicOr(A.status, ST_TIMEOUT);  // the queue never ran dry within its bound
}

// N consecutive reals from global memory into registers, in aligned pairs
// where the run allows (the loads of store_run)
template <int N, typename T>
__device__ __forceinline__ void load_run(const T *src, T *v)
{
    using V2 = std::conditional_t<sizeof(T) == 4, float2, double2>;
    if constexpr (N == 1) {
        v[0] = src[0];
    } else if constexpr (N > 1) {
        const bool odd = ((reinterpret_cast<uintptr_t>(src) / sizeof(T)) & 1u) != 0;
        if constexpr (N % 2 == 1) {
            const T one = src[odd ? 0 : N - 1];
            const V2 *p = reinterpret_cast<const V2 *>(src + (odd ? 1 : 0));
            T w[N - 1];
#pragma unroll
            for (int j = 0; j < (N - 1) / 2; ++j) {
                const V2 q = p[j];
                w[2 * j] = q.x;
                w[2 * j + 1] = q.y;
            }
            // odd start: one, w[0..N-2]; even start: w[0..N-2], one
#pragma unroll
            for (int j = 0; j < N; ++j) {
                if (j == 0) v[0] = odd ? one : w[0];
                else if (j == N - 1) v[N - 1] = odd ? w[N - 2] : one;
                else v[j] = odd ? w[j - 1] : w[j];
            }
        } else if (!odd) {
            const V2 *p = reinterpret_cast<const V2 *>(src);
#pragma unroll
            for (int j = 0; j < N / 2; ++j) {
                const V2 q = p[j];
                v[2 * j] = q.x;
                v[2 * j + 1] = q.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = src[j];
        }
    }
}

// Fix-up of the outputs several tiles produce: one thread per output (a
// gradient or H v row with its diagonal block, or a pair block) adds the
// output's partial slots, in tile order, to what the lowest tile stored;
// each float is the stored value plus its slots in slot order.  Entries:
// row vertex, position of the block in its BSR row (row start from the
// active pattern's row pointer), number of slots, first slot; vertex
// entries take threads [0, n_v), pair entries the next n_p.  Entries and
// slots are in output order, so neighbouring threads read neighbouring
// slots.
template <typename T, int VD, int MODE>
__global__ void __launch_bounds__(256) k_tile_fixup(const int4 *__restrict__ fix_v, int64_t n_v,
                                                    const int4 *__restrict__ fix_p, int64_t n_p,
                                                    const T *__restrict__ vpart, const T *__restrict__ ppart,
                                                    const int32_t *__restrict__ row_ptr, T *grad, T *bsr, T *hv)
{
    constexpr int CVH = Chunk<MODE_HESS, VD>::V, NB = VD * VD;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_v) {
        const int4 e = __ldg(fix_v + i);
        const T *p = vpart + (int64_t)e.w * CVH;
        if (grad) {
            T *out = grad + (int64_t)e.x * VD;
            T a[VD];
            load_run<VD>(out, a);
            for (int q = 0; q < e.z; ++q)
#pragma unroll
                for (int d = 0; d < VD; ++d) a[d] += p[(int64_t)q * CVH + d];
            store_run<VD>(out, a);
        }
        if constexpr (MODE == MODE_HVP) {
            T *out = hv + (int64_t)e.x * VD;
            T a[VD];
            load_run<VD>(out, a);
            for (int q = 0; q < e.z; ++q)
#pragma unroll
                for (int d = 0; d < VD; ++d) a[d] += p[(int64_t)q * CVH + VD + d];
            store_run<VD>(out, a);
        }
        if constexpr (MODE == MODE_HESS) {
            T *out = bsr + ((int64_t)__ldg(row_ptr + e.x) + e.y) * NB;
            T a[NB];
            load_run<NB>(out, a);
            for (int q = 0; q < e.z; ++q) {
                T u[VD * (VD + 1) / 2];
#pragma unroll
                for (int k = 0; k < VD * (VD + 1) / 2; ++k) u[k] = p[(int64_t)q * CVH + VD + k];
#pragma unroll
                for (int r = 0; r < VD; ++r)
#pragma unroll
                    for (int c = 0; c < VD; ++c) a[r * VD + c] += u[r <= c ? hix(r, c) : hix(c, r)];
            }
            store_run<NB>(out, a);
        }
    } else if (MODE == MODE_HESS && i < n_v + n_p) {
        const int4 e = __ldg(fix_p + (i - n_v));
        T *out = bsr + ((int64_t)__ldg(row_ptr + e.x) + e.y) * NB;
        const T *p = ppart + (int64_t)e.w * NB;
        T a[NB];
        load_run<NB>(out, a);
        for (int q = 0; q < e.z; ++q) {
            T u[NB];
            load_run<NB>(p + (int64_t)q * NB, u);
#pragma unroll
            for (int k = 0; k < NB; ++k) a[k] += u[k];
        }
        store_run<NB>(out, a);
    }
}

// zero the gradient rows and diagonal blocks of vertices no unit touches
template <typename T, int VD>
__global__ void k_zero_untouched(const int32_t *verts, const int32_t *blocks, int64_t n, T *grad, T *bsr, T *hv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int d = 0; d < VD; ++d) {
        if (grad) grad[(int64_t)verts[i] * VD + d] = T(0);
        if (hv) hv[(int64_t)verts[i] * VD + d] = T(0);
    }
    if (bsr)
#pragma unroll
        for (int k = 0; k < VD * VD; ++k) bsr[(int64_t)blocks[i] * VD * VD + k] = T(0);
}

// Launch of one (precision, mode, filtering) variant for any energy.  Each
// variant is instantiated in its own translation unit (tiled_inst.cu) so
// that they compile in parallel.  Grid: the resident blocks of the whole GPU
// (persistent), at most one per tile.
template <typename T, int MODE, bool PROJ, int TT>
void launch_tiled_threads(int energy, int n_sm, size_t smem, cudaStream_t s, const TiledArgs<T> &A)
{
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TT, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const int grid = (int)std::min<int64_t>((int64_t)per_sm * n_sm, A.tile_end - A.tile_begin);
        if (grid > 0) kern<<<grid, TT, smem, s>>>(A);
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

// Launch of one (precision, mode, filtering) variant for any energy.  Each
// variant is instantiated in its own translation unit (tiled_inst.cu) so
// that they compile in parallel.  Grid: the resident blocks of the whole GPU
// (persistent), at most one per tile.  FP32 also has a 128-thread variant
// (ADM_OPT_TILE_THREADS, the autotuner's second axis).
template <typename T, int MODE, bool PROJ>
void launch_tiled_mode(int energy, int threads, int n_sm, size_t smem, cudaStream_t s, const TiledArgs<T> &A)
{
    if constexpr (sizeof(T) == 4) {
        if (threads == 128) {
            launch_tiled_threads<T, MODE, PROJ, 128>(energy, n_sm, smem, s, A);
            return;
        }
    }
    launch_tiled_threads<T, MODE, PROJ, 256>(energy, n_sm, smem, s, A);
}

#define ADM_TILED_VARIANTS(X, T)                                                                          \
    X(T, MODE_VALUE, false) X(T, MODE_GRAD, false) X(T, MODE_HESS, false) X(T, MODE_HESS, true)           \
    X(T, MODE_HVP, false) X(T, MODE_HVP, true)
#define ADM_TILED_EXTERN(T, M, P)                                                                          \
    extern template void launch_tiled_mode<T, M, P>(int, int, int, size_t, cudaStream_t, const TiledArgs<T> &);
#define ADM_TILED_INST(T, M, P) \
    template void launch_tiled_mode<T, M, P>(int, int, int, size_t, cudaStream_t, const TiledArgs<T> &);

template <typename T>
static void launch_tiled(int energy, int mode, bool proj, int threads, int n_sm, size_t smem, cudaStream_t s,
                         const TiledArgs<T> &A)
{
    if (mode == MODE_VALUE) launch_tiled_mode<T, MODE_VALUE, false>(energy, threads, n_sm, smem, s, A);
    else if (mode == MODE_GRAD) launch_tiled_mode<T, MODE_GRAD, false>(energy, threads, n_sm, smem, s, A);
    else if (mode == MODE_HESS && !proj) launch_tiled_mode<T, MODE_HESS, false>(energy, threads, n_sm, smem, s, A);
    else if (mode == MODE_HESS) launch_tiled_mode<T, MODE_HESS, true>(energy, threads, n_sm, smem, s, A);
    else if (!proj) launch_tiled_mode<T, MODE_HVP, false>(energy, threads, n_sm, smem, s, A);
    else launch_tiled_mode<T, MODE_HVP, true>(energy, threads, n_sm, smem, s, A);
}

// buffers of the terms' filtered results, sized for FP64 (the largest
// Local: 55 reals per hinge, 28 per triangle), allocated on first use
inline adm_status ensure_filtered_locals(adm_ctx *h, TileSet &ts)
{
    if (ts.d_loc_tri && ts.d_loc_slot) return ADM_OK;
    const size_t nu = (size_t)std::max<int64_t>(h->m.nT, 1), ns = (size_t)std::max<int64_t>(ts.n_slots, 1);
    if (cudaMalloc(&ts.d_loc_tri, nu * 28 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ts.d_loc_slot, ns * 55 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ts.d_loc_tri);
        cudaFree(ts.d_loc_slot);
        ts.d_loc_tri = ts.d_loc_slot = nullptr;
        return ADM_ERR_OOM;
    }
    h->owned.push_back(ts.d_loc_tri);
    h->owned.push_back(ts.d_loc_slot);
    return ADM_OK;
}

template <typename T>
adm_status eval_tiled(adm_ctx *h, const EvalArgs &a)
{
    const HostMesh &m = h->m;
    const int vd = m.vdim;
    const bool hin = has_hinges(a.energy);
    const int kind = hin ? PAT_SHELL : PAT_TRI;
    TileSet &ts = h->tiles[kind];
    const int mode = a.hv ? MODE_HVP : (a.bsr ? MODE_HESS : (a.grad ? MODE_GRAD : MODE_VALUE));
    const int eb = (int)sizeof(T);
    int64_t &cached = ts.smem_cache[mode][vd == 3][eb == 8];
    if (cached == 0) cached = std::max<int64_t>(16, tile_smem_bytes(ts, mode, vd, eb));
    const size_t smem = (size_t)cached;
    if (smem > 227 * 1024) return ADM_ERR_UNSUPPORTED;
    cudaStream_t s = a.stream;
    StageTimer tm(h, s);
    const bool pairs = h->inter.kind == kind && h->inter.n_terms() > 0;
    if (cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return ADM_ERR_CUDA;
    if (a.energy == ADM_MASS_SPRING && (!ts.cloth_built || !h->d_xhat[a.prec])) return ADM_ERR_UNSUPPORTED;
    // queue positions start at zero every pass
    if (cudaMemsetAsync(ts.d_sync, 0, 8 * sizeof(int32_t), s) != cudaSuccess) return ADM_ERR_CUDA;
    TiledArgs<T> A;
    A.hdr = ts.d_hdr;
    A.unit = ts.d_unit;
    A.unit_dst = ts.d_unit_dst;
    A.slot_dst = ts.d_slot_dst;
    A.foot = ts.d_foot;
    A.meta = ts.d_meta;
    A.meta_off = ts.d_meta_off;
    A.tri_rest = (const T *)ts.d_tri_rest[a.prec];
    A.slot_rest = (const T *)ts.d_slot_rest[a.prec];
    A.vterm_rest = (const T *)ts.d_vterm_rest[a.prec];
    A.nU = m.nT;
    A.nS = ts.n_slots;
    A.x = (const T *)a.x;
    A.grad = (T *)a.grad;
    A.bsr = (T *)a.bsr;
    A.v = (const T *)a.v;
    A.hv = (T *)a.hv;
    A.vpart = (T *)ts.d_vpart;
    A.ppart = (T *)ts.d_ppart;
    A.epart = h->d_epart;
    A.status = h->d_status;
    A.nf_cap = (int32_t)std::max<int64_t>(ts.max_nf, 1);
    A.c = consts<T>(h, a.energy);
    A.mlp_table = nullptr;
    A.xhat = (const T *)h->d_xhat[a.prec];
    if (a.energy == ADM_MLP_MEMBRANE) {
        if (sizeof(T) != 4 || !h->d_mlp_theta || !ts.d_tri_verts) return ADM_ERR_UNSUPPORTED;
        tm.begin(ADM_STAGE_MLP);
        adm_status st = mlp_triangle_table(h->d_mlp_theta, h->d_mlp_norm, m.nT, ts.d_tri_verts,
                                           (const float *)ts.d_tri_rest[ADM_FP32], (const float *)a.x,
                                           h->d_mlp_table, h->mlp_net, h->d_status, s);
        tm.end(ADM_STAGE_MLP);
        if (st != ADM_OK) return st;
        A.mlp_table = h->d_mlp_table;
    }
    int n_sm = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    const bool filt = h->proj != 0 && (mode == MODE_HESS || mode == MODE_HVP);
    const bool split = a.n_split > 0 && a.split_mesh && a.split_ready && !pairs && a.energy != ADM_MLP_MEMBRANE && !filt &&
                       h->split_stream[0] && h->split_stream[1] && h->split_start &&
                       (int)h->split_done.size() >= a.n_split && a.n_split <= 8;
    if (a.n_split > 0 && !split)  // x arriving in ranges, consumed whole here: wait for all of them
        for (int k = 0; k < a.n_split; ++k)
            if (cudaStreamWaitEvent(s, a.split_ready[k], 0) != cudaSuccess) return ADM_ERR_CUDA;
    const int64_t nz = (int64_t)ts.zero_verts.size();
    if (nz > 0 && (a.grad || a.bsr || a.hv)) {
        tm.begin(ADM_STAGE_ZERO);
        const int blocks = (int)((nz + 255) / 256);
        if (vd == 3)
            k_zero_untouched<T, 3><<<blocks, 256, 0, s>>>(ts.d_zero_verts, ts.d_zero_blocks, nz, (T *)a.grad,
                                                           (T *)a.bsr, (T *)a.hv);
        else
            k_zero_untouched<T, 2><<<blocks, 256, 0, s>>>(ts.d_zero_verts, ts.d_zero_blocks, nz, (T *)a.grad,
                                                           (T *)a.bsr, (T *)a.hv);
        tm.end(ADM_STAGE_ZERO);
    }
    tm.begin(ADM_STAGE_TILED);
    A.loc_tri = A.loc_slot = nullptr;
    if (filt) {
        // every term's filtered result first, one thread per term
        adm_status st = ensure_filtered_locals(h, ts);
        if (st != ADM_OK) return st;
        LocalArgs<T> F;
        F.nU = m.nT;
        F.nS = ts.n_slots;
        F.tri_verts = ts.d_tri_verts;
        F.slot_verts = reinterpret_cast<const int4 *>(ts.d_slot_verts);
        F.tri_rest = A.tri_rest;
        F.slot_rest = A.slot_rest;
        F.x = A.x;
        F.mlp_table = A.mlp_table;
        F.loc_tri = (T *)ts.d_loc_tri;
        F.loc_slot = (T *)ts.d_loc_slot;
        F.c = A.c;
        const int bt = (int)((F.nU + 127) / 128);
        const bool tris = a.energy != ADM_HINGE_BENDING && a.energy != ADM_MASS_SPRING;
        if (tris && F.nU > 0) {
            switch (a.energy) {
            case ADM_SYMDIR2D: k_filtered_tris<T, ADM_SYMDIR2D><<<bt, 128, 0, s>>>(F); break;
            case ADM_STVK_MEMBRANE: k_filtered_tris<T, ADM_STVK_MEMBRANE><<<bt, 128, 0, s>>>(F); break;
            case ADM_NH_MEMBRANE: k_filtered_tris<T, ADM_NH_MEMBRANE><<<bt, 128, 0, s>>>(F); break;
            case ADM_AREA: k_filtered_tris<T, ADM_AREA><<<bt, 128, 0, s>>>(F); break;
            case ADM_MLP_MEMBRANE:
                if constexpr (sizeof(T) == 4) k_filtered_tris<T, ADM_MLP_MEMBRANE><<<bt, 128, 0, s>>>(F);
                break;
            case ADM_SHELL: k_filtered_tris<T, ADM_SHELL><<<bt, 128, 0, s>>>(F); break;
            default: break;
            }
        }
        if (F.nS > 0) {
            if (hin) k_filtered_slots<T, ADM_SHELL><<<(int)((F.nS + 255) / 256), 256, 0, s>>>(F);
            else if (a.energy == ADM_MASS_SPRING)
                k_filtered_slots<T, ADM_MASS_SPRING><<<(int)((F.nS + 255) / 256), 256, 0, s>>>(F);
        }
        A.loc_tri = F.loc_tri;
        A.loc_slot = F.loc_slot;
    }
    if (!split) {
        A.next = ts.d_sync;
        A.tile_begin = 0;
        A.tile_end = ts.n_tiles;
        launch_tiled<T>(a.energy, mode, h->proj != 0, h->tile_threads, n_sm, smem, s, A);
    } else {
        // per mesh range, on two streams in turn: wait for its x and run its
        // tiles (tiles and groups never span meshes).  The copies of later
        // ranges overlap the kernels of earlier ones, and a range's launch
        // overlaps the tail of the one before; the pass's stream resumes when
        // every range is done.
        if (cudaEventRecord(h->split_start, s) != cudaSuccess) return ADM_ERR_CUDA;
        for (int k = 0; k < a.n_split; ++k) {
            cudaStream_t ks = h->split_stream[k & 1];
            if (cudaStreamWaitEvent(ks, h->split_start, 0) != cudaSuccess ||
                cudaStreamWaitEvent(ks, a.split_ready[k], 0) != cudaSuccess)
                return ADM_ERR_CUDA;
            TiledArgs<T> B = A;
            B.next = ts.d_sync + k;
            B.tile_begin = ts.mesh_tile_off[a.split_mesh[k]];
            B.tile_end = ts.mesh_tile_off[a.split_mesh[k + 1]];
            if (B.tile_end > B.tile_begin)
                launch_tiled<T>(a.energy, mode, h->proj != 0, h->tile_threads, n_sm, smem, ks, B);
            if (cudaEventRecord(h->split_done[k], ks) != cudaSuccess) return ADM_ERR_CUDA;
        }
        for (int k = 0; k < a.n_split; ++k)
            if (cudaStreamWaitEvent(s, h->split_done[k], 0) != cudaSuccess) return ADM_ERR_CUDA;
    }
    // the later producers' parts of shared outputs, added in tile order
    const int64_t n_fv = mode >= MODE_GRAD ? (int64_t)ts.fix_v.size() / 4 : 0;
    const int64_t n_fp = mode == MODE_HESS ? (int64_t)ts.fix_p.size() / 4 : 0;
    if (n_fv + n_fp > 0) {
        const int32_t *rp = active_row_ptr(h, kind);
        const int blocks = (int)((n_fv + n_fp + 255) / 256);
        const int4 *fv = reinterpret_cast<const int4 *>(ts.d_fix_v), *fp = reinterpret_cast<const int4 *>(ts.d_fix_p);
        const T *vp = (const T *)ts.d_vpart, *pp = (const T *)ts.d_ppart;
        auto go = [&](auto kern) { kern<<<blocks, 256, 0, s>>>(fv, n_fv, fp, n_fp, vp, pp, rp, (T *)a.grad, (T *)a.bsr, (T *)a.hv); };
        if (vd == 3) {
            if (mode == MODE_HESS) go(k_tile_fixup<T, 3, MODE_HESS>);
            else if (mode == MODE_HVP) go(k_tile_fixup<T, 3, MODE_HVP>);
            else go(k_tile_fixup<T, 3, MODE_GRAD>);
        } else {
            if (mode == MODE_HESS) go(k_tile_fixup<T, 2, MODE_HESS>);
            else if (mode == MODE_HVP) go(k_tile_fixup<T, 2, MODE_HVP>);
            else go(k_tile_fixup<T, 2, MODE_GRAD>);
        }
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
