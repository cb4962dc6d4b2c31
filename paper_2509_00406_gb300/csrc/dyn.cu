// dyn.cu -- interaction terms (vertex-vertex pairs, vertex-face elements)
// and the dynamic block pattern they induce (Sec. 4.3, Sec. 6.3, Alg. 1).
//
// An interaction set replaces the previous one and extends the mesh pattern
// on the GPU, following Alg. 1.  Every term touches the blocks of its vertex
// pairs (one pair for a vertex-vertex term, six for a vertex-face element),
// the candidates.  Per-row counts (the mesh row plus the candidate blocks not
// already present), an exclusive scan into a row pointer, a copy of the mesh
// columns and an atomic append of the new ones give a pattern in which a
// block touched by several terms appears several times; each row's appended
// run is sorted, its distinct columns counted, and a second scan and copy
// give the final pattern (mesh columns first in their order, new columns
// ascending, each once).  Two pattern buffers alternate.  The tiles of the
// mesh kernel keep their per-row codes; only their row starts and
// shared-block indices are remapped.  Evaluation adds the barriers of
// Sec. 7.7 with atomic additions after the tiled mesh pass: the new blocks
// are zeroed first (several terms may share one).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "device_common.cuh"

namespace adm {

namespace {

constexpr int kDynThreads = 256;
constexpr int kScanItems = 4;  // per thread of the scan

int blocks_for(int64_t n, int per = kDynThreads) { return (int)std::max<int64_t>(1, (n + per - 1) / per); }

template <typename P>
adm_status alloc(adm_ctx *h, P **out, size_t bytes)
{
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return ADM_ERR_OOM;
    }
    h->owned.push_back(p);
    *out = (P *)p;
    return ADM_OK;
}

void release(adm_ctx *h, void *p)
{
    if (!p) return;
    auto it = std::find(h->owned.begin(), h->owned.end(), p);
    if (it != h->owned.end()) h->owned.erase(it);
    cudaFree(p);
}

// ------------------------------------------------------------- Alg. 1 --
__global__ void k_row_len(int64_t nV, const int32_t *rp, int32_t *cnt)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nV) cnt[r] = rp[r + 1] - rp[r];
    if (r == nV) cnt[r] = 0;
}

// position of column c in the sorted run col[a, b), or -1
__device__ __forceinline__ int32_t find_col(const int32_t *col, int32_t a, int32_t b, int32_t c)
{
    const int32_t end = b;
    while (a < b) {
        const int32_t m = (a + b) >> 1;
        if (col[m] < c) a = m + 1;
        else b = m;
    }
    return (a < end && col[a] == c) ? a : -1;
}

// step (1): count the new entries of every row; mark pairs whose blocks the
// mesh pattern already has
__global__ void k_count(int64_t n, const int32_t *pairs, int64_t nV, const int32_t *rp, const int32_t *col,
                        int32_t *cnt, int32_t *slot, int *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t i = pairs[2 * p], j = pairs[2 * p + 1];
    if (i < 0 || j < 0 || i >= nV || j >= nV || i == j) {
        atomicOr(status, ST_DOMAIN);
        slot[2 * p] = slot[2 * p + 1] = -1;
        return;
    }
    const int32_t k = find_col(col, rp[i], rp[i + 1], j);
    if (k >= 0) {  // in the mesh pattern: (i, j) at offset k - rp[i], (j, i) found below
        slot[2 * p] = (int32_t)(0x80000000u | (uint32_t)(k - rp[i]));
        const int32_t k2 = find_col(col, rp[j], rp[j + 1], i);
        slot[2 * p + 1] = (int32_t)(0x80000000u | (uint32_t)(k2 - rp[j]));
        return;
    }
    slot[2 * p] = slot[2 * p + 1] = 0;
    atomicAdd(&cnt[i], 1);
    atomicAdd(&cnt[j], 1);
}

// step (2): exclusive scan of n int32 in three launches
template <int THREADS>
__global__ void k_scan_local(int64_t n, const int32_t *in, int32_t *out, int32_t *bsum)
{
    __shared__ int32_t part[THREADS];
    const int64_t base = (int64_t)blockIdx.x * THREADS * kScanItems + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < THREADS; off <<= 1) {  // inclusive Hillis-Steele over thread sums
        const int32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == THREADS - 1) bsum[blockIdx.x] = part[THREADS - 1];
}

template <int THREADS>
__global__ void k_scan_sums(int nb, int32_t *bsum)
{
    __shared__ int32_t part[THREADS];
    const int per = (nb + THREADS - 1) / THREADS;
    const int b0 = threadIdx.x * per;
    int32_t s = 0;
    for (int b = b0; b < b0 + per && b < nb; ++b) s += bsum[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < THREADS; off <<= 1) {
        const int32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int b = b0; b < b0 + per && b < nb; ++b) {
        const int32_t t = bsum[b];
        bsum[b] = run;
        run += t;
    }
}

__global__ void k_scan_add(int64_t n, int32_t *out, const int32_t *bsum)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / (kDynThreads * kScanItems)];
}

// step (3): copy the mesh columns; acc = next free offset of every row
__global__ void k_copy_rows(int64_t nV, const int32_t *rp, const int32_t *col, const int32_t *rpx, int32_t *colx,
                            int32_t *acc)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nV) return;
    const int32_t a = rp[r], len = rp[r + 1] - a, o = rpx[r];
    for (int32_t k = 0; k < len; ++k) colx[o + k] = col[a + k];
    acc[r] = len;
}

// step (4): append the new columns
__global__ void k_append(int64_t n, const int32_t *pairs, const int32_t *slot, const int32_t *rpx, int32_t *acc,
                         int32_t *colx)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || slot[2 * p] != 0) return;
    const int32_t i = pairs[2 * p], j = pairs[2 * p + 1];
    colx[rpx[i] + atomicAdd(&acc[i], 1)] = j;
    colx[rpx[j] + atomicAdd(&acc[j], 1)] = i;
}

// the six vertex pairs of every vertex-face element (p, a, b, c), in the
// order (p,a) (p,b) (p,c) (a,b) (a,c) (b,c)
__global__ void k_quad_pairs(int64_t nq, const int32_t *quads, int32_t *cand)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    int32_t v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = quads[4 * q + a];
    int k = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b, ++k) {
            cand[12 * q + 2 * k] = v[a];
            cand[12 * q + 2 * k + 1] = v[b];
        }
}

// sort every row's appended run (insertion sort: runs are short) and count
// its distinct columns: cnt = mesh row length + distinct new columns
__global__ void k_sort_tails(int64_t nV, const int32_t *rp, const int32_t *rpt, int32_t *colt, int32_t *cnt)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r == nV) cnt[r] = 0;
    if (r >= nV) return;
    const int32_t len = rp[r + 1] - rp[r];
    const int32_t a = rpt[r] + len, b = rpt[r + 1];
    for (int32_t k = a + 1; k < b; ++k) {
        const int32_t c = colt[k];
        int32_t q = k - 1;
        while (q >= a && colt[q] > c) {
            colt[q + 1] = colt[q];
            --q;
        }
        colt[q + 1] = c;
    }
    int32_t u = b > a ? 1 : 0;
    for (int32_t k = a + 1; k < b; ++k) u += colt[k] != colt[k - 1];
    cnt[r] = len + u;
}

// final rows: the mesh columns, then the distinct new columns; every new
// block's index into the list of new blocks (rows before r hold
// rpx[r] - rp[r] of them)
__global__ void k_copy_unique(int64_t nV, const int32_t *rp, const int32_t *rpt, const int32_t *colt,
                              const int32_t *rpx, int32_t *colx, int32_t *newb)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nV) return;
    const int32_t len = rp[r + 1] - rp[r], o = rpx[r], t = rpt[r];
    for (int32_t k = 0; k < len; ++k) colx[o + k] = colt[t + k];
    int32_t w = o + len, nb = rpx[r] - rp[r];
    for (int32_t k = t + len; k < rpt[r + 1]; ++k) {
        if (k > t + len && colt[k] == colt[k - 1]) continue;
        colx[w] = colt[k];
        newb[nb++] = w++;
    }
}

// final block index of both blocks of every pair (bit 31: a mesh block)
__global__ void k_slots(int64_t n, const int32_t *pairs, const int32_t *rp, const int32_t *rpx, const int32_t *colx,
                        int32_t *slot, int *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t i = pairs[2 * p], j = pairs[2 * p + 1];
    if (slot[2 * p] == -1) return;
    if (slot[2 * p] & 0x80000000) {
        slot[2 * p] = (int32_t)(0x80000000u | (uint32_t)(rpx[i] + (slot[2 * p] & 0x7fffffff)));
        slot[2 * p + 1] = (int32_t)(0x80000000u | (uint32_t)(rpx[j] + (slot[2 * p + 1] & 0x7fffffff)));
        return;
    }
    slot[2 * p] = find_col(colx, rpx[i] + (rp[i + 1] - rp[i]), rpx[i + 1], j);
    slot[2 * p + 1] = find_col(colx, rpx[j] + (rp[j + 1] - rp[j]), rpx[j + 1], i);
    if (slot[2 * p] < 0 || slot[2 * p + 1] < 0) atomicOr(status, ST_DOMAIN);  // never a block index past the pattern
}

// position of every vertex's own block in its mesh-pattern row
__global__ void k_diag_off(int64_t nV, const int32_t *rp, const int32_t *col, int32_t *doff)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nV) doff[v] = find_col(col, rp[v], rp[v + 1], (int32_t)v) - rp[v];
}

// (row, offset in the row) of mesh-pattern block indices
__global__ void k_block_rows(int64_t n, const int32_t *blocks, int64_t nV, const int32_t *rp, int32_t *row,
                             int32_t *off)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t b = blocks[k];
    int64_t lo = 0, hi = nV;  // row r with rp[r] <= b < rp[r + 1]
    while (hi - lo > 1) {
        const int64_t m = (lo + hi) >> 1;
        if (rp[m] <= b) lo = m;
        else hi = m;
    }
    row[k] = (int32_t)lo;
    off[k] = b - rp[lo];
}

// tiles: the row starts in the metadata blobs follow the extended pattern
// (the tiles' codes are unchanged: a row's mesh columns come first)
__global__ void k_remap_tiles(int32_t n_tiles, const int32_t *hdr, const int32_t *foot, const int64_t *meta_off,
                              unsigned char *meta, const int32_t *rpx)
{
    const int32_t t = blockIdx.x;
    if (t >= n_tiles) return;
    const int32_t foot_begin = hdr[kHdr * t + kHdrFoot], nf = hdr[kHdr * t + kHdrNF];
    int32_t *rows = reinterpret_cast<int32_t *>(meta + meta_off[t]);
    for (int r = threadIdx.x; r < nf; r += blockDim.x)
        rows[kRowWords * r] = rpx[foot[foot_begin + r]];
}

__global__ void k_remap_zero(int64_t n, const int32_t *row, const int32_t *off, const int32_t *rpx, int32_t *blocks)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) blocks[k] = rpx[row[k]] + off[k];
}

// --------------------------------------------------------- evaluation --
template <typename T>
struct ContactArgs {
    int64_t n;
    const int32_t *verts, *slot, *rpx, *diag_off;  // NV vertices and NV(NV-1) slots per term
    const T *x, *v;
    T *grad, *bsr, *hv;
    double *term_e;
    T c, dhat, eps;
};

// one thread per term: NV = 2 a vertex-vertex pair, NV = 4 a vertex-face
// element; gradient, Hessian blocks and H v with atomic additions
template <typename T, int NV, int MODE, bool PROJ>
__global__ void __launch_bounds__(kDynThreads) k_contact(ContactArgs<T> A)
{
    constexpr int K = 3 * NV;
    const int64_t p = (int64_t)blockIdx.x * kDynThreads + threadIdx.x;
    if (p >= A.n) return;
    int32_t vid[NV];
    T x[K];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        vid[a] = A.verts[NV * p + a];
#pragma unroll
        for (int d = 0; d < 3; ++d) x[3 * a + d] = A.x[3 * (int64_t)vid[a] + d];
    }
    Local<T, K> L;
    bool active;
    if constexpr (NV == 2) active = contact_local<T, PROJ>(x, A.c, A.dhat, L, A.eps);
    else active = vf_local<T, PROJ>(x, A.c, A.dhat, L, A.eps);
    A.term_e[p] = (double)L.f;
    if (!active) return;
    auto H = [&](int i, int j) { return L.H[i <= j ? hix(i, j) : hix(j, i)]; };
    if (MODE >= MODE_GRAD && A.grad)
#pragma unroll
        for (int i = 0; i < K; ++i) atomicAdd(A.grad + 3 * (int64_t)vid[i / 3] + i % 3, L.g[i]);
    if (MODE == MODE_HVP) {
        T vl[K];
#pragma unroll
        for (int i = 0; i < K; ++i) vl[i] = A.v[3 * (int64_t)vid[i / 3] + i % 3];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            T y = -T(0);
#pragma unroll
            for (int j = 0; j < K; ++j) y += H(i, j) * vl[j];
            atomicAdd(A.hv + 3 * (int64_t)vid[i / 3] + i % 3, y);
        }
        return;
    }
    if (MODE != MODE_HESS || !A.bsr) return;
    auto add_block = [&](T *blk, int a, int b) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) atomicAdd(blk + 3 * r + s, H(3 * a + r, 3 * b + s));
    };
#pragma unroll
    for (int a = 0; a < NV; ++a) add_block(A.bsr + 9 * ((int64_t)A.rpx[vid[a]] + A.diag_off[vid[a]]), a, a);
    int k = 0;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = a + 1; b < NV; ++b, ++k) {  // (a, b) and (b, a), pair order of the candidates
            const int32_t *sl = A.slot + (int64_t)NV * (NV - 1) * p + 2 * k;
            add_block(A.bsr + 9 * (int64_t)(sl[0] & 0x7fffffff), a, b);
            add_block(A.bsr + 9 * (int64_t)(sl[1] & 0x7fffffff), b, a);
        }
}

template <typename T>
__global__ void k_zero_new(int64_t n, const int32_t *blocks, T *bsr)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 9 * n) bsr[9 * (int64_t)blocks[k / 9] + k % 9] = T(0);
}

// term energies: fixed-order sum into the total, and each term's energy
// credited to the mesh of its first vertex
template <int THREADS>
__global__ void k_term_energy(int64_t n, int stride, const int32_t *verts, const double *term_e, int n_mesh,
                              const int64_t *v_off, double *e_mesh, double *e_total)
{
    double s = 0.0;
    for (int64_t p = threadIdx.x; p < n; p += THREADS) {
        s += term_e[p];
        if (e_mesh && term_e[p] != 0.0) {
            int64_t lo = 0, hi = n_mesh;  // mesh k with v_off[k] <= i < v_off[k + 1]
            const int64_t i = verts[(int64_t)stride * p];
            while (hi - lo > 1) {
                const int64_t m = (lo + hi) >> 1;
                if (v_off[m] <= i) lo = m;
                else hi = m;
            }
            atomicAdd(&e_mesh[lo], term_e[p]);
        }
    }
    s = block_sum<THREADS>(s);
    if (threadIdx.x == 0 && e_total) *e_total += s;
}

template <typename T, int NV>
void launch_contact(const ContactArgs<T> &A, int mode, bool proj, cudaStream_t s)
{
    const int nb = blocks_for(A.n);
    if (mode == MODE_VALUE) k_contact<T, NV, MODE_VALUE, false><<<nb, kDynThreads, 0, s>>>(A);
    else if (mode == MODE_GRAD) k_contact<T, NV, MODE_GRAD, false><<<nb, kDynThreads, 0, s>>>(A);
    else if (mode == MODE_HESS && proj) k_contact<T, NV, MODE_HESS, true><<<nb, kDynThreads, 0, s>>>(A);
    else if (mode == MODE_HESS) k_contact<T, NV, MODE_HESS, false><<<nb, kDynThreads, 0, s>>>(A);
    else if (proj) k_contact<T, NV, MODE_HVP, true><<<nb, kDynThreads, 0, s>>>(A);
    else k_contact<T, NV, MODE_HVP, false><<<nb, kDynThreads, 0, s>>>(A);
}

template <typename T>
adm_status eval_contacts(adm_ctx *h, const EvalArgs &a, int mode)
{
    Interactions &I = h->inter;
    cudaStream_t s = a.stream;
    if (mode == MODE_HESS && a.bsr && I.n_new > 0)
        k_zero_new<T><<<blocks_for(9 * I.n_new), kDynThreads, 0, s>>>(I.n_new, I.d_new, (T *)a.bsr);
    ContactArgs<T> A;
    A.rpx = I.d_rp[I.active];
    A.diag_off = I.d_diag_off;
    A.x = (const T *)a.x;
    A.v = (const T *)a.v;
    A.grad = (T *)a.grad;
    A.bsr = (T *)a.bsr;
    A.hv = (T *)a.hv;
    A.c = (T)(0.5 * I.kappa * I.area * I.h * I.h);
    A.dhat = (T)I.dhat;
    A.eps = (T)h->proj_eps;
    const bool proj = h->proj != 0;
    if (I.n_pairs > 0) {
        A.n = I.n_pairs;
        A.verts = I.d_cand;
        A.slot = I.d_slot;
        A.term_e = I.d_pair_e;
        launch_contact<T, 2>(A, mode, proj, s);
    }
    if (I.n_vf > 0) {
        A.n = I.n_vf;
        A.verts = I.d_quads;
        A.slot = I.d_slot + 2 * I.n_pairs;
        A.term_e = I.d_vf_e;
        launch_contact<T, 4>(A, mode, proj, s);
    }
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

}  // namespace

adm_status interactions_eval(adm_ctx *h, const EvalArgs &a, int mode)
{
    const Interactions &I = h->inter;
    if (I.kind < 0 || I.n_terms() == 0) return ADM_OK;
    if (h->m.vdim != 3) return ADM_ERR_UNSUPPORTED;
    return a.prec == ADM_FP32 ? eval_contacts<float>(h, a, mode) : eval_contacts<double>(h, a, mode);
}

adm_status interactions_energy(adm_ctx *h, const EvalArgs &a)
{
    const Interactions &I = h->inter;
    if (I.kind < 0 || I.n_terms() == 0 || (!a.energy_total && !a.energy_per_mesh)) return ADM_OK;
    if (I.n_pairs > 0)
        k_term_energy<1024><<<1, 1024, 0, a.stream>>>(I.n_pairs, 2, I.d_cand, I.d_pair_e, h->m.n_mesh, I.d_v_off,
                                                       a.energy_per_mesh, a.energy_total);
    if (I.n_vf > 0)
        k_term_energy<1024><<<1, 1024, 0, a.stream>>>(I.n_vf, 4, I.d_quads, I.d_vf_e, h->m.n_mesh, I.d_v_off,
                                                       a.energy_per_mesh, a.energy_total);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status interactions_retile(adm_ctx *h, int kind, cudaStream_t s)
{
    Interactions &I = h->inter;
    if (I.kind != kind || !I.d_rp[I.active]) return ADM_OK;
    const Pattern &P = h->pat[kind];
    TileSet &ts = h->tiles[kind];
    if (!ts.built) return ADM_OK;
    // the tiles' shared blocks as (row, offset in the mesh row), once per tile
    // build (the tile build has just uploaded them as mesh-pattern indices);
    // then their indices in the active pattern
    const int64_t nz = (int64_t)ts.zero_blocks.size();
    if (I.zero_for_build != ts.build_id) {
        release(h, I.d_zero_row);
        release(h, I.d_zero_off);
        I.d_zero_row = I.d_zero_off = nullptr;
        adm_status st;
        if ((st = alloc(h, &I.d_zero_row, nz * 4)) != ADM_OK) return st;
        if ((st = alloc(h, &I.d_zero_off, nz * 4)) != ADM_OK) return st;
        if (nz)
            k_block_rows<<<blocks_for(nz), kDynThreads, 0, s>>>(nz, ts.d_zero_blocks, h->m.nV, P.d_row_ptr,
                                                                 I.d_zero_row, I.d_zero_off);
        I.zero_for_build = ts.build_id;
    }
    const int32_t *rpx = I.d_rp[I.active];
    k_remap_tiles<<<ts.n_tiles, 256, 0, s>>>(ts.n_tiles, ts.d_hdr, ts.d_foot, ts.d_meta_off, ts.d_meta, rpx);
    if (nz)
        k_remap_zero<<<blocks_for((int64_t)nz), kDynThreads, 0, s>>>((int64_t)nz, I.d_zero_row, I.d_zero_off, rpx,
                                                                      ts.d_zero_blocks);
    return cudaStreamSynchronize(s) == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

// device buffer of at least n elements (contents not kept when it grows)
template <typename P>
adm_status ensure(adm_ctx *h, P **buf, int64_t &cap, int64_t n)
{
    if (n <= cap && *buf) return ADM_OK;
    release(h, *buf);
    *buf = nullptr;
    cap = 0;
    adm_status st = alloc(h, buf, (size_t)std::max<int64_t>(n, 1) * sizeof(P));
    if (st == ADM_OK) cap = std::max<int64_t>(n, 1);
    return st;
}

adm_status interactions_set(adm_ctx *h, int kind, const int32_t *pairs, int64_t n, const int32_t *quads, int64_t nq,
                            double kappa, double dhat, double area, double hstep, cudaStream_t s)
{
    Interactions &I = h->inter;
    const Pattern &P = h->pat[kind];
    TileSet &ts = h->tiles[kind];
    const int64_t nV = h->m.nV;
    if (!P.built || !ts.built) return ADM_ERR_ARG;
    adm_status st;
    // one-time data of this pattern kind
    if (I.kind != kind) {
        if (I.kind >= 0) return ADM_ERR_UNSUPPORTED;  // one pattern kind per handle
        if ((st = alloc(h, &I.d_diag_off, nV * 4)) != ADM_OK) return st;
        if ((st = alloc(h, &I.d_v_off, (h->m.n_mesh + 1) * 8)) != ADM_OK) return st;
        if ((st = alloc(h, &I.d_cnt, (nV + 1) * 4)) != ADM_OK) return st;
        if ((st = alloc(h, &I.d_acc, nV * 4)) != ADM_OK) return st;
        if ((st = alloc(h, &I.d_rp_tmp, (nV + 1) * 4)) != ADM_OK) return st;
        const int nsb = blocks_for(nV + 1, kDynThreads * kScanItems);
        if ((st = alloc(h, &I.d_bsum, nsb * 4)) != ADM_OK) return st;
        for (int b = 0; b < 2; ++b)
            if ((st = alloc(h, &I.d_rp[b], (nV + 1) * 4)) != ADM_OK) return st;
        if (cudaMemcpyAsync(I.d_v_off, h->m.v_off.data(), (h->m.n_mesh + 1) * 8, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return ADM_ERR_CUDA;
        k_diag_off<<<blocks_for(nV), kDynThreads, 0, s>>>(nV, P.d_row_ptr, P.d_col, I.d_diag_off);
        I.kind = kind;
    }
    // room for the terms, their candidate pairs and the extended pattern
    // (the inactive buffer); the pattern before deduplication bounds the final one
    const int64_t nc = n + 6 * nq;
    if (P.nnzb + 2 * nc > (int64_t)INT32_MAX) return ADM_ERR_ARG;  // block indices are int32
    const int nxt = 1 - I.active;
    if ((st = ensure(h, &I.d_cand, I.cap_cand, 2 * nc)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_slot, I.cap_slot, 2 * nc)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_pair_e, I.cap_pairs, n)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_quads, I.cap_vf, 4 * nq)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_vf_e, I.cap_vf_e, nq)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_new, I.cap_new, 2 * nc)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_col_tmp, I.cap_col_tmp, P.nnzb + 2 * nc)) != ADM_OK) return st;
    if ((st = ensure(h, &I.d_col[nxt], I.col_cap[nxt], P.nnzb + 2 * nc)) != ADM_OK) return st;
    if (n > 0 && cudaMemcpyAsync(I.d_cand, pairs, n * 8, cudaMemcpyDefault, s) != cudaSuccess) return ADM_ERR_CUDA;
    if (nq > 0 && cudaMemcpyAsync(I.d_quads, quads, nq * 16, cudaMemcpyDefault, s) != cudaSuccess)
        return ADM_ERR_CUDA;
    if (cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess) return ADM_ERR_CUDA;
    int32_t *rpx = I.d_rp[nxt], *colx = I.d_col[nxt];
    const int nsb = blocks_for(nV + 1, kDynThreads * kScanItems);
    auto scan = [&](int32_t *out) {
        k_scan_local<kDynThreads><<<nsb, kDynThreads, 0, s>>>(nV + 1, I.d_cnt, out, I.d_bsum);
        k_scan_sums<1024><<<1, 1024, 0, s>>>(nsb, I.d_bsum);
        k_scan_add<<<blocks_for(nV + 1), kDynThreads, 0, s>>>(nV + 1, out, I.d_bsum);
    };
    // (1) counts, (2) scan, (3) copy, (4) append; then sorted, deduplicated
    // tails, a second scan and copy, and the slots of every candidate
    if (nq > 0) k_quad_pairs<<<blocks_for(nq), kDynThreads, 0, s>>>(nq, I.d_quads, I.d_cand + 2 * n);
    k_row_len<<<blocks_for(nV + 1), kDynThreads, 0, s>>>(nV, P.d_row_ptr, I.d_cnt);
    if (nc > 0)
        k_count<<<blocks_for(nc), kDynThreads, 0, s>>>(nc, I.d_cand, nV, P.d_row_ptr, P.d_col, I.d_cnt, I.d_slot,
                                                        h->d_status);
    scan(I.d_rp_tmp);
    k_copy_rows<<<blocks_for(nV), kDynThreads, 0, s>>>(nV, P.d_row_ptr, P.d_col, I.d_rp_tmp, I.d_col_tmp, I.d_acc);
    if (nc > 0) k_append<<<blocks_for(nc), kDynThreads, 0, s>>>(nc, I.d_cand, I.d_slot, I.d_rp_tmp, I.d_acc,
                                                                 I.d_col_tmp);
    k_sort_tails<<<blocks_for(nV + 1), kDynThreads, 0, s>>>(nV, P.d_row_ptr, I.d_rp_tmp, I.d_col_tmp, I.d_cnt);
    scan(rpx);
    k_copy_unique<<<blocks_for(nV), kDynThreads, 0, s>>>(nV, P.d_row_ptr, I.d_rp_tmp, I.d_col_tmp, rpx, colx,
                                                          I.d_new);
    if (nc > 0) k_slots<<<blocks_for(nc), kDynThreads, 0, s>>>(nc, I.d_cand, P.d_row_ptr, rpx, colx, I.d_slot,
                                                        h->d_status);
    int32_t total = 0;
    int status = 0;
    if (cudaMemcpyAsync(&total, rpx + nV, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ADM_ERR_CUDA;
    if (status != 0) {  // an invalid vertex or a repeated one within a term: back to the mesh pattern
        if (nc > 0) interactions_set(h, kind, nullptr, 0, nullptr, 0, kappa, dhat, area, hstep, s);
        return ADM_ERR_ARG;
    }
    // switch: tiles follow the new pattern
    I.active = nxt;
    if ((st = interactions_retile(h, kind, s)) != ADM_OK) return st;
    I.nnzb = total;
    I.n_new = total - P.nnzb;
    I.n_pairs = n;
    I.n_vf = nq;
    I.kappa = kappa;
    I.dhat = dhat;
    I.area = area;
    I.h = hstep;
    return ADM_OK;
}

}  // namespace adm
