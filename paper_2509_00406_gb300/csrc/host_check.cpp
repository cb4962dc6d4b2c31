// host_check.cpp -- host-only entry points over the creation-time builders
// (hinges, block pattern, slot map, tiles), compiled with the C++ compiler
// alone into libadm_host.so so that their logic is testable without a GPU.
// They run the same code adm_create / the tiled assembler run; no CUDA call
// is made.
#include <chrono>
#include <cstring>
#include <unordered_map>

#include "internal.h"
// the device path's per-term filtering, compiled for the host as well (the
// math declarations come first: nvcc provides them implicitly)
#include <cmath>
#include "spd.cuh"
#include "terms.cuh"

using namespace adm;

namespace {

HostMesh make_mesh(const double *V, int64_t nV, const int32_t *F, int64_t nT, const int64_t *v_off,
                   const int64_t *f_off, int32_t n_mesh)
{
    HostMesh m;
    m.nV = nV;
    m.nT = nT;
    m.vdim = 3;
    m.n_mesh = n_mesh;
    m.V.assign(V, V + 3 * nV);
    m.F.assign(F, F + 3 * nT);
    m.v_off.assign(v_off, v_off + n_mesh + 1);
    m.f_off.assign(f_off, f_off + n_mesh + 1);
    return m;
}

}  // namespace

extern "C" {

// Builds hinges (if with_hinges), the block pattern and the tiles, and
// reports, per block of the pattern, which tile produces it:
//   block_writer[b] = tile id if exactly one tile produces it (written with a
//   plain store), -2 if several do (the lowest stores, the others write
//   partial slots that the fix-up adds in tile order), -1 if no tile does;
//   block_adds[b] = number of tiles producing a shared block (0 otherwise).
// stats: {n_tiles, partial slots (vertex + pair), n_zero_verts, FP64
// Hessian-mode shared-memory bytes (VD = 3), nnzb, nH, build_ms, largest
// slot table of a tile, FP32 Hessian-mode shared-memory bytes (VD = 3)}
// (9 entries).  Returns 0 or an adm_status, or a negative code
// < -99 naming the check that failed.
int adm_host_tile_check(const double *V, int64_t nV, const int32_t *F, int64_t nT, const int64_t *v_off,
                        const int64_t *f_off, int32_t n_mesh, int32_t with_hinges, int32_t tile_tris,
                        int32_t *block_writer, int32_t *block_adds, int64_t nnzb_cap, double *stats)
{
    HostMesh m = make_mesh(V, nV, F, nT, v_off, f_off, n_mesh);
    adm_status s = mesh_validate(m);
    if (s != ADM_OK) return s;
    mesh_rest_triangles(m);
    if (with_hinges && (s = mesh_build_hinges(m)) != ADM_OK) return s;
    Pattern P;
    mesh_build_pattern(m, with_hinges != 0, P.row_ptr, P.col);
    P.nnzb = (int64_t)P.col.size();
    if (P.nnzb > nnzb_cap) return ADM_ERR_ARG;
    TileSet ts;
    auto t0 = std::chrono::steady_clock::now();
    s = tiles_build(m, P, with_hinges != 0, tile_tris, ts);
    auto t1 = std::chrono::steady_clock::now();
    if (s != ADM_OK) return s;
    for (int64_t b = 0; b < P.nnzb; ++b) {
        block_writer[b] = -1;
        block_adds[b] = 0;
    }
    std::vector<int32_t> producers(P.nnzb, 0);
    if ((int64_t)ts.meta_off.size() != ts.n_tiles + 1 || ts.meta_off.back() != (int64_t)ts.meta.size()) return -105;
    // fix-up entries by output: vertex -> entry, block -> entry
    if (ts.fix_v.size() % 4 || ts.fix_p.size() % 4) return -120;
    std::unordered_map<int32_t, int64_t> fixv;
    std::unordered_map<int64_t, int64_t> fixp;
    for (size_t i = 0; i < ts.fix_v.size(); i += 4) {
        const int32_t v = ts.fix_v[i];
        if (v < 0 || v >= nV || P.col[P.row_ptr[v] + ts.fix_v[i + 1]] != v || !fixv.emplace(v, (int64_t)i).second)
            return -120;
    }
    for (size_t i = 0; i < ts.fix_p.size(); i += 4) {
        const int32_t v = ts.fix_p[i], pos = ts.fix_p[i + 1];
        if (v < 0 || v >= nV || pos < 0 || P.row_ptr[v] + pos >= P.row_ptr[v + 1]) return -120;
        if (!fixp.emplace((int64_t)P.row_ptr[v] + pos, (int64_t)i).second) return -120;
    }
    std::vector<int32_t> vslot_use(ts.n_vpart, 0), pslot_use(ts.n_ppart, 0);
    std::vector<int32_t> pslot_block(ts.n_ppart, -1);  // pair slot -> its block
    for (auto &f : fixp) {
        const int32_t n = ts.fix_p[f.second + 2], first = ts.fix_p[f.second + 3];
        if (n < 1 || first < 0 || first + n > ts.n_ppart) return -120;
        for (int32_t q = first; q < first + n; ++q) {
            if (pslot_block[q] >= 0) return -124;
            pslot_block[q] = (int32_t)f.first;
        }
    }
    for (size_t i = 0; i < ts.fix_v.size(); i += 4)
        if (ts.fix_v[i + 2] < 1 || ts.fix_v[i + 3] < 0 || ts.fix_v[i + 3] + ts.fix_v[i + 2] > ts.n_vpart) return -120;
    std::vector<int32_t> vprod(nV, 0);  // producers of each vertex row so far
    std::vector<std::vector<int32_t>> who(P.nnzb);  // producing tiles of each block, in order
    for (int32_t t = 0; t < ts.n_tiles; ++t) {
        const int32_t *hd = &ts.hdr[(size_t)kHdr * t];
        const int32_t fb = hd[kHdrFoot], nf = hd[kHdrNF], nvc = hd[kHdrNVC], npc = hd[kHdrNPC];
        const int64_t m0 = ts.meta_off[t];
        if (m0 % 16 != 0 || (ts.meta_off[t + 1] - m0) % 16 != 0) return -105;
        const unsigned char *blob = ts.meta.data() + m0;
        // every chunk of the tile is written by exactly one unit role
        std::vector<int> vw(nvc, 0), pw(npc, 0);
        for (int32_t i = 0; i < hd[kHdrNUnit]; ++i) {
            const int64_t u = (int64_t)hd[kHdrUnit] + i;
            const uint16_t *r = &ts.unit[8 * u];
            const uint16_t *d = &ts.unit_dst[6 * u];
            for (int q = 0; q < 3; ++q) {
                if (d[q] >= nvc || d[3 + q] >= npc) return -110;
                vw[d[q]]++;
                pw[d[3 + q]]++;
                if (r[q] >= nf) return -111;
            }
            for (int sl = 0; sl < (r[6] & 3); ++sl) {
                if (!with_hinges || r[3 + sl] == 0xffff) continue;
                if (r[3 + sl] >= nf) return -111;
                const uint16_t *sd = &ts.slot_dst[4 * ((int64_t)hd[kHdrSlot] + r[7] + sl)];
                if (sd[0] >= nvc) return -110;
                vw[sd[0]]++;
                for (int q = 0; q < 3; ++q) {
                    if (sd[1 + q] >= npc) return -110;
                    pw[sd[1 + q]]++;
                }
            }
        }
        for (int c : vw)
            if (c != 1) return -112;
        for (int c : pw)
            if (c != 1) return -112;
        // the tile's slot table: every entry is used by exactly one output
        const int32_t npart = hd[kHdrNPart];
        std::vector<int32_t> tab(npart);
        std::memcpy(tab.data(), blob + hd[kHdrPartOff], 4 * tab.size());
        std::vector<int> tab_use(npart, 0);
        // a later producer's slot is slot (producers so far - 1) of its
        // output's contiguous run; the lowest producer stores
        auto check_slot = [&](bool part, int idx, int64_t fix_i, const std::vector<int32_t> &fix, int32_t prior,
                              std::vector<int32_t> &use) -> int {
            if (!part) return prior == 0 ? 0 : -115;
            if (prior == 0 || fix_i < 0 || idx < 0 || idx >= npart) return -115;
            tab_use[idx]++;
            const int32_t n = fix[fix_i + 2], first = fix[fix_i + 3];
            if (prior > n || tab[idx] != first + prior - 1) return -121;
            use[tab[idx]]++;
            return 0;
        };
        // rows and pair codes: segments tile the chunk arrays; blocks produced
        int64_t vcov = 0;
        std::vector<int> pcov(npc, 0);
        for (int32_t r = 0; r < nf; ++r) {
            int32_t w[kRowWords];
            std::memcpy(w, blob + 4 * kRowWords * r, sizeof w);
            const int32_t v = ts.foot[fb + r];
            const int32_t rs = w[0] & 0x7fffffff;
            if (rs != P.row_ptr[v]) return -106;
            const int nv = (int)((uint32_t)w[1] >> 24);
            const int vs0 = w[2] & 0xffff;
            if (vs0 != vcov) return -113;  // vertex segments in footprint order, back to back
            vcov += nv;
            const int32_t bd = rs + (w[3] & 0x7fff);
            if (P.col[bd] != v) return -114;
            auto it = fixv.find(v);
            const int rc = check_slot((w[3] >> 15) & 1, w[3] >> 16, it == fixv.end() ? -1 : it->second, ts.fix_v,
                                      vprod[v], vslot_use);
            if (rc) return rc;
            vprod[v]++;
            who[bd].push_back(t);
        }
        // a pair code's block: (row, position) or, if partial, the output
        // whose slot run holds the table entry's slot
        auto block_of = [&](bool part, uint32_t d, int32_t row_v) -> int32_t {
            if (!part) {
                const int32_t r = (int32_t)(d >> 9);
                if (r >= nf) return -1;
                int32_t w0;
                std::memcpy(&w0, blob + 4 * kRowWords * r, 4);
                const int32_t b = w0 + (int32_t)(d & 511u);
                return (ts.foot[fb + r] == row_v && b < P.row_ptr[row_v + 1]) ? b : -1;
            }
            if ((int)d >= npart || tab[d] < 0 || tab[d] >= ts.n_ppart) return -1;
            const int32_t b = pslot_block[tab[d]];
            return (b >= P.row_ptr[row_v] && b < P.row_ptr[row_v + 1]) ? b : -1;
        };
        for (int j = 0; j < hd[kHdrNCode]; ++j) {
            uint32_t c[2];
            std::memcpy(c, blob + hd[kHdrCodeOff] + 8 * j, 8);
            const int start = (int)(c[0] & 0x1fffu), cnt = (int)((c[0] >> 13) & 15u);
            const bool pa = (c[0] >> 17) & 1u, pb = (c[0] >> 18) & 1u;
            const uint32_t da = ((c[0] >> 19) & 511u) << 9 | (c[1] & 511u);
            const uint32_t db = ((c[1] >> 9) & 511u) << 9 | ((c[1] >> 18) & 511u);
            if (pa != pb) return -115;  // both blocks of a pair have the same producers
            if (cnt == 0 || start + cnt > npc) return -118;
            for (int q = start; q < start + cnt; ++q) pcov[q]++;
            // the pair (va, vb), va < vb: rows of blocks A and B
            int32_t va, vb;
            if (!pa) {
                const int32_t lo = (int32_t)(da >> 9), hi = (int32_t)(db >> 9);
                if (lo >= nf || hi >= nf || lo >= hi) return -117;
                va = ts.foot[fb + lo];
                vb = ts.foot[fb + hi];
            } else {
                if ((int)da >= npart || (int)db >= npart || tab[da] < 0 || tab[da] >= ts.n_ppart || tab[db] < 0 ||
                    tab[db] >= ts.n_ppart)
                    return -121;
                const int32_t b1 = pslot_block[tab[da]], b2 = pslot_block[tab[db]];
                if (b1 < 0 || b2 < 0) return -121;
                vb = P.col[b1];
                va = P.col[b2];
                if (va >= vb) return -117;
            }
            const int32_t ba = block_of(pa, da, va), bb = block_of(pb, db, vb);
            if (ba < 0 || bb < 0 || P.col[ba] != vb || P.col[bb] != va) return -116;
            for (const auto &blk : {std::make_pair(ba, da), std::make_pair(bb, db)}) {
                const int32_t b = blk.first;
                auto it = fixp.find(b);
                const int rc = check_slot(pa, (int)blk.second, it == fixp.end() ? -1 : it->second, ts.fix_p,
                                          producers[b], pslot_use);
                if (rc) return rc;
                producers[b]++;
                who[b].push_back(t);
            }
        }
        if (vcov != nvc) return -113;
        for (int c : pcov)  // every pair chunk is summed by exactly one pair code
            if (c != 1) return -119;
        for (int c : tab_use)
            if (c != 1) return -122;
    }
    // every fix-up entry lists exactly the later producers of its output,
    // and every slot belongs to one output
    for (size_t i = 0; i < ts.fix_v.size(); i += 4)
        if (vprod[ts.fix_v[i]] != ts.fix_v[i + 2] + 1) return -123;
    for (auto &f : fixp)
        if (producers[f.first] != ts.fix_p[f.second + 2] + 1) return -123;
    for (int32_t c : vslot_use)
        if (c != 1) return -124;
    for (int32_t c : pslot_use)
        if (c != 1) return -124;
    // outputs with several producers all have fix-up entries
    for (int64_t v = 0; v < nV; ++v)
        if (vprod[v] > 1 && !fixv.count((int32_t)v)) return -123;
    for (int64_t b = 0; b < P.nnzb; ++b)
        if (producers[b] > 1 && !fixp.count(b)) return -123;
    for (int64_t v = 0; v < nV; ++v)  // the diagonal blocks: producers of the vertex row
        for (int32_t b = P.row_ptr[v]; b < P.row_ptr[v + 1]; ++b)
            if (P.col[b] == v) producers[b] = vprod[v];
    for (int64_t b = 0; b < P.nnzb; ++b) {
        if (producers[b] == 0) continue;
        block_writer[b] = producers[b] >= 2 ? -2 : who[b][0];
        block_adds[b] = producers[b] >= 2 ? producers[b] : 0;
    }
    // blocks of vertices no unit touches: the per-pass zero fill
    for (int32_t b : ts.zero_blocks) {
        if (block_writer[b] != -1) return -102;
        block_writer[b] = -2;
        block_adds[b] = 2;
    }
    stats[0] = ts.n_tiles;
    stats[1] = (double)(ts.n_vpart + ts.n_ppart);
    stats[2] = (double)ts.zero_verts.size();
    stats[3] = (double)tile_smem_bytes(ts, MODE_HESS, 3, 8);
    stats[4] = (double)P.nnzb;
    stats[5] = (double)m.nH();
    stats[6] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats[7] = (double)ts.max_part;
    stats[8] = (double)tile_smem_bytes(ts, MODE_HESS, 3, 4);
    // every triangle is exactly one unit
    std::vector<char> seen_t(nT, 0);
    for (int32_t e : ts.tri_perm)
        if (e < 0 || e >= nT || seen_t[e]++) return -103;
    // every hinge is in exactly one slot
    if (with_hinges) {
        std::vector<char> seen_h(m.nH(), 0);
        for (int32_t e : ts.slot_edge)
            if (e >= 0 && seen_h[e]++) return -104;
        for (char c : seen_h)
            if (!c) return -104;
    }
    return 0;
}

// tcgen05 operand layout and instruction descriptor (internal.h): every
// element of a rows x k BF16 operand (rows and k multiples of 8) maps to its
// own 2-byte slot inside rows * k * 2 bytes, every 8-element row piece starts
// on a 16-byte boundary, and the descriptor of a 128 x 64 tile carries the
// formats, majorness, N and M where the kernel's MMAs read them.  Returns 0,
// or the number of the check that failed.
int adm_host_umma_check(int32_t rows, int32_t k)
{
    if (rows <= 0 || k <= 0 || rows % 8 || k % 8) return 9;
    const uint32_t lbo = (uint32_t)(rows / 8) * 128u, bytes = (uint32_t)rows * (uint32_t)k * 2u;
    std::vector<char> seen(bytes, 0);
    for (int r = 0; r < rows; ++r)
        for (int kk = 0; kk < k; ++kk) {
            const uint32_t o = umma_canon(r, kk, lbo);
            if (o % 2 || o + 2 > bytes) return 1;
            if (seen[o]++) return 2;
            if (kk % 8 == 0 && o % 16) return 3;
        }
    const uint32_t d = umma_idesc_bf16(128, 64);
    if (((d >> 4) & 3u) != 1 || ((d >> 7) & 7u) != 1 || ((d >> 10) & 7u) != 1 || ((d >> 13) & 15u) != 0 ||
        ((d >> 17) & 63u) != 64 / 8 || ((d >> 24) & 31u) != 128 / 16)
        return 4;
    return 0;
}

// Per-term Hessian filtering of the filtered passes (spd.cuh: edge metric,
// shifted-Cholesky test, round-robin Jacobi, clamp), run on the host on one
// term's Hessian in its edge vectors He (packed upper: 45 reals for a hinge,
// 21 for a triangle in 3D), in place, in FP64 (prec 0) or in FP32 (prec 1,
// He rounded to float first).  kind 0: hinge, 1: triangle in 3D.  Returns 0,
// or 9 for a bad kind or precision.
int adm_host_project_edges(int32_t kind, int32_t prec, double *He, double eps)
{
    auto run = [&](auto real, auto edges) {
        using T = decltype(real);
        using E = decltype(edges);
        constexpr int N = E::NE * 3, NP = N * (N + 1) / 2;
        T h[NP];
        for (int k = 0; k < NP; ++k) h[k] = (T)He[k];
        project_edges<E, 3>(h, (T)eps);
        for (int k = 0; k < NP; ++k) He[k] = (double)h[k];
    };
    if (kind == 0 && prec == 0) run(double{}, HingeEdges{});
    else if (kind == 0 && prec == 1) run(float{}, HingeEdges{});
    else if (kind == 1 && prec == 0) run(double{}, TriEdges{});
    else if (kind == 1 && prec == 1) run(float{}, TriEdges{});
    else return 9;
    return 0;
}

// The device's per-element forward mode (terms.cuh), compiled for the host:
// one triangle term -- kind 0 StVK membrane, 1 Neo-Hookean membrane (x: 9
// reals), 2 symmetric Dirichlet in 2D (x: 6 reals) -- with Dinv the rest
// edges' inverse (2x2 row-major), the rest area and E, nu, thickness (the
// membranes), or one dihedral hinge (x: 12 reals, rest angle, weight w of
// w (theta - thetabar)^2); evaluated in its edge vectors in FP64 (prec 0) or
// FP32 (prec 1), then expanded to vertex coordinates by the accessors the
// kernels write their chunks with: energy, gradient (k) and Hessian (k x k,
// row-major).  Returns 0, 1 outside the term's domain, 9 for a bad kind or
// precision.
int adm_host_tri_local(int32_t kind, int32_t prec, const double *xin, const double *Dinv, double area, double E,
                       double nu, double thick, double *f, double *g, double *H)
{
    const double mu = E / (2.0 * (1.0 + nu)), lam = E * nu / (1.0 - nu * nu);
    auto out = [&](const auto &L, int k) {
        *f = (double)local_f(L);
        for (int i = 0; i < k; ++i) g[i] = (double)local_g(L, i);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) H[k * i + j] = (double)local_H(L, i, j);
    };
    auto run = [&](auto real) {
        using T = decltype(real);
        T D[4];
        for (int q = 0; q < 4; ++q) D[q] = (T)Dinv[q];
        if (kind == 2) {
            T x[6];
            for (int q = 0; q < 6; ++q) x[q] = (T)xin[q];
            EdgeLocal<TriEdges, 2, T> L;
            const T det = uv_local<T, PsiSymDir<T>, false>(x, D, PsiSymDir<T>{(T)area}, L);
            out(L, 6);
            return det > T(0) && std::isfinite(*f);
        }
        T x[9];
        for (int q = 0; q < 9; ++q) x[q] = (T)xin[q];
        EdgeLocal<TriEdges, 3, T> L;
        if (kind == 0) membrane_local<T, PsiStVK<T>, false>(x, D, PsiStVK<T>{(T)mu, (T)lam, (T)(thick * area)}, L);
        else membrane_local<T, PsiNH<T>, false>(x, D, PsiNH<T>{(T)mu, (T)lam, (T)(thick * area)}, L);
        out(L, 9);
        return (bool)std::isfinite(*f);
    };
    if ((prec != 0 && prec != 1) || kind < 0 || kind > 2) return 9;
    const bool ok = prec == 0 ? run(double{}) : run(float{});
    return ok ? 0 : 1;
}

int adm_host_hinge_local(int32_t prec, const double *x12, double thetabar, double w, double *f, double *g, double *H)
{
    auto run = [&](auto real) {
        using T = decltype(real);
        T x[12];
        for (int k = 0; k < 12; ++k) x[k] = (T)x12[k];
        EdgeLocal<HingeEdges, 3, T> L;
        const bool ok = hinge_local<T, false>(x, (T)thetabar, (T)w, L, T(0));
        *f = (double)local_f(L);
        for (int i = 0; i < 12; ++i) g[i] = (double)local_g(L, i);
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) H[12 * i + j] = (double)local_H(L, i, j);
        return ok && std::isfinite(*f);
    };
    if (prec != 0 && prec != 1) return 9;
    const bool ok = prec == 0 ? run(double{}) : run(float{});
    return ok ? 0 : 1;
}

}  // extern "C"
