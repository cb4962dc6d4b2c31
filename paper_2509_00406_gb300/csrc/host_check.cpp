// host_check.cpp -- host-only entry points over the creation-time builders
// (hinges, block pattern, slot map, tiles), compiled with the C++ compiler
// alone into libadm_host.so so that their logic is testable without a GPU.
// They run the same code adm_create / the tiled assembler run; no CUDA call
// is made.
#include <chrono>
#include <cstring>

#include "internal.h"

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
//   plain store), -2 if several do (the lowest stores, the others add in tile
//   order), -1 if no tile does; block_adds[b] = number of tiles producing a
//   shared block (0 otherwise).
// stats: {n_tiles, wait edges (tile, lower tile), n_zero_verts, FP64
// Hessian-mode shared-memory bytes (VD = 3), nnzb, nH, build_ms, most lower
// tiles one tile waits for}.  Returns 0 or an
// adm_status, or a negative code < -99 naming the check that failed.
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
    int64_t n_wait_edges = 0;
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
        // the tiles this one waits for are lower tiles
        std::vector<int32_t> wl(hd[kHdrNWait]);
        std::memcpy(wl.data(), blob + hd[kHdrWaitOff], 4 * wl.size());
        for (int32_t w : wl)
            if (w < 0 || w >= t) return -121;
        n_wait_edges += (int64_t)wl.size();
        auto waits_for = [&](int32_t u) { return std::find(wl.begin(), wl.end(), u) != wl.end(); };
        // rows and codes: segments tile the chunk arrays; blocks produced
        int64_t vcov = 0;
        std::vector<int> pcov(npc, 0);
        std::vector<std::pair<int32_t, int>> mine;  // blocks this tile produces, with their rank
        for (int32_t r = 0; r < nf; ++r) {
            int32_t w[kRowWords];
            std::memcpy(w, blob + 4 * kRowWords * r, sizeof w);
            const int32_t v = ts.foot[fb + r];
            const int32_t rs = w[0] & 0x7fffffff;
            if (rs != P.row_ptr[v]) return -106;
            const int c0 = w[1] & 0xffff, nc = (w[1] >> 16) & 0xff, nv = (int)((uint32_t)w[1] >> 24);
            const int vs0 = w[2] & 0xffff;
            if (vs0 != vcov) return -113;  // vertex segments in footprint order, back to back
            vcov += nv;
            const int32_t bd = rs + (w[3] & 0xffff);
            if (P.col[bd] != v) return -114;
            mine.emplace_back(bd, w[3] >> 16);
            for (int c = c0; c < c0 + nc; ++c) {
                uint32_t code;
                std::memcpy(&code, blob + hd[kHdrCodeOff] + 4 * c, 4);
                const int start = (int)(code & 0x7fffu), cnt = (int)((code >> 15) & 15u);
                const int tr = (int)((code >> 19) & 1u), rank = (int)((code >> 20) & 7u);
                const int32_t b = rs + (int32_t)(code >> 23);
                if (b >= P.row_ptr[v + 1] || P.col[b] == v) return -116;
                const int32_t lc = (int32_t)(std::lower_bound(ts.foot.begin() + fb, ts.foot.begin() + fb + nf, P.col[b]) -
                                             (ts.foot.begin() + fb));
                if (lc >= nf || ts.foot[fb + lc] != P.col[b] || tr != (r > lc ? 1 : 0)) return -117;
                if (cnt == 0 || start + cnt > npc) return -118;
                for (int q = start; q < start + cnt; ++q) pcov[q]++;
                mine.emplace_back(b, rank);
            }
        }
        if (vcov != nvc) return -113;
        for (int c : pcov)  // every pair chunk is summed by its two blocks, (a, b) and (b, a)
            if (c != 2) return -119;
        // tiles are visited in order: a block of rank r in this tile has been
        // produced by exactly r lower tiles, all in this tile's wait list
        if (hd[kHdrRounds] < 1) return -123;
        for (auto &bm : mine) {
            const int32_t b = bm.first;
            if (bm.second != producers[b]) return -115;
            if (bm.second >= hd[kHdrRounds]) return -123;
            if (bm.second > 0)
                for (int32_t u : who[b])
                    if (!waits_for(u)) return -122;
            producers[b]++;
            who[b].push_back(t);
        }
    }
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
    stats[1] = (double)n_wait_edges;
    stats[2] = (double)ts.zero_verts.size();
    stats[3] = (double)tile_smem_bytes(ts, MODE_HESS, 3, 8);
    stats[4] = (double)P.nnzb;
    stats[5] = (double)m.nH();
    stats[6] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats[7] = (double)ts.max_wait;
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

}  // extern "C"
