// tiles.cpp -- host construction of the shared-memory tiles of the tiled
// assembler.
//
// The paper evaluates each term over RXMesh patches staged in shared memory
// (Sec. 2.4, Sec. 5.2) and scatters with global atomics (Sec. 5.5).  Here a
// tile is a run of about `tile_tris` triangles in Morton order of their rest
// centroids (per mesh, never across meshes) plus the hinges whose face A is
// one of them.  A tile stages the positions of its footprint vertices,
// accumulates gradient and Hessian contributions of all its elements in
// shared memory (diagonal blocks as 6 unique entries, one 3x3 block per
// unordered vertex pair), and writes every BSR row of its footprint with
// row-contiguous stores.  Blocks and gradient rows that also receive
// contributions from another tile are "shared": they are zeroed before the
// pass and written with global atomic additions; all others are written once
// with plain stores.
#include <algorithm>
#include <array>
#include <map>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace adm {

static uint32_t spread3(uint32_t v)
{
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000ff;
    v = (v | (v << 8)) & 0x0300f00f;
    v = (v | (v << 4)) & 0x030c30c3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
}

// triangle order of one mesh: Morton code of the rest centroid in the mesh's
// bounding box, ties by index
static void morton_order(const HostMesh &m, int64_t t0, int64_t t1, std::vector<int32_t> &out)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    std::vector<std::array<double, 3>> c(t1 - t0);
    for (int64_t t = t0; t < t1; ++t) {
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += m.V[3 * (int64_t)m.F[3 * t + k] + d];
            c[t - t0][d] = s / 3.0;
            lo[d] = std::min(lo[d], c[t - t0][d]);
            hi[d] = std::max(hi[d], c[t - t0][d]);
        }
    }
    std::vector<std::pair<uint32_t, int32_t>> key(t1 - t0);
    for (int64_t t = t0; t < t1; ++t) {
        uint32_t q[3];
        for (int d = 0; d < 3; ++d) {
            double span = hi[d] - lo[d];
            double u = span > 0 ? (c[t - t0][d] - lo[d]) / span : 0.0;
            q[d] = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(u * 1024.0)));
        }
        key[t - t0] = {spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2), (int32_t)t};
    }
    std::sort(key.begin(), key.end());
    for (auto &k : key) out.push_back(k.second);
}

adm_status tiles_build(const HostMesh &m, const Pattern &P, bool with_hinges, int tile_tris, TileSet &ts)
{
    const int64_t nT = m.nT, nH = with_hinges ? m.nH() : 0;
    ts = TileSet();
    ts.tile_tris = tile_tris;
    // ---- triangle order and tiles (never across meshes)
    std::vector<int32_t> order;
    order.reserve(nT);
    std::vector<int64_t> tile_tri_off(1, 0);
    std::vector<int32_t> tile_mesh;
    ts.mesh_tile_off.assign(m.n_mesh + 1, 0);
    // face -> faces across its edges, to count the hinge footprint of a
    // candidate tile (a hinge belongs to the tile of its face A)
    std::vector<int32_t> hinges_of_face;
    std::vector<int64_t> hof_off;
    if (with_hinges) {
        hof_off.assign(nT + 1, 0);
        for (int64_t h = 0; h < m.nH(); ++h) hof_off[m.H_face[h] + 1]++;
        for (int64_t t = 0; t < nT; ++t) hof_off[t + 1] += hof_off[t];
        hinges_of_face.resize(m.nH());
        std::vector<int64_t> pos(hof_off.begin(), hof_off.end() - 1);
        for (int64_t h = 0; h < m.nH(); ++h) hinges_of_face[pos[m.H_face[h]]++] = (int32_t)h;
    }
    // shared-memory units (VD = 3) of the triangles order[a, b) plus their hinges
    std::vector<int32_t> fv;
    std::vector<std::pair<int32_t, int32_t>> pp;
    auto units = [&](int64_t a, int64_t b) -> int64_t {
        fv.clear();
        pp.clear();
        auto add = [&](const int32_t *q, int n) {
            for (int i = 0; i < n; ++i) {
                fv.push_back(q[i]);
                for (int j = i + 1; j < n; ++j) pp.emplace_back(std::min(q[i], q[j]), std::max(q[i], q[j]));
            }
        };
        for (int64_t i = a; i < b; ++i) {
            add(&m.F[3 * (int64_t)order[i]], 3);
            if (with_hinges)
                for (int64_t k = hof_off[order[i]]; k < hof_off[order[i] + 1]; ++k)
                    add(&m.H[4 * (int64_t)hinges_of_face[k]], 4);
        }
        std::sort(fv.begin(), fv.end());
        std::sort(pp.begin(), pp.end());
        int64_t nf = std::unique(fv.begin(), fv.end()) - fv.begin();
        int64_t np = std::unique(pp.begin(), pp.end()) - pp.begin();
        return 12 * nf + 9 * np;
    };
    // tiles must fit the shared memory of the FP64 kernel; larger ones split
    const int64_t budget = (227 * 1024) / 8;
    for (int k = 0; k < m.n_mesh; ++k) {
        int64_t a = m.f_off[k], b = m.f_off[k + 1];
        size_t base = order.size();
        morton_order(m, a, b, order);
        int64_t n = b - a;
        int64_t ntile = (n + tile_tris - 1) / tile_tris;
        std::vector<std::pair<int64_t, int64_t>> stack;
        for (int64_t i = ntile - 1; i >= 0; --i)  // balanced split, processed in order
            stack.emplace_back((int64_t)base + (n * i) / ntile, (int64_t)base + (n * (i + 1)) / ntile);
        while (!stack.empty()) {
            auto [s0, s1] = stack.back();
            stack.pop_back();
            if (s1 - s0 > 1 && units(s0, s1) > budget) {
                int64_t mid = (s0 + s1) / 2;
                stack.emplace_back(mid, s1);
                stack.emplace_back(s0, mid);
                continue;
            }
            tile_tri_off.push_back(s1);
            tile_mesh.push_back(k);
        }
        ts.mesh_tile_off[k + 1] = (int32_t)tile_mesh.size();
    }
    const int32_t n_tiles = (int32_t)tile_mesh.size();
    ts.n_tiles = n_tiles;
    std::vector<int32_t> tri_tile(nT);
    for (int32_t t = 0; t < n_tiles; ++t)
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i) tri_tile[order[i]] = t;
    // ---- hinges grouped by the tile of face A (canonical order inside a tile)
    std::vector<int64_t> tile_hinge_off(n_tiles + 1, 0);
    std::vector<int32_t> horder(nH);
    for (int64_t h = 0; h < nH; ++h) tile_hinge_off[tri_tile[m.H_face[h]] + 1]++;
    for (int32_t t = 0; t < n_tiles; ++t) tile_hinge_off[t + 1] += tile_hinge_off[t];
    {
        std::vector<int64_t> pos(tile_hinge_off.begin(), tile_hinge_off.end() - 1);
        for (int64_t h = 0; h < nH; ++h) horder[pos[tri_tile[m.H_face[h]]]++] = (int32_t)h;
    }
    // ---- global ownership of blocks and gradient rows: owner tile or -2 if shared
    std::vector<int32_t> blk_owner(P.nnzb, -1), v_owner(m.nV, -1);
    auto touch_block = [&](int32_t blk, int32_t t) {
        int32_t &o = blk_owner[blk];
        o = (o == -1 || o == t) ? t : -2;
    };
    auto touch_v = [&](int32_t v, int32_t t) {
        int32_t &o = v_owner[v];
        o = (o == -1 || o == t) ? t : -2;
    };
    auto block_of = [&](int32_t i, int32_t j) -> int32_t {
        auto b = P.col.begin() + P.row_ptr[i], e = P.col.begin() + P.row_ptr[i + 1];
        return (int32_t)(std::lower_bound(b, e, j) - P.col.begin());
    };
    for (int64_t t = 0; t < nT; ++t) {
        const int32_t *f = &m.F[3 * t];
        for (int a = 0; a < 3; ++a) {
            touch_v(f[a], tri_tile[t]);
            for (int b = 0; b < 3; ++b) touch_block(block_of(f[a], f[b]), tri_tile[t]);
        }
    }
    for (int64_t h = 0; h < nH; ++h) {
        const int32_t *q = &m.H[4 * h];
        int32_t t = tri_tile[m.H_face[h]];
        for (int a = 0; a < 4; ++a) {
            touch_v(q[a], t);
            for (int b = 0; b < 4; ++b) touch_block(block_of(q[a], q[b]), t);
        }
    }
    // ---- per tile: footprint, pair slots, element local data, row codes
    ts.hdr.assign((size_t)n_tiles * 8, 0);
    ts.tri_loc.resize(nT * 6);
    ts.hinge_loc.resize(nH * 10);
    ts.tri_perm.resize(nT);
    ts.hinge_perm.resize(nH);
    int64_t max_smem_units = 0, max_smem_units2 = 0;
    std::vector<int32_t> foot;
    std::vector<int32_t> lid(m.nV, -1);
    std::map<std::pair<int32_t, int32_t>, int32_t> pair_slot;
    for (int32_t t = 0; t < n_tiles; ++t) {
        foot.clear();
        pair_slot.clear();
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i)
            for (int a = 0; a < 3; ++a) foot.push_back(m.F[3 * (int64_t)order[i] + a]);
        for (int64_t i = tile_hinge_off[t]; i < tile_hinge_off[t + 1]; ++i)
            for (int a = 0; a < 4; ++a) foot.push_back(m.H[4 * (int64_t)horder[i] + a]);
        std::sort(foot.begin(), foot.end());
        foot.erase(std::unique(foot.begin(), foot.end()), foot.end());
        if (foot.size() > 65535) return ADM_ERR_UNSUPPORTED;
        for (size_t r = 0; r < foot.size(); ++r) lid[foot[r]] = (int32_t)r;
        auto slot = [&](int32_t la, int32_t lb) -> int32_t {
            auto key = std::make_pair(std::min(la, lb), std::max(la, lb));
            auto it = pair_slot.find(key);
            if (it != pair_slot.end()) return it->second;
            int32_t s = (int32_t)pair_slot.size();
            pair_slot.emplace(key, s);
            return s;
        };
        static const int TP[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        static const int HP[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i) {
            const int32_t *f = &m.F[3 * (int64_t)order[i]];
            ts.tri_perm[i] = order[i];
            for (int a = 0; a < 3; ++a) ts.tri_loc[6 * i + a] = (uint16_t)lid[f[a]];
            for (int p = 0; p < 3; ++p) ts.tri_loc[6 * i + 3 + p] = 0;  // filled after slot renumbering
        }
        for (int64_t i = tile_hinge_off[t]; i < tile_hinge_off[t + 1]; ++i) {
            const int32_t *q = &m.H[4 * (int64_t)horder[i]];
            ts.hinge_perm[i] = horder[i];
            for (int a = 0; a < 4; ++a) ts.hinge_loc[10 * i + a] = (uint16_t)lid[q[a]];
        }
        // pair slots numbered in (lo, hi) order so that the accumulator walks
        // rows in order
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i)
            for (int p = 0; p < 3; ++p) slot(ts.tri_loc[6 * i + TP[p][0]], ts.tri_loc[6 * i + TP[p][1]]);
        for (int64_t i = tile_hinge_off[t]; i < tile_hinge_off[t + 1]; ++i)
            for (int p = 0; p < 6; ++p) slot(ts.hinge_loc[10 * i + HP[p][0]], ts.hinge_loc[10 * i + HP[p][1]]);
        {
            int32_t s = 0;
            for (auto &kv : pair_slot) kv.second = s++;  // std::map iterates in (lo, hi) order
        }
        if (pair_slot.size() > 8191) return ADM_ERR_UNSUPPORTED;
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i)
            for (int p = 0; p < 3; ++p)
                ts.tri_loc[6 * i + 3 + p] = (uint16_t)slot(ts.tri_loc[6 * i + TP[p][0]], ts.tri_loc[6 * i + TP[p][1]]);
        for (int64_t i = tile_hinge_off[t]; i < tile_hinge_off[t + 1]; ++i)
            for (int p = 0; p < 6; ++p)
                ts.hinge_loc[10 * i + 4 + p] =
                    (uint16_t)slot(ts.hinge_loc[10 * i + HP[p][0]], ts.hinge_loc[10 * i + HP[p][1]]);
        // row codes: for every footprint row, every block of its BSR row
        const int32_t foot_begin = (int32_t)ts.foot.size();
        const int32_t code_begin = (int32_t)ts.codes.size();
        for (size_t r = 0; r < foot.size(); ++r) {
            const int32_t v = foot[r];
            ts.foot.push_back(v);
            uint32_t rs = (uint32_t)P.row_ptr[v];
            if (v_owner[v] == -2) rs |= 0x80000000u;
            ts.row_start.push_back((int32_t)rs);
            ts.code_off.push_back((int32_t)ts.codes.size());
            for (int32_t b = P.row_ptr[v]; b < P.row_ptr[v + 1]; ++b) {
                const int32_t c = P.col[b];
                const int32_t lc = lid[c];
                uint16_t code = 0;  // kind 0: not produced by this tile
                if (lc >= 0 && blk_owner[b] != -1) {
                    const bool mine = blk_owner[b] == t || blk_owner[b] == -2;
                    if (lc == (int32_t)r) {
                        code = (uint16_t)(1u << 14);  // diagonal, slot = row
                    } else {
                        auto it = pair_slot.find(std::make_pair(std::min<int32_t>(lc, (int32_t)r),
                                                                std::max<int32_t>(lc, (int32_t)r)));
                        if (it != pair_slot.end())
                            code = (uint16_t)(((int32_t)r < lc ? 2u : 3u) << 14 | (uint32_t)it->second);
                    }
                    if (!mine) code = 0;
                    if (code && blk_owner[b] == -2) code |= (uint16_t)(1u << 13);
                }
                ts.codes.push_back(code);
            }
        }
        ts.code_off.push_back((int32_t)ts.codes.size());  // sentinel of the tile's last row
        int32_t *hd = &ts.hdr[8 * (size_t)t];
        hd[0] = (int32_t)tile_tri_off[t];
        hd[1] = (int32_t)(tile_tri_off[t + 1] - tile_tri_off[t]);
        hd[2] = (int32_t)tile_hinge_off[t];
        hd[3] = (int32_t)(tile_hinge_off[t + 1] - tile_hinge_off[t]);
        hd[4] = foot_begin;
        hd[5] = (int32_t)foot.size();
        hd[6] = (int32_t)pair_slot.size();
        hd[7] = code_begin;
        // shared-memory accumulator units: x (3) + grad (3) + diag (6) per
        // footprint vertex, 9 per pair
        max_smem_units = std::max<int64_t>(max_smem_units, 12 * (int64_t)foot.size() + 9 * (int64_t)pair_slot.size());
        max_smem_units2 = std::max<int64_t>(max_smem_units2, 7 * (int64_t)foot.size() + 4 * (int64_t)pair_slot.size());
        for (int32_t v : foot) lid[v] = -1;
    }
    // code_off has one sentinel per tile: index of footprint row r of tile t is
    // foot_begin + r + t (the t sentinels before it)
    ts.max_smem_units = max_smem_units;
    ts.max_smem_units2 = max_smem_units2;
    // ---- shared outputs zeroed before every pass
    for (int64_t b = 0; b < P.nnzb; ++b)
        if (blk_owner[b] == -2) ts.zero_blocks.push_back((int32_t)b);
    for (int64_t v = 0; v < m.nV; ++v)
        if (v_owner[v] == -2) ts.zero_verts.push_back((int32_t)v);
    ts.built = true;
    return ADM_OK;
}

}  // namespace adm
