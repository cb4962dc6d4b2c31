// tiles.cpp -- host construction of the shared-memory tiles of the tiled
// assembler.
//
// The paper evaluates each term over RXMesh patches staged in shared memory
// (Sec. 2.4, Sec. 5.2) and scatters with global atomics (Sec. 5.5).  Here a
// tile is a run of about `tile_tris` triangles in Morton order of their rest
// centroids (per mesh, never across meshes) plus the hinges whose face A is
// one of them.  A tile stages the positions of its footprint vertices,
// accumulates gradient and Hessian contributions of all its elements in
// shared memory (diagonal blocks as their upper-triangle entries, one block
// per unordered vertex pair), and writes every BSR row of its footprint with
// row-contiguous stores.  Blocks and gradient rows that also receive
// contributions from another tile are "shared": they are zeroed before the
// pass and written with global atomic additions; all others are written once
// with plain stores.  Tiles are built in parallel on the host.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "internal.h"

namespace adm {

namespace {

uint32_t spread3(uint32_t v)
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
void morton_order(const HostMesh &m, int64_t t0, int64_t t1, int32_t *out)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    std::vector<std::array<double, 3>> c(t1 - t0);
    for (int64_t t = t0; t < t1; ++t)
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += m.V[3 * (int64_t)m.F[3 * t + k] + d];
            c[t - t0][d] = s / 3.0;
            lo[d] = std::min(lo[d], c[t - t0][d]);
            hi[d] = std::max(hi[d], c[t - t0][d]);
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
    for (size_t i = 0; i < key.size(); ++i) out[i] = key[i].second;
}

unsigned worker_count() { return std::max(1u, std::min(16u, std::thread::hardware_concurrency())); }

template <class F>
void parallel_for(int64_t n, unsigned nt, F &&f)
{
    if (n < 64 || nt == 1) {
        for (int64_t i = 0; i < n; ++i) f(i, 0u);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (unsigned k = 0; k < nt; ++k)
        th.emplace_back([&, k] {
            for (int64_t i; (i = next.fetch_add(1)) < n;) f(i, k);
        });
    for (auto &t : th) t.join();
}

constexpr int TP[3][2] = {{0, 1}, {0, 2}, {1, 2}};
constexpr int HP[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// per-thread scratch: vertex -> local id map and an open-addressing set of
// local vertex pairs (keys lo << 16 | hi)
struct Work {
    std::vector<int32_t> lid;   // nV, -1 when unused
    std::vector<uint32_t> hkey; // 0xffffffff = empty
    std::vector<uint16_t> hval; // slot per key
    std::vector<uint32_t> hused;
    std::vector<int32_t> foot;
    std::vector<uint32_t> pairs;
    explicit Work(int64_t nV) : lid(nV, -1), hkey(1u << 16, 0xffffffffu), hval(1u << 16, 0) {}
    static uint32_t hash(uint32_t k) { return (k * 2654435761u) >> 16; }
    bool insert(uint32_t k)  // true if new
    {
        uint32_t h = hash(k);
        while (hkey[h] != 0xffffffffu) {
            if (hkey[h] == k) return false;
            h = (h + 1) & 0xffffu;
        }
        hkey[h] = k;
        hused.push_back(h);
        return true;
    }
    uint16_t &value(uint32_t k)
    {
        uint32_t h = hash(k);
        while (hkey[h] != k) h = (h + 1) & 0xffffu;
        return hval[h];
    }
    void clear_pairs()
    {
        for (uint32_t h : hused) hkey[h] = 0xffffffffu;
        hused.clear();
        pairs.clear();
    }
};

uint32_t pkey(uint32_t a, uint32_t b) { return a < b ? (a << 16 | b) : (b << 16 | a); }

// out[j] = in[m_j], where m_j runs over m mod q, then m div q, q = ceil(n / 32):
// stored neighbours are about n/32 apart in the input order.  Concurrent lanes
// then rarely accumulate into the same shared-memory entry, and each warp's
// loads stay contiguous.
void interleave32(const std::vector<int32_t> &in, int32_t *out)
{
    const int64_t n = (int64_t)in.size(), q = (n + 31) / 32;
    int64_t j = 0;
    for (int64_t r = 0; r < q; ++r)
        for (int64_t m = r; m < n; m += q) out[j++] = in[m];
}

// Warp groups with few shared-memory bank conflicts.  Element e of a tile has
// R "roles" (its vertices and its pairs, in their fixed order); in role r one
// warp instruction of the kernel touches, for each of its 32 lanes, the
// accumulator of that lane's element, whose bank is key[e][r] = (slot index)
// mod 32 (the accumulator strides are odd).  Consecutive runs of 32 stored
// elements are one warp's lanes, so the stored order is built group by group:
// each element, in the given order, joins the group (with room left) where
// its keys collide least with those already there.  Distinct banks also mean
// distinct addresses, so colliding float atomics retry less.
void bank_groups(int64_t n, int R, const std::vector<uint8_t> &key, std::vector<int32_t> &perm)
{
    const int64_t G = (n + 31) / 32;
    std::vector<uint8_t> occ((size_t)G * R * 32, 0);
    std::vector<int32_t> fill(G, 0);
    std::vector<std::vector<int32_t>> members(G);
    for (int64_t e = 0; e < n; ++e) {
        int64_t best = -1, best_c = 0;
        for (int64_t g = 0; g < G; ++g) {
            const int64_t capg = g + 1 < G ? 32 : n - 32 * (G - 1);
            if (fill[g] >= capg) continue;
            int64_t c = 0;
            for (int r = 0; r < R; ++r) c += occ[((size_t)g * R + r) * 32 + key[(size_t)e * R + r]];
            if (best < 0 || c < best_c) {
                best = g;
                best_c = c;
                if (c == 0) break;
            }
        }
        for (int r = 0; r < R; ++r) occ[((size_t)best * R + r) * 32 + key[(size_t)e * R + r]]++;
        fill[best]++;
        members[best].push_back((int32_t)e);
    }
    perm.clear();
    for (auto &m : members) perm.insert(perm.end(), m.begin(), m.end());
}

// reorder n records of W uint16 (and their permutation entries) by perm
void apply_order(const std::vector<int32_t> &perm, int W, uint16_t *loc, int32_t *elem_perm)
{
    const size_t n = perm.size();
    std::vector<uint16_t> l(loc, loc + n * W);
    std::vector<int32_t> ep(elem_perm, elem_perm + n);
    for (size_t j = 0; j < n; ++j) {
        for (int w = 0; w < W; ++w) loc[j * W + w] = l[(size_t)perm[j] * W + w];
        elem_perm[j] = ep[perm[j]];
    }
}

}  // namespace

int64_t tile_meta_bytes(int64_t nf, int64_t ncodes) { return (4 * nf + 2 * (nf + 1) + 2 * ncodes + 15) & ~int64_t(15); }

int64_t tile_smem_bytes(int elem_bytes, int64_t units, int64_t nf, int64_t ncodes)
{
    return ((elem_bytes * units + 15) & ~int64_t(15)) + tile_meta_bytes(nf, ncodes);
}

adm_status tiles_build(const HostMesh &m, const Pattern &P, bool with_hinges, int tile_tris, TileSet &ts)
{
    const int64_t nT = m.nT, nH = with_hinges ? m.nH() : 0;
    ts = TileSet();
    ts.tile_tris = tile_tris;
    // hinges by face A
    std::vector<int64_t> hof_off(nT + 1, 0);
    std::vector<int32_t> hinges_of_face(nH);
    for (int64_t h = 0; h < nH; ++h) hof_off[m.H_face[h] + 1]++;
    for (int64_t t = 0; t < nT; ++t) hof_off[t + 1] += hof_off[t];
    {
        std::vector<int64_t> pos(hof_off.begin(), hof_off.end() - 1);
        for (int64_t h = 0; h < nH; ++h) hinges_of_face[pos[m.H_face[h]]++] = (int32_t)h;
    }
    const unsigned nthr = worker_count();
    std::vector<Work> work;
    work.reserve(nthr);
    for (unsigned k = 0; k < nthr; ++k) work.emplace_back(m.nV);

    // shared-memory bytes of the FP64 kernel (VD = 3) for the triangles
    // order[a, b) and their hinges: accumulators plus the row metadata; a
    // tile whose rows hold 65,536 or more BSR blocks counts as too large
    std::vector<int32_t> order(nT);
    auto units = [&](Work &w, int64_t a, int64_t b) -> int64_t {
        w.foot.clear();
        w.clear_pairs();
        int64_t np = 0;
        auto add = [&](const int32_t *q, int n) {
            for (int i = 0; i < n; ++i)
                if (w.lid[q[i]] < 0) {
                    w.lid[q[i]] = (int32_t)w.foot.size();
                    w.foot.push_back(q[i]);
                }
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j) np += w.insert(pkey(w.lid[q[i]], w.lid[q[j]]));
        };
        for (int64_t i = a; i < b; ++i) {
            add(&m.F[3 * (int64_t)order[i]], 3);
            for (int64_t k = hof_off[order[i]]; k < hof_off[order[i] + 1]; ++k)
                add(&m.H[4 * (int64_t)hinges_of_face[k]], 4);
        }
        int64_t ncodes = 0;
        for (int32_t v : w.foot) ncodes += P.row_ptr[v + 1] - P.row_ptr[v];
        const int64_t nf = (int64_t)w.foot.size();
        const int64_t bytes = tile_smem_bytes(8, 13 * nf + 9 * np, nf, ncodes);
        for (int32_t v : w.foot) w.lid[v] = -1;
        w.clear_pairs();
        return ncodes < 65536 ? bytes : INT64_MAX;
    };

    // ---- triangle order and tiles per mesh (never across meshes); tiles
    // must fit the shared memory of the FP64 kernel, larger ones split
    const int64_t budget = 227 * 1024;
    std::vector<std::vector<std::pair<int64_t, int64_t>>> mesh_tiles(m.n_mesh);
    parallel_for(m.n_mesh, nthr, [&](int64_t k, unsigned th) {
        const int64_t a = m.f_off[k], b = m.f_off[k + 1];
        morton_order(m, a, b, order.data() + a);
        const int64_t n = b - a;
        const int64_t ntile = (n + tile_tris - 1) / tile_tris;
        std::vector<std::pair<int64_t, int64_t>> stack;
        for (int64_t i = ntile - 1; i >= 0; --i)  // balanced split, processed in order
            stack.emplace_back(a + (n * i) / ntile, a + (n * (i + 1)) / ntile);
        while (!stack.empty()) {
            auto [s0, s1] = stack.back();
            stack.pop_back();
            if (s1 - s0 > 1 && units(work[th], s0, s1) > budget) {
                const int64_t mid = (s0 + s1) / 2;
                stack.emplace_back(mid, s1);
                stack.emplace_back(s0, mid);
                continue;
            }
            mesh_tiles[k].emplace_back(s0, s1);
        }
    });
    std::vector<int64_t> tile_tri_off(1, 0);
    ts.mesh_tile_off.assign(m.n_mesh + 1, 0);
    for (int k = 0; k < m.n_mesh; ++k) {
        for (auto &r : mesh_tiles[k]) tile_tri_off.push_back(r.second);
        ts.mesh_tile_off[k + 1] = (int32_t)(tile_tri_off.size() - 1);
    }
    const int32_t n_tiles = (int32_t)tile_tri_off.size() - 1;
    ts.n_tiles = n_tiles;
    // hinges grouped by tile, in the order of their faces A inside the tile
    std::vector<int64_t> tile_hinge_off(n_tiles + 1, 0);
    for (int32_t t = 0; t < n_tiles; ++t) {
        int64_t c = 0;
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i) c += hof_off[order[i] + 1] - hof_off[order[i]];
        tile_hinge_off[t + 1] = tile_hinge_off[t] + c;
    }

    // ---- per tile: footprint (sorted global ids = local ids), pair slots
    // (rank in (lo, hi) order), element local ids and slots
    ts.hdr.assign((size_t)n_tiles * 8, 0);
    ts.tri_loc.resize(nT * 6);
    ts.hinge_loc.resize(nH * 10);
    ts.tri_perm.resize(nT);
    ts.hinge_perm.resize(nH);
    std::vector<std::vector<int32_t>> foots(n_tiles);
    std::vector<std::vector<uint32_t>> pairs(n_tiles);
    std::atomic<int> fail(0);
    parallel_for(n_tiles, nthr, [&](int64_t t, unsigned th) {
        Work &w = work[th];
        std::vector<int32_t> &foot = foots[t];
        auto visit = [&](const int32_t *q, int n) {
            for (int i = 0; i < n; ++i)
                if (w.lid[q[i]] < 0) {
                    w.lid[q[i]] = 0;
                    foot.push_back(q[i]);
                }
        };
        // elements in Morton order, then stored interleaved so that the 32
        // lanes of a warp (consecutive stored elements) are far apart in it
        std::vector<int32_t> tri_m, hinge_m;
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i) {
            visit(&m.F[3 * (int64_t)order[i]], 3);
            tri_m.push_back(order[i]);
            for (int64_t k = hof_off[order[i]]; k < hof_off[order[i] + 1]; ++k) {
                const int32_t h = hinges_of_face[k];
                visit(&m.H[4 * (int64_t)h], 4);
                hinge_m.push_back(h);
            }
        }
        interleave32(tri_m, &ts.tri_perm[tile_tri_off[t]]);
        interleave32(hinge_m, &ts.hinge_perm[tile_hinge_off[t]]);
        std::sort(foot.begin(), foot.end());
        if (foot.size() > 65535) fail = ADM_ERR_UNSUPPORTED;
        for (size_t r = 0; r < foot.size(); ++r) w.lid[foot[r]] = (int32_t)r;
        w.clear_pairs();
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i) {
            const int32_t *f = &m.F[3 * (int64_t)ts.tri_perm[i]];
            for (int a = 0; a < 3; ++a) ts.tri_loc[6 * i + a] = (uint16_t)w.lid[f[a]];
            for (int p = 0; p < 3; ++p) {
                const uint32_t k = pkey(w.lid[f[TP[p][0]]], w.lid[f[TP[p][1]]]);
                if (w.insert(k)) w.pairs.push_back(k);
            }
        }
        for (int64_t i = tile_hinge_off[t]; i < tile_hinge_off[t + 1]; ++i) {
            const int32_t *q = &m.H[4 * (int64_t)ts.hinge_perm[i]];
            for (int a = 0; a < 4; ++a) ts.hinge_loc[10 * i + a] = (uint16_t)w.lid[q[a]];
            for (int p = 0; p < 6; ++p) {
                const uint32_t k = pkey(w.lid[q[HP[p][0]]], w.lid[q[HP[p][1]]]);
                if (w.insert(k)) w.pairs.push_back(k);
            }
        }
        std::sort(w.pairs.begin(), w.pairs.end());
        if (w.pairs.size() > 8191) fail = ADM_ERR_UNSUPPORTED;
        for (size_t s = 0; s < w.pairs.size(); ++s) w.value(w.pairs[s]) = (uint16_t)s;
        for (int64_t i = tile_tri_off[t]; i < tile_tri_off[t + 1]; ++i)
            for (int p = 0; p < 3; ++p)
                ts.tri_loc[6 * i + 3 + p] = w.value(pkey(ts.tri_loc[6 * i + TP[p][0]], ts.tri_loc[6 * i + TP[p][1]]));
        for (int64_t i = tile_hinge_off[t]; i < tile_hinge_off[t + 1]; ++i)
            for (int p = 0; p < 6; ++p)
                ts.hinge_loc[10 * i + 4 + p] =
                    w.value(pkey(ts.hinge_loc[10 * i + HP[p][0]], ts.hinge_loc[10 * i + HP[p][1]]));
        // final stored order: bank-aware warp groups (keys: local ids and
        // pair slots mod 32, in the kernel's role order)
        {
            std::vector<uint8_t> key;
            std::vector<int32_t> perm;
            const int64_t t0 = tile_tri_off[t], nt = tile_tri_off[t + 1] - t0;
            key.resize((size_t)nt * 6);
            for (int64_t i = 0; i < nt; ++i)
                for (int r = 0; r < 6; ++r) key[(size_t)i * 6 + r] = (uint8_t)(ts.tri_loc[6 * (t0 + i) + r] & 31);
            bank_groups(nt, 6, key, perm);
            apply_order(perm, 6, &ts.tri_loc[6 * t0], &ts.tri_perm[t0]);
            const int64_t h0 = tile_hinge_off[t], nh = tile_hinge_off[t + 1] - h0;
            if (nh > 0) {
                key.resize((size_t)nh * 10);
                for (int64_t i = 0; i < nh; ++i)
                    for (int r = 0; r < 10; ++r)
                        key[(size_t)i * 10 + r] = (uint8_t)(ts.hinge_loc[10 * (h0 + i) + r] & 31);
                bank_groups(nh, 10, key, perm);
                apply_order(perm, 10, &ts.hinge_loc[10 * h0], &ts.hinge_perm[h0]);
            }
        }
        pairs[t] = w.pairs;
        w.clear_pairs();
        for (int32_t v : foot) w.lid[v] = -1;
    });
    if (fail) return (adm_status)fail.load();

    // ---- ownership: vertices touched by several tiles, and the vertex pairs
    // added into by several tiles (only pairs of two such vertices can be)
    std::vector<int32_t> v_owner(m.nV, -1);  // tile, or -2 if shared
    for (int32_t t = 0; t < n_tiles; ++t)
        for (int32_t v : foots[t]) v_owner[v] = (v_owner[v] == -1) ? t : -2;
    std::vector<std::pair<uint64_t, int32_t>> bnd;
    for (int32_t t = 0; t < n_tiles; ++t) {
        const std::vector<int32_t> &foot = foots[t];
        for (uint32_t k : pairs[t]) {
            const int32_t a = foot[k >> 16], b = foot[k & 0xffff];
            if (v_owner[a] == -2 && v_owner[b] == -2) bnd.emplace_back((uint64_t)a * (uint64_t)m.nV + b, t);
        }
    }
    std::sort(bnd.begin(), bnd.end());
    std::vector<uint64_t> shared_pairs;
    for (size_t i = 0; i < bnd.size();) {
        size_t j = i;
        while (j < bnd.size() && bnd[j].first == bnd[i].first) ++j;
        if (j - i > 1) shared_pairs.push_back(bnd[i].first);
        i = j;
    }
    auto pair_shared = [&](int32_t a, int32_t b) {  // global ids, a < b
        return std::binary_search(shared_pairs.begin(), shared_pairs.end(), (uint64_t)a * (uint64_t)m.nV + b);
    };

    // ---- row codes: the columns a tile touches in footprint row r are, in
    // ascending order, the lower partners of r (pairs (c, r)), r itself and
    // the upper partners (pairs (r, c)); walk them against the BSR row
    std::vector<std::vector<uint16_t>> t_codes(n_tiles);
    std::vector<std::vector<int32_t>> t_code_off(n_tiles), t_row_start(n_tiles), t_zero(n_tiles);
    parallel_for(n_tiles, nthr, [&](int64_t t, unsigned) {
        const std::vector<int32_t> &foot = foots[t];
        const std::vector<uint32_t> &pp = pairs[t];
        const int32_t nf = (int32_t)foot.size();
        std::vector<int32_t> lo_off(nf + 1, 0), up_off(nf + 1, 0);
        for (uint32_t k : pp) {
            up_off[(k >> 16) + 1]++;
            lo_off[(k & 0xffff) + 1]++;
        }
        for (int32_t r = 0; r < nf; ++r) {
            up_off[r + 1] += up_off[r];
            lo_off[r + 1] += lo_off[r];
        }
        // lower partners of every row, ascending (pp is sorted by lo)
        std::vector<uint32_t> lower(pp.size());  // partner << 16 | slot
        {
            std::vector<int32_t> pos(lo_off.begin(), lo_off.end() - 1);
            for (size_t s = 0; s < pp.size(); ++s) lower[pos[pp[s] & 0xffff]++] = (pp[s] >> 16) << 16 | (uint32_t)s;
        }
        std::vector<uint16_t> &codes = t_codes[t];
        for (int32_t r = 0; r < nf; ++r) {
            const int32_t v = foot[r];
            const bool v_sh = v_owner[v] == -2;
            t_row_start[t].push_back((int32_t)((uint32_t)P.row_ptr[v] | (v_sh ? 0x80000000u : 0u)));
            t_code_off[t].push_back((int32_t)codes.size());
            int32_t li = lo_off[r], ui = up_off[r];
            bool diag_done = false;
            for (int32_t b = P.row_ptr[v]; b < P.row_ptr[v + 1]; ++b) {
                const int32_t c = P.col[b];
                uint16_t code = 0;  // kind 0: block not produced by this tile
                if (li < lo_off[r + 1] && foot[lower[li] >> 16] == c) {
                    code = (uint16_t)(3u << 14 | (lower[li] & 0xffffu));  // transposed pair (c, v)
                    if (v_sh && v_owner[c] == -2 && pair_shared(c, v)) code |= (uint16_t)(1u << 13);
                    ++li;
                } else if (!diag_done && c == v) {
                    code = (uint16_t)(1u << 14);  // diagonal
                    if (v_sh) code |= (uint16_t)(1u << 13);
                    diag_done = true;
                } else if (ui < up_off[r + 1] && foot[pp[ui] & 0xffff] == c) {
                    code = (uint16_t)(2u << 14 | (uint32_t)ui);  // pair (v, c)
                    if (v_sh && v_owner[c] == -2 && pair_shared(v, c)) code |= (uint16_t)(1u << 13);
                    ++ui;
                }
                codes.push_back(code);
                if (code & 0x2000) t_zero[t].push_back(b);
            }
            if (li != lo_off[r + 1] || ui != up_off[r + 1] || !diag_done) fail = ADM_ERR_MESH;
        }
    });
    if (fail) return (adm_status)fail.load();

    // ---- concatenate; per tile, the metadata blob the kernel copies into
    // shared memory: row starts (int32), row code offsets relative to the
    // tile (uint16, nf + 1) and the codes (uint16), padded to 16 bytes
    for (auto &x : ts.smem_bytes) x[0] = x[1] = 0;
    ts.meta_off.assign(n_tiles + 1, 0);
    ts.meta.clear();
    for (int32_t t = 0; t < n_tiles; ++t) {
        const int32_t nf = (int32_t)foots[t].size(), np = (int32_t)pairs[t].size();
        const int32_t foot_begin = (int32_t)ts.foot.size();
        const int32_t code_begin = (int32_t)ts.codes.size();
        ts.foot.insert(ts.foot.end(), foots[t].begin(), foots[t].end());
        ts.row_start.insert(ts.row_start.end(), t_row_start[t].begin(), t_row_start[t].end());
        for (int32_t c : t_code_off[t]) ts.code_off.push_back(c + code_begin);
        ts.code_off.push_back(code_begin + (int32_t)t_codes[t].size());  // sentinel of the last row
        ts.codes.insert(ts.codes.end(), t_codes[t].begin(), t_codes[t].end());
        ts.zero_blocks.insert(ts.zero_blocks.end(), t_zero[t].begin(), t_zero[t].end());
        int32_t *hd = &ts.hdr[8 * (size_t)t];
        hd[0] = (int32_t)tile_tri_off[t];
        hd[1] = (int32_t)(tile_tri_off[t + 1] - tile_tri_off[t]);
        hd[2] = (int32_t)tile_hinge_off[t];
        hd[3] = (int32_t)(tile_hinge_off[t + 1] - tile_hinge_off[t]);
        hd[4] = foot_begin;
        hd[5] = nf;
        hd[6] = np;
        hd[7] = code_begin;
        const int64_t ncodes = (int64_t)t_codes[t].size();
        if (ncodes >= 65536) return ADM_ERR_UNSUPPORTED;
        const int64_t mb = tile_meta_bytes(nf, ncodes);
        const size_t m0 = ts.meta.size();
        ts.meta.resize(m0 + mb, 0);
        unsigned char *blob = ts.meta.data() + m0;
        std::memcpy(blob, t_row_start[t].data(), 4 * (size_t)nf);
        for (int32_t r = 0; r <= nf; ++r) {
            const uint16_t c = (uint16_t)(r < nf ? t_code_off[t][r] : ncodes);
            std::memcpy(blob + 4 * nf + 2 * r, &c, 2);
        }
        std::memcpy(blob + 6 * nf + 2, t_codes[t].data(), 2 * (size_t)ncodes);
        ts.meta_off[t + 1] = (int64_t)ts.meta.size();
        for (int p = 0; p < 2; ++p) {
            const int eb = p == 0 ? 8 : 4;  // index: ADM_FP64 = 0, ADM_FP32 = 1
            ts.smem_bytes[1][p] =
                std::max(ts.smem_bytes[1][p], tile_smem_bytes(eb, 13 * (int64_t)nf + 9 * (int64_t)np, nf, ncodes));
            ts.smem_bytes[0][p] =
                std::max(ts.smem_bytes[0][p], tile_smem_bytes(eb, 7 * (int64_t)nf + 5 * (int64_t)np, nf, ncodes));
        }
    }
    // code_off has one sentinel per tile: footprint row r of tile t is at
    // index foot_begin + t + r
    // shared outputs zeroed before every pass, each listed once
    std::sort(ts.zero_blocks.begin(), ts.zero_blocks.end());
    ts.zero_blocks.erase(std::unique(ts.zero_blocks.begin(), ts.zero_blocks.end()), ts.zero_blocks.end());
    for (int64_t v = 0; v < m.nV; ++v)
        if (v_owner[v] == -2) ts.zero_verts.push_back((int32_t)v);
    // vertices no element touches: no tile writes their gradient row or
    // diagonal block, so both are zeroed with the shared ones every pass
    for (int64_t v = 0; v < m.nV; ++v)
        if (v_owner[v] == -1) {
            ts.zero_verts.push_back((int32_t)v);
            const auto b = P.col.begin() + P.row_ptr[v], e = P.col.begin() + P.row_ptr[v + 1];
            ts.zero_blocks.push_back((int32_t)(std::lower_bound(b, e, (int32_t)v) - P.col.begin()));
        }
    std::sort(ts.zero_verts.begin(), ts.zero_verts.end());
    std::sort(ts.zero_blocks.begin(), ts.zero_blocks.end());
    static std::atomic<int64_t> builds(0);
    ts.build_id = ++builds;
    ts.built = true;
    return ADM_OK;
}

// Mass-spring elements on a built triangle tile set (Sec. 7.1: per-edge
// springs, per-vertex inertia and gravity).  An edge belongs to the tile of
// the first triangle (in tile order) that has it, so both its vertices are in
// that tile's footprint and their pair has a slot there (read from that
// triangle's record); a vertex belongs to the first tile whose footprint has
// it.  Both lists are stored in bank-aware warp groups like the triangles.
adm_status tiles_build_cloth(const HostMesh &m, TileSet &ts)
{
    if (!ts.built || ts.n_tiles == 0) return ADM_ERR_ARG;
    const int32_t n_tiles = ts.n_tiles;
    struct Cand {
        uint64_t key;   // lo * nV + hi
        int64_t pos;    // triangle position in tile order
        int32_t pair;   // which of its 3 pairs
    };
    std::vector<Cand> cand;
    cand.reserve(3 * (size_t)m.nT);
    for (int32_t t = 0; t < n_tiles; ++t) {
        const int32_t *hd = &ts.hdr[8 * (size_t)t];
        for (int64_t i = hd[0]; i < (int64_t)hd[0] + hd[1]; ++i) {
            const int32_t *f = &m.F[3 * (int64_t)ts.tri_perm[i]];
            for (int p = 0; p < 3; ++p) {
                const int64_t a = f[TP[p][0]], b = f[TP[p][1]];
                cand.push_back({(uint64_t)std::min(a, b) * (uint64_t)m.nV + (uint64_t)std::max(a, b), i, p});
            }
        }
    }
    std::stable_sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.key < y.key; });
    std::vector<int32_t> tile_of_pos(m.nT);
    for (int32_t t = 0; t < n_tiles; ++t)
        for (int64_t i = ts.hdr[8 * (size_t)t]; i < (int64_t)ts.hdr[8 * (size_t)t] + ts.hdr[8 * (size_t)t + 1]; ++i)
            tile_of_pos[i] = t;
    std::vector<std::vector<int64_t>> tile_edges(n_tiles);  // index into cand of the owning record
    for (size_t i = 0; i < cand.size();) {
        size_t j = i;
        while (j < cand.size() && cand[j].key == cand[i].key) ++j;
        tile_edges[tile_of_pos[cand[i].pos]].push_back((int64_t)i);  // first in tile order (stable sort)
        i = j;
    }
    std::vector<char> vseen(m.nV, 0);
    ts.cloth_hdr.assign(4 * (size_t)n_tiles, 0);
    ts.edge_loc.clear();
    ts.vert_loc.clear();
    ts.edge_l2.clear();
    ts.vert_area3.clear();
    std::vector<double> area3(m.nV, 0.0);
    for (int64_t t = 0; t < m.nT; ++t)
        for (int c = 0; c < 3; ++c) area3[m.F[3 * t + c]] += m.tri_area[t] / 3.0;
    for (int32_t t = 0; t < n_tiles; ++t) {
        const int32_t *hd = &ts.hdr[8 * (size_t)t];
        const int32_t foot_begin = hd[4], nf = hd[5];
        // edges in bank-aware warp groups (keys: both local ids, the pair slot)
        const int64_t ne = (int64_t)tile_edges[t].size();
        std::vector<uint8_t> key((size_t)ne * 3);
        for (int64_t q = 0; q < ne; ++q) {
            const Cand &c = cand[tile_edges[t][q]];
            const uint16_t *tl = &ts.tri_loc[6 * c.pos];
            key[(size_t)q * 3] = (uint8_t)(tl[TP[c.pair][0]] & 31);
            key[(size_t)q * 3 + 1] = (uint8_t)(tl[TP[c.pair][1]] & 31);
            key[(size_t)q * 3 + 2] = (uint8_t)(tl[3 + c.pair] & 31);
        }
        std::vector<int32_t> il;
        bank_groups(ne, 3, key, il);
        ts.cloth_hdr[4 * (size_t)t] = (int32_t)(ts.edge_loc.size() / 3);
        ts.cloth_hdr[4 * (size_t)t + 1] = (int32_t)ne;
        for (int32_t q : il) {
            const Cand &c = cand[tile_edges[t][q]];
            const uint16_t *tl = &ts.tri_loc[6 * c.pos];
            ts.edge_loc.push_back(tl[TP[c.pair][0]]);
            ts.edge_loc.push_back(tl[TP[c.pair][1]]);
            ts.edge_loc.push_back(tl[3 + c.pair]);
            const int64_t a = ts.foot[foot_begin + tl[TP[c.pair][0]]], b = ts.foot[foot_begin + tl[TP[c.pair][1]]];
            double l2 = 0.0;
            for (int d = 0; d < 3; ++d) l2 += (m.V[3 * a + d] - m.V[3 * b + d]) * (m.V[3 * a + d] - m.V[3 * b + d]);
            if (!(l2 > 0.0)) return ADM_ERR_MESH;
            ts.edge_l2.push_back(l2);
        }
        // vertices first seen in this tile, in bank-aware warp groups
        std::vector<int32_t> vl;
        for (int32_t r = 0; r < nf; ++r) {
            const int32_t v = ts.foot[foot_begin + r];
            if (!vseen[v]) {
                vseen[v] = 1;
                vl.push_back(r);
            }
        }
        std::vector<uint8_t> vkey(vl.size());
        for (size_t q = 0; q < vl.size(); ++q) vkey[q] = (uint8_t)(vl[q] & 31);
        std::vector<int32_t> vperm, vil(vl.size());
        bank_groups((int64_t)vl.size(), 1, vkey, vperm);
        for (size_t q = 0; q < vl.size(); ++q) vil[q] = vl[vperm[q]];
        ts.cloth_hdr[4 * (size_t)t + 2] = (int32_t)ts.vert_loc.size();
        ts.cloth_hdr[4 * (size_t)t + 3] = (int32_t)vil.size();
        for (int32_t r : vil) {
            ts.vert_loc.push_back((uint16_t)r);
            ts.vert_area3.push_back(area3[ts.foot[foot_begin + r]]);
        }
    }
    ts.cloth_built = true;
    return ADM_OK;
}

}  // namespace adm
