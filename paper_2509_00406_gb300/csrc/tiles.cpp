// tiles.cpp -- host construction of the tiles of the staged-gather assembler.
//
// The paper evaluates each term over RXMesh patches staged in shared memory
// (Sec. 2.4, Sec. 5.2) and scatters with global atomics (Sec. 5.5).  Here a
// tile is a run of units (a triangle and its attached edges, see TileSet in
// internal.h) in Morton order of their rest centroids, per mesh.  The builder
// lays out, per tile, where every unit writes its contributions ("chunks",
// sorted by the output they add to), the segments the gather sums, the codes
// that map segments to BSR positions, and the groups of outputs that several
// tiles produce.  Everything is built once per mesh, in parallel over meshes
// and tiles; nothing here runs per pass.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
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
    if (n < 2 || nt == 1) {
        for (int64_t i = 0; i < n; ++i) f(i, 0u);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (unsigned k = 0; k < std::min<int64_t>(nt, n); ++k)
        th.emplace_back([&, k] {
            for (int64_t i; (i = next.fetch_add(1)) < n;) f(i, k);
        });
    for (auto &t : th) t.join();
}

uint64_t pkey(int64_t a, int64_t b, int64_t nV)
{
    return a < b ? (uint64_t)a * (uint64_t)nV + (uint64_t)b : (uint64_t)b * (uint64_t)nV + (uint64_t)a;
}

// A face with its rotation and attached edges, as a unit.
struct UnitRec {
    int32_t face;
    int32_t t[3];       // vertices (global), in the triangle's own order
    int32_t extra[3];   // per slot: the vertex across the slot's edge, -1 if none (boundary)
    int32_t hinge[3];   // per slot: canonical hinge index, -1 if none or no hinges
    int nslot;
    int rot;            // slot s is the edge (t_k, t_k+1) of k = (rot + s) mod 3
};

}  // namespace

static int64_t align16(int64_t b) { return (b + 15) & ~int64_t(15); }

int64_t tile_smem_bytes(const TileSet &ts, int mode, int vd, int elem_bytes)
{
    int64_t best = 0;
    for (int32_t t = 0; t < ts.n_tiles; ++t) {
        const int32_t *hd = &ts.hdr[(size_t)kHdr * t];
        const TileLayout L = tile_layout((int)ts.max_nf, hd[kHdrNVC], hd[kHdrNPC],
                                         (int)(ts.meta_off[t + 1] - ts.meta_off[t]), mode, vd, elem_bytes);
        best = std::max<int64_t>(best, L.total);
    }
    return best;
}

namespace {

// per tile: the sizes that decide its shared memory (HESS, VD = 3)
struct TileCount {
    int64_t nf = 0, nvc = 0, npc = 0, ncodes = 0;
};

int64_t hess_bytes(const TileCount &c, int elem_bytes)
{
    // x, staging (vertex and pair chunks of 9), metadata bound (rows, code
    // words, and at most one slot-table entry per row and per pair block)
    return align16(c.nf * 3 * elem_bytes) + align16((c.nvc + c.npc) * 9 * elem_bytes) +
           align16(16 * c.nf + 4 * c.ncodes + 4 * (c.nf + c.ncodes));
}

}  // namespace

// FP32 tiles run two blocks per SM (at most about 112 KB each), FP64 tiles
// one.  A tile's own count takes its x at its own footprint; the kernel
// sizes that region for the set's largest footprint (kMaxFootRows rows at
// most, 6 KB in FP32 and 12 KB in FP64 above the tile's own), so the budgets
// leave that much room
constexpr int64_t kBudget32 = 104 * 1024, kBudget64 = 208 * 1024;

adm_status tiles_build(const HostMesh &m, const Pattern &P, bool with_hinges, int tile_units, TileSet &ts)
{
    const int64_t nT = m.nT, nV = m.nV;
    ts = TileSet();
    ts.tile_units = tile_units = std::max(1, std::min(tile_units, 4096));
    const unsigned nthr = worker_count();

    // ---- edges: partner face and across vertex of every directed face edge
    std::vector<int32_t> partner(3 * nT, -1), across(3 * nT, -1);
    {
        std::vector<std::pair<uint64_t, int64_t>> de(3 * nT);  // (undirected key, 3 t + k)
        parallel_for(m.n_mesh, nthr, [&](int64_t k, unsigned) {
            for (int64_t t = m.f_off[k]; t < m.f_off[k + 1]; ++t)
                for (int c = 0; c < 3; ++c)
                    de[3 * t + c] = {pkey(m.F[3 * t + c], m.F[3 * t + (c + 1) % 3], nV), 3 * t + c};
            std::sort(de.begin() + 3 * m.f_off[k], de.begin() + 3 * m.f_off[k + 1]);
        });
        for (int64_t i = 0; i < 3 * nT;) {
            int64_t j = i;
            while (j < 3 * nT && de[j].first == de[i].first) ++j;
            if (j - i == 2) {  // two faces: a manifold interior edge if they traverse it oppositely
                const int64_t a = de[i].second, b = de[i + 1].second;
                const int64_t ta = a / 3, tb = b / 3;
                const int ka = (int)(a % 3), kb = (int)(b % 3);
                if (m.F[3 * ta + ka] == m.F[3 * tb + (kb + 1) % 3]) {
                    partner[a] = (int32_t)b;
                    partner[b] = (int32_t)a;
                    across[a] = m.F[3 * tb + (kb + 2) % 3];
                    across[b] = m.F[3 * ta + (ka + 2) % 3];
                }
            }
            i = j;
        }
    }
    // ---- attach every edge to one of its faces, at most two per face where
    // the counts allow (greedy over faces, then edges)
    std::vector<uint8_t> att(nT, 0), natt(nT, 0);
    parallel_for(m.n_mesh, nthr, [&](int64_t k, unsigned) {
        for (int64_t t = m.f_off[k]; t < m.f_off[k + 1]; ++t)
            for (int c = 0; c < 3; ++c) {
                const int64_t e = 3 * t + c, p = partner[e];
                if (p < 0) {  // boundary (or non-manifold) edge: its own face
                    att[t] |= (uint8_t)(1u << c);
                    natt[t]++;
                    continue;
                }
                if (p < e) continue;  // decided from the other side
                const int64_t tp = p / 3;
                const int cp = (int)(p % 3);
                if (natt[t] <= natt[tp]) {
                    att[t] |= (uint8_t)(1u << c);
                    natt[t]++;
                } else {
                    att[tp] |= (uint8_t)(1u << cp);
                    natt[tp]++;
                }
            }
    });
    // canonical hinge of an edge (hinges sorted by (e0, e1), e0 < e1)
    auto hinge_of = [&](int32_t a, int32_t b) -> int32_t {
        const int32_t e0 = std::min(a, b), e1 = std::max(a, b);
        int64_t lo = 0, hi = m.nH();
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            const int32_t x0 = m.H[4 * mid], x1 = m.H[4 * mid + 1];
            if (x0 < e0 || (x0 == e0 && x1 < e1)) lo = mid + 1;
            else hi = mid;
        }
        return (lo < m.nH() && m.H[4 * lo] == e0 && m.H[4 * lo + 1] == e1) ? (int32_t)lo : -1;
    };
    // ---- units: rotation so that the attached edges are slots 0, 1, 2
    std::vector<UnitRec> U(nT);
    parallel_for(m.n_mesh, nthr, [&](int64_t k, unsigned) {
        for (int64_t t = m.f_off[k]; t < m.f_off[k + 1]; ++t) {
            const int a = att[t];
            const int n = __builtin_popcount(a);
            int r = 0;
            if (n == 1) r = a == 1 ? 0 : (a == 2 ? 1 : 2);
            else if (n == 2) {
                const int k1 = (a & 1) ? 0 : 1, k2 = (a & 4) ? 2 : 1;  // the two set bits, k1 < k2
                r = ((k1 + 1) % 3 == k2) ? k1 : k2;
            }
            UnitRec &u = U[t];
            u.face = (int32_t)t;
            u.nslot = n;
            u.rot = r;
            for (int i = 0; i < 3; ++i) u.t[i] = m.F[3 * t + i];
            for (int s = 0; s < 3; ++s) {
                u.extra[s] = -1;
                u.hinge[s] = -1;
                if (s >= n) continue;
                const int k = (r + s) % 3;  // the slot's edge (t_k, t_k+1)
                const int64_t e = 3 * t + k;
                if (with_hinges && partner[e] >= 0) {
                    u.extra[s] = across[e];
                    u.hinge[s] = hinge_of(u.t[k], u.t[(k + 1) % 3]);
                    if (u.hinge[s] < 0) u.extra[s] = -1;
                }
            }
        }
    });

    // ---- tiles per mesh (never across meshes): runs of units in Morton
    // order of balanced size, split further until they fit shared memory
    std::vector<int32_t> order(nT);
    std::vector<std::vector<std::pair<int64_t, int64_t>>> mesh_tiles(m.n_mesh);
    struct Scratch {
        std::vector<int32_t> mark;
        explicit Scratch(int64_t n) : mark(n, -1) {}
    };
    std::vector<Scratch> scr;
    scr.reserve(nthr);
    for (unsigned k = 0; k < nthr; ++k) scr.emplace_back(nV);
    auto count_range = [&](Scratch &w, int64_t a, int64_t b) {
        TileCount c;
        std::vector<uint64_t> pairs;
        std::vector<int32_t> touched;
        for (int64_t i = a; i < b; ++i) {
            const UnitRec &u = U[order[i]];
            int32_t vs[6];
            int nv = 0;
            for (int q = 0; q < 3; ++q) vs[nv++] = u.t[q];
            for (int s = 0; s < u.nslot; ++s)
                if (u.extra[s] >= 0) vs[nv++] = u.extra[s];
            for (int q = 0; q < nv; ++q)
                if (w.mark[vs[q]] < 0) {
                    w.mark[vs[q]] = 1;
                    touched.push_back(vs[q]);
                }
            c.nvc += nv;
            for (int p = 0; p < 3; ++p) pairs.push_back(pkey(u.t[p], u.t[(p + 1) % 3], nV));
            for (int s = 0; s < u.nslot; ++s)
                if (u.extra[s] >= 0) {
                    c.npc += 3;
                    for (int q = 0; q < 3; ++q) pairs.push_back(pkey(u.extra[s], u.t[q], nV));
                }
            c.npc += 3;
        }
        for (int32_t v : touched) w.mark[v] = -1;
        std::sort(pairs.begin(), pairs.end());
        c.nf = (int64_t)touched.size();
        c.ncodes = 2 * (int64_t)(std::unique(pairs.begin(), pairs.end()) - pairs.begin());
        return c;
    };
    std::atomic<int> fail(0);
    parallel_for(m.n_mesh, nthr, [&](int64_t k, unsigned th) {
        const int64_t a = m.f_off[k], b = m.f_off[k + 1];
        morton_order(m, a, b, order.data() + a);
        const int64_t n = b - a;
        const int64_t ntile = (n + tile_units - 1) / tile_units;
        std::vector<std::pair<int64_t, int64_t>> stack;
        for (int64_t i = ntile - 1; i >= 0; --i) stack.emplace_back(a + (n * i) / ntile, a + (n * (i + 1)) / ntile);
        while (!stack.empty()) {
            auto [s0, s1] = stack.back();
            stack.pop_back();
            const TileCount c = count_range(scr[th], s0, s1);
            const bool fits = hess_bytes(c, 4) <= kBudget32 && hess_bytes(c, 8) <= kBudget64 && c.nf <= kMaxFootRows &&
                              c.npc < 8192 && c.nvc < 65536 && c.ncodes < 65536;
            if (!fits) {
                if (s1 - s0 <= 1) {
                    fail = ADM_ERR_UNSUPPORTED;
                    return;
                }
                const int64_t mid = (s0 + s1) / 2;
                stack.emplace_back(mid, s1);
                stack.emplace_back(s0, mid);
                continue;
            }
            mesh_tiles[k].emplace_back(s0, s1);
        }
    });
    if (fail) return (adm_status)fail.load();
    std::vector<int64_t> tile_off(1, 0);
    ts.mesh_tile_off.assign(m.n_mesh + 1, 0);
    std::vector<int32_t> tile_mesh;
    for (int k = 0; k < m.n_mesh; ++k) {
        for (auto &r : mesh_tiles[k]) {
            tile_off.push_back(r.second);
            tile_mesh.push_back(k);
        }
        ts.mesh_tile_off[k + 1] = (int32_t)(tile_off.size() - 1);
    }
    const int32_t n_tiles = (int32_t)tile_off.size() - 1;
    ts.n_tiles = n_tiles;

    // ---- per tile: unit order (more slots first, then Morton), footprint,
    // chunks sorted by target, destinations, segments, codes
    struct TileOut {
        std::vector<int32_t> units;                 // canonical faces, in tile order
        std::vector<int32_t> foot;
        std::vector<uint16_t> unit, unit_dst, slot_dst;
        std::vector<int32_t> slot_hinge;            // per slot
        std::vector<std::array<int32_t, 4>> slot_v; // per slot: t_k, t_k+1, t_k+2, extra (-1: none)
        std::vector<int32_t> rows;                  // kRowWords per footprint row (shared fields later)
        std::vector<uint32_t> codes;
        std::vector<uint64_t> pair_keys;            // produced unordered pairs (global key)
        int64_t nvc = 0, npc = 0;
    };
    std::vector<TileOut> T(n_tiles);
    const int64_t maxrow = 512;
    std::atomic<int> fail_big(0);  // a tile too large for the code fields: smaller tiles
    parallel_for(n_tiles, nthr, [&](int64_t t, unsigned th) {
        TileOut &o = T[t];
        Scratch &w = scr[th];
        std::vector<int32_t> &un = o.units;
        for (int64_t i = tile_off[t]; i < tile_off[t + 1]; ++i) un.push_back(order[i]);
        std::stable_sort(un.begin(), un.end(), [&](int32_t x, int32_t y) { return U[x].nslot > U[y].nslot; });
        // footprint (sorted global ids) and local ids
        for (int32_t f : un) {
            const UnitRec &u = U[f];
            for (int q = 0; q < 3; ++q) o.foot.push_back(u.t[q]);
            for (int s = 0; s < u.nslot; ++s)
                if (u.extra[s] >= 0) o.foot.push_back(u.extra[s]);
        }
        std::sort(o.foot.begin(), o.foot.end());
        o.foot.erase(std::unique(o.foot.begin(), o.foot.end()), o.foot.end());
        for (size_t r = 0; r < o.foot.size(); ++r) w.mark[o.foot[r]] = (int32_t)r;
        // chunk records: (target, unit, role) -> position after sorting
        struct VRec {
            int32_t lid, unit, role;
        };
        struct PRec {
            int32_t lo, hi, unit, role;
        };
        std::vector<VRec> vr;
        std::vector<PRec> pr;
        int32_t slot = 0;
        std::vector<int32_t> slot_first(un.size());
        for (size_t i = 0; i < un.size(); ++i) {
            const UnitRec &u = U[un[i]];
            slot_first[i] = slot;
            const int32_t l[3] = {w.mark[u.t[0]], w.mark[u.t[1]], w.mark[u.t[2]]};
            for (int q = 0; q < 3; ++q) vr.push_back({l[q], (int32_t)i, q});
            const int pp[3][2] = {{0, 1}, {0, 2}, {1, 2}};
            for (int p = 0; p < 3; ++p)
                pr.push_back({std::min(l[pp[p][0]], l[pp[p][1]]), std::max(l[pp[p][0]], l[pp[p][1]]), (int32_t)i, p});
            for (int s = 0; s < u.nslot; ++s, ++slot) {
                if (u.extra[s] < 0) continue;
                const int32_t lx = w.mark[u.extra[s]];
                vr.push_back({lx, (int32_t)i, 3 + s});
                for (int q = 0; q < 3; ++q) {  // hinge vertex q = tri vertex (rot + s + q) % 3
                    const int32_t lq = l[(u.rot + s + q) % 3];
                    pr.push_back({std::min(lx, lq), std::max(lx, lq), (int32_t)i, 3 + 3 * s + q});
                }
            }
        }
        std::sort(vr.begin(), vr.end(), [](const VRec &x, const VRec &y) {
            return x.lid != y.lid ? x.lid < y.lid : (x.unit != y.unit ? x.unit < y.unit : x.role < y.role);
        });
        std::sort(pr.begin(), pr.end(), [](const PRec &x, const PRec &y) {
            if (x.lo != y.lo) return x.lo < y.lo;
            if (x.hi != y.hi) return x.hi < y.hi;
            return x.unit != y.unit ? x.unit < y.unit : x.role < y.role;
        });
        o.nvc = (int64_t)vr.size();
        o.npc = (int64_t)pr.size();
        o.unit.assign(8 * un.size(), 0xffff);
        o.unit_dst.assign(6 * un.size(), 0xffff);
        o.slot_dst.assign(4 * (size_t)slot, 0xffff);
        o.slot_hinge.assign(slot, -1);
        o.slot_v.assign(slot, {-1, -1, -1, -1});
        std::vector<int32_t> vseg_start(o.foot.size(), 0), vseg_n(o.foot.size(), 0);
        for (size_t c = 0; c < vr.size(); ++c) {
            const VRec &r = vr[c];
            if (vseg_n[r.lid]++ == 0) vseg_start[r.lid] = (int32_t)c;
            if (r.role < 3) o.unit_dst[6 * r.unit + r.role] = (uint16_t)c;
            else o.slot_dst[4 * (slot_first[r.unit] + r.role - 3)] = (uint16_t)c;
        }
        // pair segments, keyed by (lo, hi) local ids
        std::vector<std::array<int32_t, 4>> pseg;  // lo, hi, start, count
        for (size_t c = 0; c < pr.size(); ++c) {
            const PRec &r = pr[c];
            if (pseg.empty() || pseg.back()[0] != r.lo || pseg.back()[1] != r.hi)
                pseg.push_back({r.lo, r.hi, (int32_t)c, 0});
            pseg.back()[3]++;
            if (r.role < 3) o.unit_dst[6 * r.unit + 3 + r.role] = (uint16_t)c;
            else {
                const int s = (r.role - 3) / 3, q = (r.role - 3) % 3;
                o.slot_dst[4 * (slot_first[r.unit] + s) + 1 + q] = (uint16_t)c;
            }
        }
        for (auto &p : pseg) o.pair_keys.push_back(pkey(o.foot[p[0]], o.foot[p[1]], nV));
        // unit records
        for (size_t i = 0; i < un.size(); ++i) {
            const UnitRec &u = U[un[i]];
            uint16_t *r = &o.unit[8 * i];
            for (int q = 0; q < 3; ++q) r[q] = (uint16_t)w.mark[u.t[q]];
            for (int s = 0; s < 3; ++s) r[3 + s] = (s < u.nslot && u.extra[s] >= 0) ? (uint16_t)w.mark[u.extra[s]] : 0xffff;
            r[6] = (uint16_t)(u.nslot | u.rot << 5);
            r[7] = (uint16_t)slot_first[i];
            for (int s = 0; s < u.nslot; ++s) {
                const int k = (u.rot + s) % 3;
                o.slot_hinge[slot_first[i] + s] = u.hinge[s];
                o.slot_v[slot_first[i] + s] = {u.t[k], u.t[(k + 1) % 3], u.t[(k + 2) % 3], u.extra[s]};
            }
        }
        // rows: BSR row start, vertex segment, diagonal block; pair codes,
        // one per pair segment (2 words): chunk start (13 bits) | count << 13
        // (4 bits) | partial A << 17 | partial B << 18 | row A << 19 (9 bits);
        // position A (9 bits) | row B << 9 | position B << 18.  Block A is
        // (lo, hi) in row lo, block B its transpose (hi, lo) in row hi; a
        // partial block's (row << 9 | position) is its slot-table index.
        const int32_t nf = (int32_t)o.foot.size();
        if (nf > 512 || o.npc > 8191) fail_big = 1;
        auto pos_in_row = [&](int32_t v, int32_t c) -> int32_t {
            const int32_t *b0 = P.col.data() + P.row_ptr[v], *b1 = P.col.data() + P.row_ptr[v + 1];
            const int32_t *it = std::lower_bound(b0, b1, c);
            return (it != b1 && *it == c) ? (int32_t)(it - b0) : -1;
        };
        o.rows.assign((size_t)kRowWords * nf, 0);
        for (int32_t r = 0; r < nf; ++r) {
            const int32_t v = o.foot[r];
            const int32_t b0 = P.row_ptr[v], b1 = P.row_ptr[v + 1];
            if (b1 - b0 > maxrow) fail = ADM_ERR_UNSUPPORTED;
            const int32_t diag = pos_in_row(v, v);
            if (diag < 0 || vseg_n[r] > 255 || vseg_n[r] == 0) fail = ADM_ERR_MESH;
            int32_t *row = &o.rows[(size_t)kRowWords * r];
            row[0] = b0;
            row[1] = (int32_t)((uint32_t)vseg_n[r] << 24);
            row[2] = vseg_start[r];
            row[3] = diag;
        }
        for (auto &ps : pseg) {
            const int32_t lo = ps[0], hi = ps[1];
            const int32_t pa = pos_in_row(o.foot[lo], o.foot[hi]), pb = pos_in_row(o.foot[hi], o.foot[lo]);
            if (pa < 0 || pb < 0) fail = ADM_ERR_MESH;
            if (ps[3] >= 16) fail = ADM_ERR_UNSUPPORTED;
            o.codes.push_back((uint32_t)ps[2] | (uint32_t)ps[3] << 13 | (uint32_t)lo << 19);
            o.codes.push_back((uint32_t)pa | (uint32_t)hi << 9 | (uint32_t)pb << 18);
        }
        for (int32_t v : o.foot) w.mark[v] = -1;
    });
    if (fail_big && !fail) {
        if (tile_units <= 16) return ADM_ERR_UNSUPPORTED;
        return tiles_build(m, P, with_hinges, tile_units / 2, ts);
    }
    if (fail) return (adm_status)fail.load();

    // ---- outputs several tiles produce: rows (a vertex in several
    // footprints) and pair blocks (a pair produced by several tiles).  The
    // lowest-index tile of such an output stores its part in the output;
    // every other one stores its part in a partial slot of its own.  The
    // slots of one output are contiguous, in tile order, and a fix-up pass
    // adds them to the output in that order after the tiles have run, so the
    // sum is the same on every pass.  Tile sets never span meshes, so meshes
    // are handled in parallel (mesh-local slots, offset afterwards).
    struct MeshFix {
        std::vector<std::array<int32_t, 4>> fv, fp;  // (row vertex, position in the row, slots, first slot)
        int64_t nv = 0, np = 0;                      // vertex and pair slots of the mesh
    };
    std::vector<MeshFix> mfix(m.n_mesh);
    std::vector<std::vector<int64_t>> ptab(n_tiles);  // per tile: its slots (bit 62: a pair slot), mesh-local
    std::atomic<int> fail_part(0);
    auto row_pos = [&](int32_t v, int32_t c) -> int32_t {
        for (int32_t b = P.row_ptr[v]; b < P.row_ptr[v + 1]; ++b)
            if (P.col[b] == c) return b - P.row_ptr[v];
        return -1;
    };
    parallel_for(m.n_mesh, nthr, [&](int64_t k, unsigned) {
        const int32_t t0 = ts.mesh_tile_off[k], t1 = ts.mesh_tile_off[k + 1];
        MeshFix &mf = mfix[k];
        std::vector<std::pair<int32_t, int32_t>> vt;
        std::vector<std::pair<uint64_t, int32_t>> pt;
        for (int32_t t = t0; t < t1; ++t) {
            for (int32_t v : T[t].foot) vt.emplace_back(v, t);
            for (uint64_t p : T[t].pair_keys) pt.emplace_back(p, t);
        }
        std::sort(vt.begin(), vt.end());
        std::sort(pt.begin(), pt.end());
        // later producers of every shared output: (key, tile, rank >= 1),
        // sorted by (key, tile).  Slots are allocated in output order
        // (vertex order; block order for pair blocks) so that the fix-up
        // streams through them.
        std::vector<std::array<int64_t, 3>> vrank, prank;
        for (size_t i = 0; i < vt.size();) {
            size_t j = i;
            while (j < vt.size() && vt[j].first == vt[i].first) ++j;
            const int32_t n = (int32_t)(j - i) - 1;
            if (n > 0) {
                const int32_t v = vt[i].first;
                mf.fv.push_back({v, row_pos(v, v), n, (int32_t)mf.nv});
                for (int32_t q = 1; q <= n; ++q) vrank.push_back({v, vt[i + q].second, q});
                mf.nv += n;
            }
            i = j;
        }
        for (size_t i = 0; i < pt.size();) {
            size_t j = i;
            while (j < pt.size() && pt[j].first == pt[i].first) ++j;
            const int32_t n = (int32_t)(j - i) - 1;
            if (n > 0) {
                // blocks (a, b) in row a and (b, a) in row b
                const int32_t a = (int32_t)(pt[i].first / (uint64_t)nV), b = (int32_t)(pt[i].first % (uint64_t)nV);
                mf.fp.push_back({a, b, n, 0});
                mf.fp.push_back({b, a, n, 0});
                for (int32_t q = 1; q <= n; ++q) prank.push_back({(int64_t)pt[i].first, pt[i + q].second, q});
            }
            i = j;
        }
        // pair outputs in block order (row, then column): slot runs, then
        // the column becomes the block's position in its row
        std::sort(mf.fp.begin(), mf.fp.end());
        std::vector<std::array<int32_t, 2>> pcols(mf.fp.size());  // (row, column) of each pair output
        for (size_t i = 0; i < mf.fp.size(); ++i) {
            auto &e = mf.fp[i];
            pcols[i] = {e[0], e[1]};
            e[3] = (int32_t)mf.np;
            mf.np += e[2];
            e[1] = row_pos(e[0], e[1]);
        }
        for (auto &e : mf.fv)
            if (e[1] < 0) fail_part = ADM_ERR_MESH;
        for (auto &e : mf.fp)
            if (e[1] < 0) fail_part = ADM_ERR_MESH;
        auto rank_of = [](const std::vector<std::array<int64_t, 3>> &rk, int64_t key, int64_t t) -> int64_t {
            auto it = std::lower_bound(rk.begin(), rk.end(), std::array<int64_t, 3>{key, t, INT64_MIN});
            return (it != rk.end() && (*it)[0] == key && (*it)[1] == t) ? (*it)[2] : 0;
        };
        // per tile: rows and codes of a later producer point into its table
        for (int32_t t = t0; t < t1; ++t) {
            TileOut &o = T[t];
            std::vector<int64_t> &tab = ptab[t];
            const int32_t nf = (int32_t)o.foot.size();
            for (int32_t r = 0; r < nf; ++r) {
                int32_t *row = &o.rows[(size_t)kRowWords * r];
                const int32_t v = o.foot[r];
                const int64_t qv = rank_of(vrank, v, t);
                if (qv > 0) {
                    auto it = std::lower_bound(mf.fv.begin(), mf.fv.end(), std::array<int32_t, 4>{v, INT32_MIN, 0, 0});
                    if (tab.size() >= 32768) fail_part = 1;
                    row[3] = (row[3] & 0x7fff) | 1 << 15 | (int32_t)(tab.size() << 16);
                    tab.push_back((*it)[3] + qv - 1);
                }
            }
            for (size_t j = 0; 2 * j < o.codes.size(); ++j) {
                uint32_t &x = o.codes[2 * j], &y = o.codes[2 * j + 1];
                const int32_t va = o.foot[(x >> 19) & 511], vb = o.foot[(y >> 9) & 511];
                const int64_t qp = rank_of(prank, (int64_t)pkey(va, vb, nV), t);
                if (qp == 0) continue;
                auto run = [&](int32_t r, int32_t c) {
                    const size_t oi = (size_t)(std::lower_bound(pcols.begin(), pcols.end(), std::array<int32_t, 2>{r, c}) -
                                               pcols.begin());
                    return mf.fp[oi][3] + qp - 1;
                };
                if (tab.size() + 2 > (1u << 18)) fail_part = 1;
                const uint32_t ia = (uint32_t)tab.size(), ib = ia + 1;
                tab.push_back(run(va, vb) | (int64_t)1 << 62);
                tab.push_back(run(vb, va) | (int64_t)1 << 62);
                x = (x & 0x1ffffu) | 1u << 17 | 1u << 18 | (ia >> 9) << 19;
                y = (ia & 511u) | (ib >> 9) << 9 | (ib & 511u) << 18;
            }
        }
    });
    if (fail_part == 1) {
        // a tile with more shared outputs than its table indexes: smaller tiles
        if (tile_units <= 16) return ADM_ERR_UNSUPPORTED;
        return tiles_build(m, P, with_hinges, tile_units / 2, ts);
    }
    if (fail_part) return (adm_status)fail_part.load();
    std::vector<int64_t> voff(m.n_mesh + 1, 0), poff(m.n_mesh + 1, 0);
    for (int k = 0; k < m.n_mesh; ++k) {
        voff[k + 1] = voff[k] + mfix[k].nv;
        poff[k + 1] = poff[k] + mfix[k].np;
    }
    if (voff.back() >= INT32_MAX || poff.back() >= INT32_MAX) return ADM_ERR_UNSUPPORTED;
    ts.n_vpart = voff.back();
    ts.n_ppart = poff.back();
    ts.fix_v.clear();
    ts.fix_p.clear();
    for (int k = 0; k < m.n_mesh; ++k) {
        for (auto e : mfix[k].fv) {
            e[3] += (int32_t)voff[k];
            ts.fix_v.insert(ts.fix_v.end(), e.begin(), e.end());
        }
        for (auto e : mfix[k].fp) {
            e[3] += (int32_t)poff[k];
            ts.fix_p.insert(ts.fix_p.end(), e.begin(), e.end());
        }
    }
    ts.hdr.assign((size_t)kHdr * n_tiles, 0);

    // ---- concatenate
    ts.meta_off.assign(n_tiles + 1, 0);
    ts.meta.clear();
    for (int32_t t = 0; t < n_tiles; ++t) {
        TileOut &o = T[t];
        int32_t *hd = &ts.hdr[(size_t)kHdr * t];
        const int32_t nf = (int32_t)o.foot.size();
        hd[kHdrUnit] = (int32_t)tile_off[t];
        hd[kHdrNUnit] = (int32_t)(tile_off[t + 1] - tile_off[t]);
        hd[kHdrSlot] = (int32_t)ts.slot_edge.size();
        hd[kHdrNSlot] = (int32_t)o.slot_hinge.size();
        hd[kHdrFoot] = (int32_t)ts.foot.size();
        hd[kHdrNF] = nf;
        hd[kHdrNVC] = (int32_t)o.nvc;
        hd[kHdrNPC] = (int32_t)o.npc;
        hd[kHdrNCode] = (int32_t)(o.codes.size() / 2);  // pair codes of 2 words
        // the tile's partial slots, global: vertex slots offset by the
        // mesh's first vertex slot, pair slots by its first pair slot
        const int32_t km = tile_mesh[t];
        std::vector<int32_t> tab(ptab[t].size());
        for (size_t j = 0; j < tab.size(); ++j) {
            const int64_t e = ptab[t][j];
            tab[j] = (e >> 62) & 1 ? (int32_t)((e & ~((int64_t)1 << 62)) + poff[km]) : (int32_t)(e + voff[km]);
        }
        hd[kHdrNPart] = (int32_t)tab.size();
        const int64_t rows_b = 4 * (int64_t)kRowWords * nf;
        const int64_t codes_b = 4 * (int64_t)o.codes.size();
        const int64_t tab_b = 4 * (int64_t)tab.size();
        hd[kHdrCodeOff] = (int32_t)rows_b;
        hd[kHdrPartOff] = (int32_t)(rows_b + codes_b);
        const int64_t mb = align16(rows_b + codes_b + tab_b);
        const size_t m0 = ts.meta.size();
        ts.meta.resize(m0 + mb, 0);
        unsigned char *blob = ts.meta.data() + m0;
        std::memcpy(blob, o.rows.data(), rows_b);
        std::memcpy(blob + rows_b, o.codes.data(), codes_b);
        std::memcpy(blob + rows_b + codes_b, tab.data(), tab_b);
        ts.meta_off[t + 1] = (int64_t)ts.meta.size();
        ts.max_meta = std::max(ts.max_meta, mb);
        ts.max_nf = std::max<int64_t>(ts.max_nf, nf);
        ts.max_nvc = std::max(ts.max_nvc, o.nvc);
        ts.max_npc = std::max(ts.max_npc, o.npc);
        ts.max_part = std::max<int64_t>(ts.max_part, (int64_t)tab.size());
        // unit data
        ts.foot.insert(ts.foot.end(), o.foot.begin(), o.foot.end());
        ts.unit.insert(ts.unit.end(), o.unit.begin(), o.unit.end());
        ts.unit_dst.insert(ts.unit_dst.end(), o.unit_dst.begin(), o.unit_dst.end());
        ts.slot_dst.insert(ts.slot_dst.end(), o.slot_dst.begin(), o.slot_dst.end());
        for (size_t s = 0; s < o.slot_hinge.size(); ++s) {
            ts.slot_edge.push_back(o.slot_hinge[s]);
            ts.slot_verts.insert(ts.slot_verts.end(), o.slot_v[s].begin(), o.slot_v[s].end());
            const int32_t h = o.slot_hinge[s];
            if (h >= 0) {
                ts.slot_rest.push_back(m.h_thetabar[h]);
                ts.slot_rest.push_back(m.h_abar[h] / 3.0);
            } else {  // a spring: squared rest length of the edge
                const double *a = &m.V[3 * (int64_t)o.slot_v[s][0]], *b = &m.V[3 * (int64_t)o.slot_v[s][1]];
                double l2 = 0.0;
                for (int d = 0; d < 3; ++d) l2 += (a[d] - b[d]) * (a[d] - b[d]);
                ts.slot_rest.push_back(l2);
                ts.slot_rest.push_back(0.0);
            }
        }
        for (int32_t f : o.units) {
            ts.tri_perm.push_back(f);
            for (int q = 0; q < 3; ++q) ts.tri_verts.push_back(m.F[3 * (int64_t)f + q]);
            for (int q = 0; q < 4; ++q) ts.tri_rest.push_back(m.tri_Dinv[4 * (int64_t)f + q]);
            ts.tri_rest.push_back(m.tri_area[f]);
        }
    }
    ts.n_slots = (int64_t)ts.slot_edge.size();
    // vertices no unit touches: their gradient row and diagonal block are
    // zeroed every pass
    {
        std::vector<char> seen(nV, 0);
        for (int32_t v : ts.foot) seen[v] = 1;
        for (int64_t v = 0; v < nV; ++v)
            if (!seen[v]) {
                ts.zero_verts.push_back((int32_t)v);
                const auto b = P.col.begin() + P.row_ptr[v], e = P.col.begin() + P.row_ptr[v + 1];
                ts.zero_blocks.push_back((int32_t)(std::lower_bound(b, e, (int32_t)v) - P.col.begin()));
            }
    }
    static std::atomic<int64_t> builds(0);
    ts.build_id = ++builds;
    ts.built = true;
    return ADM_OK;
}

// Cloth data on a triangle tile set (Sec. 7.1): every slot already carries
// its edge's squared rest length (a spring); here every vertex becomes the
// inertia-and-gravity term of the first unit (in tile order) that has it.
adm_status tiles_build_cloth(const HostMesh &m, TileSet &ts)
{
    if (!ts.built || ts.n_tiles == 0) return ADM_ERR_ARG;
    std::vector<double> area3(m.nV, 0.0);
    for (int64_t t = 0; t < m.nT; ++t)
        for (int c = 0; c < 3; ++c) area3[m.F[3 * t + c]] += m.tri_area[t] / 3.0;
    std::vector<char> seen(m.nV, 0);
    ts.vterm_rest.clear();
    for (int32_t t = 0; t < ts.n_tiles; ++t) {
        int32_t *hd = &ts.hdr[(size_t)kHdr * t];
        hd[kHdrVTerm] = (int32_t)ts.vterm_rest.size();
        int32_t n = 0;
        for (int32_t i = 0; i < hd[kHdrNUnit]; ++i) {
            const int64_t u = (int64_t)hd[kHdrUnit] + i;
            uint16_t *r = &ts.unit[8 * u];
            r[6] &= (uint16_t)~(7u << 2);  // the vertex-term mask (slots and rotation kept)
            r[3] = (uint16_t)n;  // first vertex term of the unit, within the tile
            for (int q = 0; q < 3; ++q) {
                const int32_t v = ts.tri_verts[3 * u + q];
                if (seen[v]) continue;
                seen[v] = 1;
                r[6] |= (uint16_t)(1u << (2 + q));
                ts.vterm_rest.push_back(area3[v]);
                ++n;
            }
        }
        if (n >= 65536) return ADM_ERR_UNSUPPORTED;
        hd[kHdrNVTerm] = n;
    }
    ts.n_vterms = (int64_t)ts.vterm_rest.size();
    ts.cloth_built = true;
    return ADM_OK;
}

}  // namespace adm
