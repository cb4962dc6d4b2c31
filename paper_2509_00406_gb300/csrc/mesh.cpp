// mesh.cpp -- one-time host construction of connectivity, rest data, block
// patterns and slot maps (the "problem analysis and sparse preallocation" of
// Sec. 6.1; its cost is excluded from timings as in Sec. 7).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace adm {

adm_status mesh_validate(const HostMesh &m)
{
    if (m.nV <= 0 || m.nT <= 0 || m.n_mesh <= 0) return ADM_ERR_ARG;
    if ((int64_t)m.v_off.size() != m.n_mesh + 1 || (int64_t)m.f_off.size() != m.n_mesh + 1)
        return ADM_ERR_ARG;
    if (m.v_off[0] != 0 || m.f_off[0] != 0 || m.v_off[m.n_mesh] != m.nV ||
        m.f_off[m.n_mesh] != m.nT)
        return ADM_ERR_ARG;
    if (m.nV >= (int64_t)INT32_MAX / 4 || m.nT >= (int64_t)INT32_MAX / 24) return ADM_ERR_ARG;
    for (int k = 0; k < m.n_mesh; ++k) {
        if (m.v_off[k + 1] < m.v_off[k] || m.f_off[k + 1] < m.f_off[k]) return ADM_ERR_ARG;
        for (int64_t t = m.f_off[k]; t < m.f_off[k + 1]; ++t) {
            const int32_t *f = &m.F[3 * t];
            for (int c = 0; c < 3; ++c)
                if (f[c] < m.v_off[k] || f[c] >= m.v_off[k + 1]) return ADM_ERR_MESH;
            if (f[0] == f[1] || f[1] == f[2] || f[0] == f[2]) return ADM_ERR_MESH;
        }
    }
    for (double v : m.V)
        if (!std::isfinite(v)) return ADM_ERR_MESH;
    return ADM_OK;
}

// Rest frame of triangle (a, b, c): e1 along b - a, e2 = n x e1 with n the
// counter-clockwise normal.  In that frame the rest edge matrix is upper
// triangular, Dm = [[|u|, u.w/|u|], [0, |u x w|/|u|]], u = b - a, w = c - a.
void mesh_rest_triangles(HostMesh &m)
{
    m.tri_Dinv.assign(4 * m.nT, 0.0);
    m.tri_area.assign(m.nT, 0.0);
    for (int64_t t = 0; t < m.nT; ++t) {
        const double *a = &m.V[3 * (int64_t)m.F[3 * t + 0]];
        const double *b = &m.V[3 * (int64_t)m.F[3 * t + 1]];
        const double *c = &m.V[3 * (int64_t)m.F[3 * t + 2]];
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cx = u[1] * w[2] - u[2] * w[1];
        double cy = u[2] * w[0] - u[0] * w[2];
        double cz = u[0] * w[1] - u[1] * w[0];
        double cr = std::sqrt(cx * cx + cy * cy + cz * cz);
        double lu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double d00 = lu, d01 = (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) / lu, d11 = cr / lu;
        m.tri_Dinv[4 * t + 0] = 1.0 / d00;
        m.tri_Dinv[4 * t + 1] = -d01 / (d00 * d11);
        m.tri_Dinv[4 * t + 2] = 0.0;
        m.tri_Dinv[4 * t + 3] = 1.0 / d11;
        m.tri_area[t] = 0.5 * cr;
    }
}

// vertex -> incident faces, CSR
static void vertex_faces(const HostMesh &m, std::vector<int64_t> &off, std::vector<int32_t> &fl)
{
    off.assign(m.nV + 1, 0);
    for (int64_t i = 0; i < 3 * m.nT; ++i) off[m.F[i] + 1]++;
    for (int64_t v = 0; v < m.nV; ++v) off[v + 1] += off[v];
    fl.assign(3 * m.nT, 0);
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int64_t t = 0; t < m.nT; ++t)
        for (int c = 0; c < 3; ++c) fl[pos[m.F[3 * t + c]]++] = (int32_t)t;
}

// Interior edges with exactly two faces become hinges (Sec. 7.7 stencil).
// Every hinge is emitted once, from the face holding the directed edge e0->e1
// with e0 < e1 (face A); its partner face must hold e1->e0 (face B).
adm_status mesh_build_hinges(HostMesh &m)
{
    if (m.hinges_built) return m.hinge_error ? ADM_ERR_MESH : ADM_OK;
    m.hinges_built = true;
    std::vector<int64_t> off;
    std::vector<int32_t> fl;
    vertex_faces(m, off, fl);
    struct Rec {
        int32_t e0, e1, a, b, fa;
    };
    std::vector<Rec> recs;
    recs.reserve((size_t)(1.5 * m.nT) + 16);
    for (int64_t t = 0; t < m.nT; ++t) {
        for (int c = 0; c < 3; ++c) {
            int32_t p = m.F[3 * t + c], q = m.F[3 * t + (c + 1) % 3], o = m.F[3 * t + (c + 2) % 3];
            // other faces around p that contain q
            int n_other = 0, n_same_dir = 0;
            int32_t opp = -1;
            for (int64_t k = off[p]; k < off[p + 1]; ++k) {
                int32_t g = fl[k];
                if (g == t) continue;
                const int32_t *f = &m.F[3 * (int64_t)g];
                for (int d = 0; d < 3; ++d) {
                    if (f[d] == q && f[(d + 1) % 3] == p) {  // g traverses q -> p
                        ++n_other;
                        opp = f[(d + 2) % 3];
                    } else if (f[d] == p && f[(d + 1) % 3] == q) {  // same direction
                        ++n_other;
                        ++n_same_dir;
                    }
                }
            }
            if (n_other > 1 || n_same_dir > 0) {
                m.hinge_error = 1;
                m.H.clear();
                return ADM_ERR_MESH;
            }
            if (n_other == 1 && p < q) recs.push_back({p, q, o, opp, (int32_t)t});
        }
    }
    std::sort(recs.begin(), recs.end(), [](const Rec &x, const Rec &y) {
        return x.e0 != y.e0 ? x.e0 < y.e0 : x.e1 < y.e1;
    });
    int64_t nH = (int64_t)recs.size();
    m.H.resize(4 * nH);
    m.H_face.resize(nH);
    for (int64_t i = 0; i < nH; ++i) {
        m.H[4 * i + 0] = recs[i].e0;
        m.H[4 * i + 1] = recs[i].e1;
        m.H[4 * i + 2] = recs[i].a;
        m.H[4 * i + 3] = recs[i].b;
        m.H_face[i] = recs[i].fa;
    }
    // per-mesh hinge ranges (hinges sorted by e0, meshes own vertex ranges)
    m.h_off.assign(m.n_mesh + 1, 0);
    {
        int64_t i = 0;
        for (int k = 0; k < m.n_mesh; ++k) {
            while (i < nH && m.H[4 * i] < m.v_off[k + 1]) ++i;
            m.h_off[k + 1] = i;
        }
    }
    // rest angle: theta = atan2(-|e| det[e,u,v], (e.v)(e.u) - (e.e)(u.v)),
    // e = x1 - x0, u = xa - x0, v = xb - x1; mean area of the two faces
    m.h_thetabar.resize(nH);
    m.h_abar.resize(nH);
    for (int64_t i = 0; i < nH; ++i) {
        const double *x0 = &m.V[3 * (int64_t)m.H[4 * i + 0]];
        const double *x1 = &m.V[3 * (int64_t)m.H[4 * i + 1]];
        const double *xa = &m.V[3 * (int64_t)m.H[4 * i + 2]];
        const double *xb = &m.V[3 * (int64_t)m.H[4 * i + 3]];
        double e[3], u[3], v[3], w[3];
        for (int d = 0; d < 3; ++d) {
            e[d] = x1[d] - x0[d];
            u[d] = xa[d] - x0[d];
            v[d] = xb[d] - x1[d];
            w[d] = xb[d] - x0[d];
        }
        double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        double ev = e[0] * v[0] + e[1] * v[1] + e[2] * v[2];
        double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
        double det = e[0] * (u[1] * v[2] - u[2] * v[1]) + e[1] * (u[2] * v[0] - u[0] * v[2]) +
                     e[2] * (u[0] * v[1] - u[1] * v[0]);
        m.h_thetabar[i] = std::atan2(-std::sqrt(ee) * det, ev * eu - ee * uv);
        auto tri_area = [](const double *p, const double *q) {
            double cx = p[1] * q[2] - p[2] * q[1], cy = p[2] * q[0] - p[0] * q[2],
                   cz = p[0] * q[1] - p[1] * q[0];
            return 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
        };
        m.h_abar[i] = 0.5 * (tri_area(e, u) + tri_area(e, w));
    }
    return ADM_OK;
}

// Block pattern: row v holds v itself, every vertex sharing a face with v
// and, with hinges, the opposite wing of every hinge whose wing is v.
void mesh_build_pattern(const HostMesh &m, bool with_hinges, std::vector<int32_t> &row_ptr,
                        std::vector<int32_t> &col)
{
    std::vector<int64_t> off;
    std::vector<int32_t> fl;
    vertex_faces(m, off, fl);
    std::vector<std::vector<int32_t>> wing;
    if (with_hinges) {
        wing.resize(m.nV);
        for (int64_t i = 0; i < m.nH(); ++i) {
            wing[m.H[4 * i + 2]].push_back(m.H[4 * i + 3]);
            wing[m.H[4 * i + 3]].push_back(m.H[4 * i + 2]);
        }
    }
    row_ptr.assign(m.nV + 1, 0);
    col.clear();
    col.reserve((size_t)(m.nV * (with_hinges ? 13 : 7)));
    std::vector<int32_t> nb;
    for (int64_t v = 0; v < m.nV; ++v) {
        nb.clear();
        nb.push_back((int32_t)v);
        for (int64_t k = off[v]; k < off[v + 1]; ++k)
            for (int c = 0; c < 3; ++c) nb.push_back(m.F[3 * (int64_t)fl[k] + c]);
        if (with_hinges)
            for (int32_t w : wing[v]) nb.push_back(w);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        col.insert(col.end(), nb.begin(), nb.end());
        row_ptr[v + 1] = (int32_t)col.size();
    }
}

static int32_t block_of(const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                        int32_t i, int32_t j)
{
    auto b = col.begin() + row_ptr[i], e = col.begin() + row_ptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int32_t)(it - col.begin()) : -1;
}

void mesh_build_slots(const HostMesh &m, const std::vector<int32_t> &row_ptr,
                      const std::vector<int32_t> &col, bool hinges, std::vector<int32_t> &tri_slots,
                      std::vector<int32_t> &hinge_slots)
{
    tri_slots.resize(9 * m.nT);
    for (int64_t t = 0; t < m.nT; ++t)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                tri_slots[9 * t + 3 * a + b] = block_of(row_ptr, col, m.F[3 * t + a], m.F[3 * t + b]);
    hinge_slots.clear();
    if (!hinges) return;
    hinge_slots.resize(16 * m.nH());
    for (int64_t i = 0; i < m.nH(); ++i)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                hinge_slots[16 * i + 4 * a + b] = block_of(row_ptr, col, m.H[4 * i + a], m.H[4 * i + b]);
}

// one-rings: the edge-adjacent neighbours of every vertex, ascending (CSR)
adm_status mesh_build_rings(HostMesh &m)
{
    if (m.rings_built) return ADM_OK;
    std::vector<std::vector<int32_t>> nb(m.nV);
    for (int64_t t = 0; t < m.nT; ++t)
        for (int c = 0; c < 3; ++c) {
            const int32_t a = m.F[3 * t + c], b = m.F[3 * t + (c + 1) % 3];
            nb[a].push_back(b);
            nb[b].push_back(a);
        }
    m.ring_off.assign(m.nV + 1, 0);
    m.ring.clear();
    for (int64_t v = 0; v < m.nV; ++v) {
        std::sort(nb[v].begin(), nb[v].end());
        nb[v].erase(std::unique(nb[v].begin(), nb[v].end()), nb[v].end());
        if ((int)nb[v].size() > kMaxValence) return ADM_ERR_UNSUPPORTED;
        m.ring.insert(m.ring.end(), nb[v].begin(), nb[v].end());
        m.ring_off[v + 1] = (int32_t)m.ring.size();
    }
    m.rings_built = true;
    return ADM_OK;
}

// block pattern of one-ring terms: a term couples every pair of vertices of a
// closed one-ring, so row a holds every vertex within two edges of a
void mesh_build_ring_pattern(const HostMesh &m, std::vector<int32_t> &row_ptr, std::vector<int32_t> &col)
{
    row_ptr.assign(m.nV + 1, 0);
    col.clear();
    std::vector<int32_t> nb;
    for (int64_t a = 0; a < m.nV; ++a) {
        nb.clear();
        nb.push_back((int32_t)a);
        for (int32_t k = m.ring_off[a]; k < m.ring_off[a + 1]; ++k) {
            const int32_t w = m.ring[k];  // a is in the closed ring of w and of every neighbour of w
            nb.push_back(w);
            for (int32_t q = m.ring_off[w]; q < m.ring_off[w + 1]; ++q) nb.push_back(m.ring[q]);
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        col.insert(col.end(), nb.begin(), nb.end());
        row_ptr[a + 1] = (int32_t)col.size();
    }
}

// ring slot map: for vertex v with closed ring (v, n_0, .., n_{k-1}), the
// block of every ordered pair (a, b) of it, row-major over (k + 1)^2
void mesh_build_ring_slots(const HostMesh &m, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                           std::vector<int32_t> &slots, std::vector<int32_t> &slot_off)
{
    slot_off.assign(m.nV + 1, 0);
    slots.clear();
    std::vector<int32_t> r;
    for (int64_t v = 0; v < m.nV; ++v) {
        r.assign(1, (int32_t)v);
        r.insert(r.end(), m.ring.begin() + m.ring_off[v], m.ring.begin() + m.ring_off[v + 1]);
        for (int32_t a : r)
            for (int32_t b : r) slots.push_back(block_of(row_ptr, col, a, b));
        slot_off[v + 1] = (int32_t)slots.size();
    }
}

}  // namespace adm
