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
// reports, per block of the pattern, which tile writes it:
//   block_writer[b] = tile id if exactly one tile writes it with a plain
//   store, -2 if it is shared (zeroed and atomically added), -1 if no tile
//   writes it; block_adds[b] = number of tiles that add into it.
// stats: {n_tiles, n_zero_blocks, n_zero_verts, FP64 shared-memory bytes (VD = 3), nnzb, nH,
//         build_ms}.  Returns 0 or an adm_status.
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
    for (int32_t t = 0; t < ts.n_tiles; ++t) {
        const int32_t *hd = &ts.hdr[8 * (size_t)t];
        const int32_t foot_begin = hd[4], nf = hd[5];
        for (int32_t r = 0; r < nf; ++r) {
            const int32_t rs = ts.row_start[foot_begin + r] & 0x7fffffff;
            const int32_t c0 = ts.code_off[foot_begin + t + r], c1 = ts.code_off[foot_begin + t + r + 1];
            for (int32_t e = 0; e < c1 - c0; ++e) {
                const uint16_t code = ts.codes[c0 + e];
                if ((code >> 14) == 0) continue;
                const int64_t b = rs + e;
                if (code & 0x2000) {
                    if (block_writer[b] >= 0) return -100;  // plain store and atomic add on one block
                    block_writer[b] = -2;
                    block_adds[b]++;
                } else {
                    if (block_writer[b] != -1) return -101;  // two plain writers
                    block_writer[b] = t;
                }
            }
        }
    }
    stats[0] = ts.n_tiles;
    stats[1] = (double)ts.zero_blocks.size();
    stats[2] = (double)ts.zero_verts.size();
    stats[3] = (double)ts.smem_bytes[1][0];
    stats[4] = (double)P.nnzb;
    stats[5] = (double)m.nH();
    stats[6] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    // every zeroed block is shared, or the diagonal block of a vertex no
    // element touches (written by nothing but the zero fill; reported as -2)
    for (int32_t b : ts.zero_blocks) {
        if (block_writer[b] == -1) {
            const int32_t r = (int32_t)(std::upper_bound(P.row_ptr.begin(), P.row_ptr.end(), b) - P.row_ptr.begin()) - 1;
            if (P.col[b] != r) return -102;
            block_writer[b] = -2;
            block_adds[b] = 2;
            continue;
        }
        if (block_writer[b] != -2) return -102;
    }
    // each tile's metadata blob holds its rows' starts, code offsets and codes
    if ((int64_t)ts.meta_off.size() != ts.n_tiles + 1 || ts.meta_off.back() != (int64_t)ts.meta.size()) return -105;
    for (int32_t t = 0; t < ts.n_tiles; ++t) {
        const int32_t *hd = &ts.hdr[8 * (size_t)t];
        const int32_t foot_begin = hd[4], nf = hd[5];
        const int64_t m0 = ts.meta_off[t];
        if (m0 % 16 != 0 || (ts.meta_off[t + 1] - m0) % 16 != 0) return -105;
        const unsigned char *blob = ts.meta.data() + m0;
        const int32_t cbase = ts.code_off[foot_begin + t];
        for (int32_t r = 0; r <= nf; ++r) {
            uint16_t c;
            std::memcpy(&c, blob + 4 * nf + 2 * r, 2);
            if (c != ts.code_off[foot_begin + t + r] - cbase) return -106;
            if (r == nf) break;
            int32_t rs;
            std::memcpy(&rs, blob + 4 * r, 4);
            if (rs != ts.row_start[foot_begin + r]) return -106;
        }
        const int32_t nc = ts.code_off[foot_begin + t + nf] - cbase;
        if (6 * nf + 2 + 2 * nc > ts.meta_off[t + 1] - m0) return -106;
        if (std::memcmp(blob + 6 * nf + 2, &ts.codes[cbase], 2 * (size_t)nc) != 0) return -106;
    }
    // every triangle and hinge belongs to exactly one tile
    std::vector<char> seen_t(nT, 0), seen_h(m.nH(), 0);
    for (int32_t e : ts.tri_perm)
        if (e < 0 || e >= nT || seen_t[e]++) return -103;
    if (with_hinges)
        for (int32_t e : ts.hinge_perm)
            if (e < 0 || e >= m.nH() || seen_h[e]++) return -104;
    return 0;
}

}  // extern "C"
