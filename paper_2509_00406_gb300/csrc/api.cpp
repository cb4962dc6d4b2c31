// api.cpp -- the C ABI of libadm (declared in include/adm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace adm;

namespace {

constexpr int kElemThreads = 128;  // must match the kernels' block size
constexpr int kChunk = 8192;        // gradient entries per norm chunk

template <typename P>
adm_status dev_alloc(adm_ctx *h, P **out, size_t bytes)
{
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return ADM_ERR_OOM;
    }
    h->owned.push_back(p);
    *out = (P *)p;
    return ADM_OK;
}

template <typename P>
adm_status upload(adm_ctx *h, P **out, const void *src, size_t bytes)
{
    adm_status s = dev_alloc(h, out, bytes);
    if (s != ADM_OK) return s;
    if (bytes && cudaMemcpy(*out, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return ADM_ERR_CUDA;
    return ADM_OK;
}

void dev_free(adm_ctx *h, void *p)
{
    if (!p) return;
    auto it = std::find(h->owned.begin(), h->owned.end(), p);
    if (it != h->owned.end()) h->owned.erase(it);
    cudaFree(p);
}

// SoA rest arrays in both precisions
adm_status upload_rest(adm_ctx *h, void **dst, const std::vector<std::vector<double>> &fields, int64_t n)
{
    std::vector<double> d(fields.size() * n);
    std::vector<float> f(fields.size() * n);
    for (size_t k = 0; k < fields.size(); ++k)
        for (int64_t i = 0; i < n; ++i) {
            d[k * n + i] = fields[k][i];
            f[k * n + i] = (float)fields[k][i];
        }
    adm_status s = upload(h, &dst[ADM_FP64], d.data(), d.size() * sizeof(double));
    if (s != ADM_OK) return s;
    return upload(h, &dst[ADM_FP32], f.data(), f.size() * sizeof(float));
}

// element blocks of `threads` elements that never straddle a mesh
adm_status build_blocks(adm_ctx *h, BlockTable &bt, const std::vector<int64_t> &elem_off, int threads)
{
    std::vector<int32_t> b, e;
    bt.mesh_block_off.assign(elem_off.size(), 0);
    for (size_t k = 0; k + 1 < elem_off.size(); ++k) {
        for (int64_t s = elem_off[k]; s < elem_off[k + 1]; s += threads) {
            b.push_back((int32_t)s);
            e.push_back((int32_t)std::min<int64_t>(s + threads, elem_off[k + 1]));
        }
        bt.mesh_block_off[k + 1] = (int32_t)b.size();
    }
    bt.n_blocks = (int32_t)b.size();
    bt.threads = threads;
    adm_status s;
    if ((s = upload(h, &bt.d_begin, b.data(), b.size() * 4)) != ADM_OK) return s;
    if ((s = upload(h, &bt.d_end, e.data(), e.size() * 4)) != ADM_OK) return s;
    if ((s = upload(h, &bt.d_mesh_block_off, bt.mesh_block_off.data(), bt.mesh_block_off.size() * 4)) != ADM_OK)
        return s;
    bt.built = true;
    return ADM_OK;
}

adm_status ensure_epart(adm_ctx *h)
{
    size_t need = std::max((size_t)h->tri_blocks.n_blocks + (size_t)h->hinge_blocks.n_blocks,
                           (size_t)h->vert_blocks.n_blocks) + 1;
    if (need <= h->epart_cap) return ADM_OK;
    dev_free(h, h->d_epart);
    h->d_epart = nullptr;
    adm_status s = dev_alloc(h, &h->d_epart, need * sizeof(double));
    if (s == ADM_OK) h->epart_cap = need;
    return s;
}

adm_status build_pattern(adm_ctx *h, int kind)
{
    Pattern &P = h->pat[kind];
    if (P.built) return ADM_OK;
    if (kind == PAT_RING) {  // one-ring terms: two-ring pattern, rings and their slot map
        adm_status s = mesh_build_rings(h->m);
        if (s != ADM_OK) return s;
        std::vector<int32_t> sl, so;
        mesh_build_ring_pattern(h->m, P.row_ptr, P.col);
        P.nnzb = (int64_t)P.col.size();
        mesh_build_ring_slots(h->m, P.row_ptr, P.col, sl, so);
        if ((s = upload(h, &P.d_row_ptr, P.row_ptr.data(), P.row_ptr.size() * 4)) != ADM_OK) return s;
        if ((s = upload(h, &P.d_col, P.col.data(), P.col.size() * 4)) != ADM_OK) return s;
        if ((s = upload(h, &P.d_ring_off, h->m.ring_off.data(), h->m.ring_off.size() * 4)) != ADM_OK) return s;
        if ((s = upload(h, &P.d_ring, h->m.ring.data(), std::max<size_t>(1, h->m.ring.size()) * 4)) != ADM_OK)
            return s;
        if ((s = upload(h, &P.d_ring_slots, sl.data(), sl.size() * 4)) != ADM_OK) return s;
        if ((s = upload(h, &P.d_ring_slot_off, so.data(), so.size() * 4)) != ADM_OK) return s;
        if ((s = build_blocks(h, h->vert_blocks, h->m.v_off, kElemThreads)) != ADM_OK) return s;
        if ((s = ensure_epart(h)) != ADM_OK) return s;
        P.built = true;
        return ADM_OK;
    }
    std::vector<int32_t> ts, hs;
    mesh_build_pattern(h->m, kind == PAT_SHELL, P.row_ptr, P.col);
    P.nnzb = (int64_t)P.col.size();
    mesh_build_slots(h->m, P.row_ptr, P.col, kind == PAT_SHELL, ts, hs);
    adm_status s;
    if ((s = upload(h, &P.d_row_ptr, P.row_ptr.data(), P.row_ptr.size() * 4)) != ADM_OK) return s;
    if ((s = upload(h, &P.d_col, P.col.data(), P.col.size() * 4)) != ADM_OK) return s;
    if ((s = upload(h, &P.d_tri_slots, ts.data(), ts.size() * 4)) != ADM_OK) return s;
    if (kind == PAT_SHELL)
        if ((s = upload(h, &P.d_hinge_slots, hs.data(), hs.size() * 4)) != ADM_OK) return s;
    P.built = true;
    return ADM_OK;
}

// hinges, their rest data, block table and the shell pattern
adm_status ensure_shell(adm_ctx *h)
{
    if (h->pat[PAT_SHELL].built) return ADM_OK;
    if (h->m.vdim != 3) return ADM_ERR_UNSUPPORTED;
    adm_status s = mesh_build_hinges(h->m);
    if (s != ADM_OK) return s;
    const int64_t nH = h->m.nH();
    if (!h->d_H && (s = upload(h, &h->d_H, h->m.H.data(), h->m.H.size() * 4)) != ADM_OK) return s;
    std::vector<double> abar3(nH);
    for (int64_t i = 0; i < nH; ++i) abar3[i] = h->m.h_abar[i] / 3.0;
    if ((s = upload_rest(h, h->d_hinge_rest, {h->m.h_thetabar, abar3}, nH)) != ADM_OK) return s;
    if ((s = build_blocks(h, h->hinge_blocks, h->m.h_off, kElemThreads)) != ADM_OK) return s;
    if ((s = ensure_epart(h)) != ADM_OK) return s;
    return build_pattern(h, PAT_SHELL);
}

// units (triangles) per tile: the option, else 192 (two blocks per SM in
// FP32, one in FP64) shrunk for small meshes so that there are about two
// tiles per SM of the 152, never below 32; the builder splits tiles further
// until they fit shared memory
int tile_tris_for(const adm_ctx *h)
{
    if (h->tile_tris > 0) return h->tile_tris;
    const int64_t per = h->m.nT / (2 * 152);
    return (int)std::min<int64_t>(192, std::max<int64_t>(32, per));
}

// device arrays of a tile set (freed before a rebuild)
void free_tiles(adm_ctx *h, TileSet &ts)
{
    void *ptrs[] = {ts.d_hdr, ts.d_foot, ts.d_tri_perm, ts.d_tri_verts, ts.d_unit, ts.d_unit_dst, ts.d_slot_dst,
                    ts.d_meta, ts.d_meta_off, ts.d_zero_verts, ts.d_zero_blocks,
                    ts.d_mesh_tile_off, ts.d_sync, ts.d_fix_v, ts.d_fix_p, ts.d_vpart, ts.d_ppart, ts.d_slot_verts,
                    ts.d_loc_tri, ts.d_loc_slot, ts.d_tri_rest[0],
                    ts.d_tri_rest[1], ts.d_slot_rest[0], ts.d_slot_rest[1], ts.d_vterm_rest[0], ts.d_vterm_rest[1]};
    for (void *p : ptrs) dev_free(h, p);
    ts = TileSet();
}

// tiles of the tiled assembler for one pattern kind, with rest data in unit order
adm_status ensure_tiles(adm_ctx *h, int kind)
{
    TileSet &ts = h->tiles[kind];
    if (ts.built) return ADM_OK;
    if (ts.d_hdr) {  // a rebuild: no pass may still read the old set
        if (cudaDeviceSynchronize() != cudaSuccess) return ADM_ERR_CUDA;
        free_tiles(h, ts);
    }
    adm_status s = build_pattern(h, kind);
    if (s != ADM_OK) return s;
    s = tiles_build(h->m, h->pat[kind], kind == PAT_SHELL, tile_tris_for(h), ts);
    if (s != ADM_OK) {
        ts = TileSet();
        return s;
    }
    auto up = [&](auto **dst, const auto &v) {
        return v.empty() ? dev_alloc(h, dst, 16) : upload(h, dst, v.data(), v.size() * sizeof(v[0]));
    };
    if ((s = up(&ts.d_hdr, ts.hdr)) != ADM_OK) return s;
    if ((s = up(&ts.d_foot, ts.foot)) != ADM_OK) return s;
    if ((s = up(&ts.d_tri_perm, ts.tri_perm)) != ADM_OK) return s;
    if ((s = up(&ts.d_tri_verts, ts.tri_verts)) != ADM_OK) return s;
    if ((s = up(&ts.d_slot_verts, ts.slot_verts)) != ADM_OK) return s;
    if ((s = up(&ts.d_unit, ts.unit)) != ADM_OK) return s;
    if ((s = up(&ts.d_unit_dst, ts.unit_dst)) != ADM_OK) return s;
    if ((s = up(&ts.d_slot_dst, ts.slot_dst)) != ADM_OK) return s;
    if ((s = up(&ts.d_meta, ts.meta)) != ADM_OK) return s;
    if ((s = up(&ts.d_meta_off, ts.meta_off)) != ADM_OK) return s;
    if ((s = up(&ts.d_zero_verts, ts.zero_verts)) != ADM_OK) return s;
    if ((s = up(&ts.d_zero_blocks, ts.zero_blocks)) != ADM_OK) return s;
    if ((s = up(&ts.d_mesh_tile_off, ts.mesh_tile_off)) != ADM_OK) return s;
    if ((s = dev_alloc(h, &ts.d_sync, 8 * sizeof(int32_t))) != ADM_OK) return s;
    if ((s = up(&ts.d_fix_v, ts.fix_v)) != ADM_OK) return s;
    if ((s = up(&ts.d_fix_p, ts.fix_p)) != ADM_OK) return s;
    {
        // partial slots, sized for FP64 and the largest vertex chunk
        const size_t cvh = h->m.vdim == 3 ? 9 : 5, nb = (size_t)h->m.vdim * h->m.vdim;
        if ((s = dev_alloc(h, &ts.d_vpart, std::max<size_t>(16, ts.n_vpart * cvh * 8))) != ADM_OK) return s;
        if ((s = dev_alloc(h, &ts.d_ppart, std::max<size_t>(16, ts.n_ppart * nb * 8))) != ADM_OK) return s;
    }
    {
        const int64_t nU = (int64_t)ts.tri_perm.size();
        std::vector<std::vector<double>> f(5, std::vector<double>(nU));
        for (int64_t i = 0; i < nU; ++i)
            for (int k = 0; k < 5; ++k) f[k][i] = ts.tri_rest[5 * i + k];
        if ((s = upload_rest(h, ts.d_tri_rest, f, nU)) != ADM_OK) return s;
        const int64_t nS = std::max<int64_t>(ts.n_slots, 1);
        std::vector<std::vector<double>> g(2, std::vector<double>(nS, 0.0));
        for (int64_t i = 0; i < ts.n_slots; ++i)
            for (int k = 0; k < 2; ++k) g[k][i] = ts.slot_rest[2 * i + k];
        if ((s = upload_rest(h, ts.d_slot_rest, g, nS)) != ADM_OK) return s;
    }
    if ((size_t)ts.n_tiles + 1 > h->epart_cap) {
        dev_free(h, h->d_epart);
        h->d_epart = nullptr;
        if ((s = dev_alloc(h, &h->d_epart, ((size_t)ts.n_tiles + 1) * sizeof(double))) != ADM_OK) return s;
        h->epart_cap = (size_t)ts.n_tiles + 1;
    }
    ts.built = true;
    return interactions_retile(h, kind, 0);  // pair-extended pattern: remap the new tiles
}

bool energy_ok(int energy, int vdim)
{
    switch (energy) {
    case ADM_SYMDIR2D:
    case ADM_ARAP2D_RESIDUAL: return vdim == 2;
    case ADM_STVK_MEMBRANE:
    case ADM_HINGE_BENDING:
    case ADM_SHELL:
    case ADM_NH_MEMBRANE:
    case ADM_MLP_MEMBRANE:
    case ADM_AREA:
    case ADM_MASS_SPRING: return vdim == 3;
    case ADM_UMBRELLA: return true;
    default: return false;
    }
}

bool needs_hinges(int energy) { return energy == ADM_HINGE_BENDING || energy == ADM_SHELL; }

// the tile set's cloth data (once): vertex terms in the unit records, their
// rest data; and the default inertial target (the rest shape) if none was set
adm_status ensure_cloth(adm_ctx *h)
{
    TileSet &ts = h->tiles[PAT_TRI];
    adm_status s = ADM_OK;
    if (!ts.cloth_built) {
        if ((s = tiles_build_cloth(h->m, ts)) != ADM_OK) return s;
        if (cudaMemcpy(ts.d_unit, ts.unit.data(), ts.unit.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(ts.d_hdr, ts.hdr.data(), ts.hdr.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return ADM_ERR_CUDA;
        std::vector<std::vector<double>> fv{ts.vterm_rest};
        if (fv[0].empty()) fv[0].push_back(0.0);
        if ((s = upload_rest(h, ts.d_vterm_rest, fv, (int64_t)fv[0].size())) != ADM_OK) return s;
    }
    if (!h->d_xhat[ADM_FP64]) return adm_set_inertia_target(h, h->m.V.data());
    return ADM_OK;
}

// tiles are built for the tiled assembler, and for the matrix-free product
// (which only the tiled kernel implements) whatever the assembler option
adm_status prepare(adm_ctx *h, int energy, bool need_tiles = false)
{
    if (!energy_ok(energy, h->m.vdim)) return ADM_ERR_UNSUPPORTED;
    if (energy == ADM_UMBRELLA) return build_pattern(h, PAT_RING);  // its own per-vertex kernel, no tiles
    adm_status s = needs_hinges(energy) ? ensure_shell(h) : build_pattern(h, PAT_TRI);
    if (energy == ADM_MLP_MEMBRANE && h->assembler != 0) return ADM_ERR_UNSUPPORTED;
    const bool cloth = energy == ADM_MASS_SPRING;
    if (s != ADM_OK || (h->assembler != 0 && !need_tiles && !h->proj && !cloth) || energy == ADM_ARAP2D_RESIDUAL)
        return s;
    s = ensure_tiles(h, needs_hinges(energy) ? PAT_SHELL : PAT_TRI);
    if (s == ADM_OK && cloth) s = ensure_cloth(h);
    if (s == ADM_OK && energy == ADM_MLP_MEMBRANE && !h->d_mlp_table)
        s = dev_alloc(h, &h->d_mlp_table, (size_t)h->m.nT * 10 * sizeof(float));
    return s;
}

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

void drop_graphs(adm_ctx *h)
{
    for (auto &g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    h->graphs.clear();
}

// direct launch, or capture once and replay (ADM_OPT_GRAPH)
adm_status run_pass(adm_ctx *h, const EvalArgs &a)
{
    if (!h->use_graph) return launch_eval(h, a);
    GraphEntry *hit = nullptr;
    for (auto &g : h->graphs)
        if (g.energy == a.energy && g.prec == a.prec && g.x == a.x && g.grad == a.grad && g.bsr == a.bsr &&
            g.e_total == a.energy_total && g.e_mesh == a.energy_per_mesh && g.gnorm == a.gnorm_per_mesh &&
            g.v == a.v && g.hv == a.hv)
            hit = &g;
    if (!hit) {
        if (!h->capture_stream &&
            cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return ADM_ERR_CUDA;
        GraphEntry g;
        g.energy = a.energy;
        g.prec = a.prec;
        g.x = a.x;
        g.grad = a.grad;
        g.bsr = a.bsr;
        g.e_total = a.energy_total;
        g.e_mesh = a.energy_per_mesh;
        g.gnorm = a.gnorm_per_mesh;
        g.v = a.v;
        g.hv = a.hv;
        EvalArgs c = a;
        c.stream = h->capture_stream;
        const int ring = h->prof_ring;
        h->prof_ring = 0;  // no per-stage events inside a graph
        if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            h->prof_ring = ring;
            return ADM_ERR_CUDA;
        }
        adm_status s = launch_eval(h, c);
        cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g.graph);
        h->prof_ring = ring;
        if (s != ADM_OK || e != cudaSuccess) {
            if (g.graph) cudaGraphDestroy(g.graph);
            cudaGetLastError();
            return s != ADM_OK ? s : ADM_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
            cudaGraphDestroy(g.graph);
            cudaGetLastError();
            return ADM_ERR_CUDA;
        }
        if (h->graphs.size() >= 8) {
            cudaGraphExecDestroy(h->graphs.front().exec);
            cudaGraphDestroy(h->graphs.front().graph);
            h->graphs.erase(h->graphs.begin());
        }
        h->graphs.push_back(g);
        hit = &h->graphs.back();
    }
    StageTimer tm(h, a.stream);
    tm.begin(ADM_STAGE_GRAPH);
    if (cudaGraphLaunch(hit->exec, a.stream) != cudaSuccess) return ADM_ERR_CUDA;
    tm.end(ADM_STAGE_GRAPH);
    return ADM_OK;
}

}  // namespace

extern "C" {

adm_status adm_create(const double *V, int64_t nV, const int32_t *F, int64_t nF, int32_t var_dim,
                      adm_handle *out)
{
    int64_t v_off[2] = {0, nV}, f_off[2] = {0, nF};
    return adm_create_batch(V, v_off, F, f_off, 1, var_dim, out);
}

adm_status adm_create_batch(const double *V, const int64_t *v_off, const int32_t *F,
                            const int64_t *f_off, int32_t n_mesh, int32_t var_dim, adm_handle *out)
{
    if (!out) return ADM_ERR_ARG;
    *out = nullptr;
    if (!V || !v_off || !F || !f_off || n_mesh <= 0 || (var_dim != 2 && var_dim != 3)) return ADM_ERR_ARG;
    adm_ctx *h = new (std::nothrow) adm_ctx();
    if (!h) return ADM_ERR_OOM;
    HostMesh &m = h->m;
    m.n_mesh = n_mesh;
    m.vdim = var_dim;
    m.v_off.assign(v_off, v_off + n_mesh + 1);
    m.f_off.assign(f_off, f_off + n_mesh + 1);
    m.nV = m.v_off[n_mesh];
    m.nT = m.f_off[n_mesh];
    adm_status s = ADM_OK;
    if (m.nV <= 0 || m.nT <= 0) s = ADM_ERR_ARG;
    if (s == ADM_OK) {
        m.V.assign(V, V + 3 * m.nV);
        m.F.assign(F, F + 3 * m.nT);
        s = mesh_validate(m);
    }
    if (s == ADM_OK) {
        mesh_rest_triangles(m);
        for (int64_t t = 0; t < m.nT; ++t)
            if (!(m.tri_area[t] > 0.0) || !std::isfinite(m.tri_Dinv[4 * t + 1])) {
                s = ADM_ERR_MESH;
                break;
            }
    }
    if (s == ADM_OK && cudaGetDevice(&h->device) != cudaSuccess) s = ADM_ERR_CUDA;
    if (s == ADM_OK) s = dev_alloc(h, &h->d_status, sizeof(int));
    if (s == ADM_OK && cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) s = ADM_ERR_CUDA;
    if (s == ADM_OK) s = upload(h, &h->d_F, m.F.data(), m.F.size() * 4);
    if (s == ADM_OK) {
        std::vector<std::vector<double>> fields(5, std::vector<double>(m.nT));
        for (int64_t t = 0; t < m.nT; ++t) {
            for (int k = 0; k < 4; ++k) fields[k][t] = m.tri_Dinv[4 * t + k];
            fields[4][t] = m.tri_area[t];
        }
        s = upload_rest(h, h->d_tri_rest, fields, m.nT);
    }
    if (s == ADM_OK) s = build_blocks(h, h->tri_blocks, m.f_off, kElemThreads);
    if (s == ADM_OK) s = ensure_epart(h);
    if (s == ADM_OK) {
        // gradient-norm chunks
        std::vector<int32_t> cb, ce, co(1, 0);
        for (int k = 0; k < n_mesh; ++k) {
            int64_t a = m.v_off[k] * var_dim, b = m.v_off[k + 1] * var_dim;
            for (int64_t c = a; c < b; c += kChunk) {
                cb.push_back((int32_t)c);
                ce.push_back((int32_t)std::min<int64_t>(c + kChunk, b));
            }
            co.push_back((int32_t)cb.size());
        }
        h->chunks.n_chunks = (int32_t)cb.size();
        s = upload(h, &h->chunks.d_begin, cb.data(), cb.size() * 4);
        if (s == ADM_OK) s = upload(h, &h->chunks.d_end, ce.data(), ce.size() * 4);
        if (s == ADM_OK) s = upload(h, &h->chunks.d_mesh_chunk_off, co.data(), co.size() * 4);
        if (s == ADM_OK) s = dev_alloc(h, &h->d_gpart, cb.size() * sizeof(double));
        if (s == ADM_OK) s = dev_alloc(h, &h->d_emesh, (size_t)n_mesh * sizeof(double));
        h->chunks.built = true;
    }
    if (s == ADM_OK) s = build_pattern(h, PAT_TRI);
    if (s != ADM_OK) {
        adm_destroy(h);
        return s;
    }
    *out = h;
    return ADM_OK;
}

adm_status adm_set_params(adm_handle h, adm_energy energy, const double *p, int32_t np)
{
    if (!h || np < 0 || (np > 0 && !p)) return ADM_ERR_ARG;
    EnergyParams q;
    if (energy == ADM_HINGE_BENDING) {
        if (np > 2) return ADM_ERR_ARG;
        if (np > 0) q.kb = p[0];
        if (np > 1) q.h = p[1];
    } else if (energy == ADM_SHELL || energy == ADM_STVK_MEMBRANE || energy == ADM_NH_MEMBRANE ||
               energy == ADM_MLP_MEMBRANE) {
        if (np > (energy == ADM_SHELL ? 5 : 3)) return ADM_ERR_ARG;
        if (np > 0) q.E = p[0];
        if (np > 1) q.nu = p[1];
        if (np > 2) q.t = p[2];
        if (np > 3) q.kb = p[3];
        if (np > 4) q.h = p[4];
    } else if (energy == ADM_UMBRELLA) {
        if (np > 1 || (np == 1 && !std::isfinite(p[0]))) return ADM_ERR_ARG;
        if (np == 1) q.w = p[0];
    } else if (energy == ADM_MASS_SPRING) {
        if (np > 6) return ADM_ERR_ARG;
        double *dst[6] = {&q.k, &q.dt, &q.rho, &q.g[0], &q.g[1], &q.g[2]};
        for (int i = 0; i < np; ++i) {
            if (!std::isfinite(p[i])) return ADM_ERR_ARG;
            *dst[i] = p[i];
        }
    } else if (np != 0) {
        return ADM_ERR_ARG;
    }
    h->params[energy] = q;
    drop_graphs(h);
    return ADM_OK;
}

adm_status adm_set_option(adm_handle h, adm_option option, int64_t value)
{
    if (!h) return ADM_ERR_ARG;
    if (option != ADM_OPT_PROFILE) drop_graphs(h);
    switch (option) {
    case ADM_OPT_GRAPH:
        if (value != 0 && value != 1) return ADM_ERR_ARG;
        h->use_graph = (int)value;
        return ADM_OK;
    case ADM_OPT_ASSEMBLER:
        if (value != 0 && value != 1) return ADM_ERR_ARG;
        h->assembler = (int)value;
        return ADM_OK;
    case ADM_OPT_TILE_THREADS:
        if (value != 0 && value != 128 && value != 256) return ADM_ERR_ARG;
        if ((value == 0 ? 256 : (int)value) != h->tile_threads) drop_graphs(h);
        h->tile_threads = value == 0 ? 256 : (int)value;
        return ADM_OK;
    case ADM_OPT_MLP_NET:  // 0 mma.sync, 1 tcgen05 (the default)
        if (value != 0 && value != 1) return ADM_ERR_ARG;
        if ((int)value != h->mlp_net) drop_graphs(h);
        h->mlp_net = (int)value;
        return ADM_OK;
    case ADM_OPT_TILE_TRIS:
        if (value != 0 && (value < 1 || value > 4096)) return ADM_ERR_ARG;
        if (value != h->tile_tris)
            for (auto &ts : h->tiles) ts.built = false;  // rebuilt on next use
        h->tile_tris = (int)value;
        return ADM_OK;
    case ADM_OPT_BLOCK_THREADS:
        if (value != kElemThreads) return ADM_ERR_UNSUPPORTED;
        return ADM_OK;
    case ADM_OPT_PROFILE: {
        if (value < 0 || value > 4096) return ADM_ERR_ARG;
        for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
        h->prof_ev.clear();
        h->prof_ran.clear();
        h->prof_ring = 0;
        h->prof_next = h->prof_count = 0;
        if (value == 0) return ADM_OK;
        h->prof_ev.resize((size_t)value * ADM_N_STAGES * 2);
        h->prof_ran.assign((size_t)value * ADM_N_STAGES, 0);
        for (auto &e : h->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return ADM_ERR_CUDA;
        h->prof_ring = (int)value;
        return ADM_OK;
    }
    default: return ADM_ERR_ARG;
    }
}

// the block count a pass on pattern `kind` writes
static int64_t pass_nnzb(const adm_ctx *h, int kind)
{
    return pattern_extended(h, kind) ? h->inter.nnzb : h->pat[kind].nnzb;
}

adm_status adm_pattern(adm_handle h, adm_energy energy, int32_t *block, int64_t *n_rows, int64_t *nnzb,
                       const int32_t **row_ptr_dev, const int32_t **col_dev)
{
    if (!h) return ADM_ERR_ARG;
    if (energy == ADM_ARAP2D_RESIDUAL) energy = ADM_SYMDIR2D;  // J^T J lives on the triangle pattern
    adm_status s = prepare(h, energy);
    if (s != ADM_OK) return s;
    const int kind = energy == ADM_UMBRELLA ? PAT_RING : (needs_hinges(energy) ? PAT_SHELL : PAT_TRI);
    const Pattern &P = h->pat[kind];
    const Interactions &I = h->inter;
    const bool ext = pattern_extended(h, kind);  // extended by contact terms
    if (block) *block = h->m.vdim;
    if (n_rows) *n_rows = h->m.nV;
    if (nnzb) *nnzb = pass_nnzb(h, kind);
    if (row_ptr_dev) *row_ptr_dev = ext ? I.d_rp[I.active] : P.d_row_ptr;
    if (col_dev) *col_dev = ext ? I.d_col[I.active] : P.d_col;
    return ADM_OK;
}

adm_status adm_jac_pattern(adm_handle h, adm_energy energy, int64_t *n_rows, int64_t *n_cols, int64_t *nnz,
                           const int32_t **row_ptr_dev, const int32_t **col_dev)
{
    if (!h) return ADM_ERR_ARG;
    if (energy != ADM_ARAP2D_RESIDUAL || h->m.vdim != 2) return ADM_ERR_UNSUPPORTED;
    const HostMesh &m = h->m;
    if (!h->d_jac_row_ptr) {
        std::vector<int32_t> rp(4 * m.nT + 1), col(24 * m.nT);
        for (int64_t r = 0; r <= 4 * m.nT; ++r) rp[r] = (int32_t)(6 * r);
        for (int64_t t = 0; t < m.nT; ++t) {
            int32_t v[3] = {m.F[3 * t], m.F[3 * t + 1], m.F[3 * t + 2]};
            std::sort(v, v + 3);
            for (int i = 0; i < 4; ++i)
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 2; ++d) col[24 * t + 6 * i + 2 * a + d] = 2 * v[a] + d;
        }
        adm_status s = upload(h, &h->d_jac_row_ptr, rp.data(), rp.size() * 4);
        if (s == ADM_OK) s = upload(h, &h->d_jac_col, col.data(), col.size() * 4);
        if (s != ADM_OK) return s;
    }
    if (n_rows) *n_rows = 4 * m.nT;
    if (n_cols) *n_cols = 2 * m.nV;
    if (nnz) *nnz = 24 * m.nT;
    if (row_ptr_dev) *row_ptr_dev = h->d_jac_row_ptr;
    if (col_dev) *col_dev = h->d_jac_col;
    return ADM_OK;
}

adm_status adm_hinges(adm_handle h, const int32_t **hinges_dev, int64_t *n_hinges)
{
    if (!h) return ADM_ERR_ARG;
    adm_status s = ensure_shell(h);
    if (s != ADM_OK) return s;
    if (hinges_dev) *hinges_dev = h->d_H;
    if (n_hinges) *n_hinges = h->m.nH();
    return ADM_OK;
}

adm_status adm_slot_map(adm_handle h, adm_energy energy, const int32_t **slots_dev, int64_t *n_entries)
{
    if (!h) return ADM_ERR_ARG;
    // triangle and hinge elements only (the one-ring and mass-spring terms
    // have no per-triangle slot map)
    if (energy == ADM_UMBRELLA || energy == ADM_MASS_SPRING) return ADM_ERR_UNSUPPORTED;
    adm_status s = prepare(h, energy);
    if (s != ADM_OK) return s;
    const bool hin = needs_hinges(energy);
    Pattern &P = h->pat[hin ? PAT_SHELL : PAT_TRI];
    const bool tri = energy != ADM_HINGE_BENDING;
    const int64_t nt = tri ? 9 * h->m.nT : 0, nh = hin ? 16 * h->m.nH() : 0;
    if (!P.d_all_slots || P.n_all_slots != nt + nh) {
        dev_free(h, P.d_all_slots);
        P.d_all_slots = nullptr;
        if ((s = dev_alloc(h, &P.d_all_slots, (nt + nh) * 4)) != ADM_OK) return s;
        if (nt && cudaMemcpy(P.d_all_slots, P.d_tri_slots, nt * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
            return ADM_ERR_CUDA;
        if (nh && cudaMemcpy(P.d_all_slots + nt, P.d_hinge_slots, nh * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
            return ADM_ERR_CUDA;
        P.n_all_slots = nt + nh;
    }
    if (slots_dev) *slots_dev = P.d_all_slots;
    if (n_entries) *n_entries = nt + nh;
    return ADM_OK;
}

adm_status adm_eval_batch(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev,
                          double *energy_per_mesh_dev, double *gnorm_dev, void *grad_dev, void *bsr_vals_dev,
                          void *stream)
{
    if (!h || !x_dev || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    if (gnorm_dev && !grad_dev) return ADM_ERR_ARG;
    if (energy == ADM_ARAP2D_RESIDUAL) return ADM_ERR_UNSUPPORTED;
    if (energy == ADM_MLP_MEMBRANE && (prec != ADM_FP32 || !h->d_mlp_theta)) return ADM_ERR_UNSUPPORTED;
    adm_status s = prepare(h, energy);
    if (s != ADM_OK) return s;
    EvalArgs a;
    a.energy = energy;
    a.prec = prec;
    a.vdim = h->m.vdim;
    a.x = x_dev;
    a.grad = grad_dev;
    a.bsr = bsr_vals_dev;
    a.energy_total = nullptr;
    a.energy_per_mesh = energy_per_mesh_dev;
    a.gnorm_per_mesh = gnorm_dev;
    a.stream = as_stream(stream);
    return run_pass(h, a);
}

adm_status adm_eval(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev, double *energy_dev,
                    void *grad_dev, void *bsr_vals_dev, void *stream)
{
    if (!h || !x_dev || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    if (energy == ADM_ARAP2D_RESIDUAL) return ADM_ERR_UNSUPPORTED;
    if (energy == ADM_MLP_MEMBRANE && (prec != ADM_FP32 || !h->d_mlp_theta)) return ADM_ERR_UNSUPPORTED;
    adm_status s = prepare(h, energy);
    if (s != ADM_OK) return s;
    EvalArgs a;
    a.energy = energy;
    a.prec = prec;
    a.vdim = h->m.vdim;
    a.x = x_dev;
    a.grad = grad_dev;
    a.bsr = bsr_vals_dev;
    a.energy_total = energy_dev;
    a.energy_per_mesh = nullptr;
    a.gnorm_per_mesh = nullptr;
    a.stream = as_stream(stream);
    return run_pass(h, a);
}

adm_status adm_set_contacts(adm_handle h, adm_energy energy, const int32_t *pairs, int64_t n_pairs,
                            const int32_t *vf, int64_t n_vf, double kappa, double dhat, double area, double h_step,
                            void *stream)
{
    if (!h || n_pairs < 0 || n_vf < 0 || (n_pairs > 0 && !pairs) || (n_vf > 0 && !vf) || !(dhat > 0.0) ||
        !std::isfinite(kappa) || !std::isfinite(area) || !std::isfinite(h_step))
        return ADM_ERR_ARG;
    if (h->m.vdim != 3 || !energy_ok(energy, 3) || energy == ADM_ARAP2D_RESIDUAL || energy == ADM_UMBRELLA)
        return ADM_ERR_UNSUPPORTED;
    adm_status s = prepare(h, energy, true);
    if (s != ADM_OK) return s;
    drop_graphs(h);
    return interactions_set(h, needs_hinges(energy) ? PAT_SHELL : PAT_TRI, pairs, n_pairs, vf, n_vf, kappa, dhat,
                            area, h_step, as_stream(stream));
}

adm_status adm_set_interactions(adm_handle h, adm_energy energy, const int32_t *pairs, int64_t n_pairs,
                                double kappa, double dhat, double area, double h_step, void *stream)
{
    return adm_set_contacts(h, energy, pairs, n_pairs, nullptr, 0, kappa, dhat, area, h_step, stream);
}

adm_status adm_set_inertia_target(adm_handle h, const double *xhat_host)
{
    if (!h || !xhat_host) return ADM_ERR_ARG;
    if (h->m.vdim != 3) return ADM_ERR_UNSUPPORTED;
    const int64_t n = h->m.nV * 3;
    std::vector<std::vector<double>> f(1, std::vector<double>(xhat_host, xhat_host + n));  // vertex-major like x
    for (double v : f[0])
        if (!std::isfinite(v)) return ADM_ERR_ARG;
    dev_free(h, h->d_xhat[0]);
    dev_free(h, h->d_xhat[1]);
    h->d_xhat[0] = h->d_xhat[1] = nullptr;
    drop_graphs(h);
    return upload_rest(h, h->d_xhat, f, n);
}

adm_status adm_set_projection(adm_handle h, int32_t enable, double eps)
{
    if (!h || (enable != 0 && enable != 1) || !(eps >= 0.0) || !std::isfinite(eps)) return ADM_ERR_ARG;
    if (h->proj != enable || h->proj_eps != eps) drop_graphs(h);
    h->proj = enable;
    h->proj_eps = eps;
    return ADM_OK;
}

adm_status adm_eval_hvp(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev, const void *v_dev,
                        double *energy_dev, void *grad_dev, void *hv_dev, void *stream)
{
    if (!h || !x_dev || !v_dev || !hv_dev || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    if (energy == ADM_ARAP2D_RESIDUAL) return ADM_ERR_UNSUPPORTED;
    if (energy == ADM_MLP_MEMBRANE && (prec != ADM_FP32 || !h->d_mlp_theta)) return ADM_ERR_UNSUPPORTED;
    adm_status s = prepare(h, energy, true);
    if (s != ADM_OK) return s;
    EvalArgs a;
    a.energy = energy;
    a.prec = prec;
    a.vdim = h->m.vdim;
    a.x = x_dev;
    a.grad = grad_dev;
    a.bsr = nullptr;
    a.energy_total = energy_dev;
    a.energy_per_mesh = nullptr;
    a.gnorm_per_mesh = nullptr;
    a.stream = as_stream(stream);
    a.v = v_dev;
    a.hv = hv_dev;
    return run_pass(h, a);
}

adm_status adm_eval_batch_host(adm_handle h, adm_energy energy, adm_precision prec, const void *x_host,
                               double *energy_per_mesh_host, double *gnorm_host, void *grad_host,
                               void *bsr_vals_host)
{
    if (!h || !x_host || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    adm_status s = prepare(h, energy);
    if (s != ADM_OK) return s;
    const HostMesh &m = h->m;
    const size_t es = prec == ADM_FP32 ? 4 : 8;
    const size_t xb = es * m.nV * m.vdim;
    // the block count of the pattern the pass writes: extended by contact
    // terms when they are set on it
    const int kind = energy == ADM_UMBRELLA ? PAT_RING : (needs_hinges(energy) ? PAT_SHELL : PAT_TRI);
    const int64_t nnzb = pass_nnzb(h, kind);
    const size_t bb = es * nnzb * m.vdim * m.vdim;
    if (!h->own_stream && cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return ADM_ERR_CUDA;
    auto grow = [&](void **p, size_t &cap, size_t need) -> adm_status {
        if (need <= cap) return ADM_OK;
        dev_free(h, *p);
        *p = nullptr;
        cap = 0;
        adm_status r = dev_alloc(h, p, need);
        if (r == ADM_OK) cap = need;
        return r;
    };
    if ((s = grow(&h->d_stage_x, h->stage_x_bytes, xb)) != ADM_OK) return s;
    if ((s = grow(&h->d_stage_grad, h->stage_grad_bytes, xb)) != ADM_OK) return s;
    if ((s = grow(&h->d_stage_bsr, h->stage_bsr_bytes, bb)) != ADM_OK) return s;
    if (!h->d_stage_e) {
        if ((s = dev_alloc(h, &h->d_stage_e, m.n_mesh * sizeof(double))) != ADM_OK) return s;
        if ((s = dev_alloc(h, &h->d_stage_gn, m.n_mesh * sizeof(double))) != ADM_OK) return s;
    }
    cudaStream_t st = h->own_stream;
    // A batch on the tiled path is fed in mesh ranges: range k's copy runs on
    // the copy stream while the kernels of the ranges before it run, and its
    // own kernels wait for it.
    const int kSplit = 4;
    const bool tiled = h->assembler == 0 || energy == ADM_MASS_SPRING || h->proj;
    const bool split = m.n_mesh >= 2 && tiled && h->inter.n_terms() == 0 && energy != ADM_MLP_MEMBRANE &&
                       energy != ADM_UMBRELLA && energy != ADM_ARAP2D_RESIDUAL && energy_ok(energy, m.vdim);
    if (split) {
        if (!h->copy_stream && cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            return ADM_ERR_CUDA;
        const int n_split = std::min<int>(kSplit, (int)m.n_mesh);
        for (cudaStream_t &cs : h->split_stream)
            if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return ADM_ERR_CUDA;
        if (!h->split_start && cudaEventCreateWithFlags(&h->split_start, cudaEventDisableTiming) != cudaSuccess)
            return ADM_ERR_CUDA;
        for (auto *evs : {&h->split_ev, &h->split_done})
            while ((int)evs->size() < n_split) {
                cudaEvent_t e;
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return ADM_ERR_CUDA;
                evs->push_back(e);
            }
        // the first range is half the size of the others, so that the
        // kernels start after a short copy: boundaries at (2k - 1) / (2n - 1)
        // of the vertices, each range at least one mesh
        h->split_mesh.assign(1, 0);
        for (int k = 1; k < n_split; ++k) {
            const int64_t target = m.nV * (2 * k - 1) / (2 * n_split - 1);
            int32_t mk = (int32_t)(std::lower_bound(m.v_off.begin(), m.v_off.end(), target) - m.v_off.begin());
            mk = std::max(mk, h->split_mesh.back() + 1);
            mk = std::min(mk, (int32_t)m.n_mesh - (n_split - k));
            h->split_mesh.push_back(mk);
        }
        h->split_mesh.push_back((int32_t)m.n_mesh);
        const size_t vb = es * m.vdim;  // bytes of one vertex of x
        for (int k = 0; k < n_split; ++k) {
            const int64_t v0 = m.v_off[h->split_mesh[k]], v1 = m.v_off[h->split_mesh[k + 1]];
            if (cudaMemcpyAsync((char *)h->d_stage_x + v0 * vb, (const char *)x_host + v0 * vb, (v1 - v0) * vb,
                                cudaMemcpyHostToDevice, h->copy_stream) != cudaSuccess ||
                cudaEventRecord(h->split_ev[k], h->copy_stream) != cudaSuccess)
                return ADM_ERR_CUDA;
        }
        EvalArgs a;
        a.energy = energy;
        a.prec = prec;
        a.vdim = m.vdim;
        a.x = h->d_stage_x;
        a.grad = h->d_stage_grad;
        a.bsr = h->d_stage_bsr;
        a.energy_total = nullptr;
        a.energy_per_mesh = h->d_stage_e;
        a.gnorm_per_mesh = h->d_stage_gn;
        a.stream = st;
        a.n_split = n_split;
        a.split_mesh = h->split_mesh.data();
        a.split_ready = h->split_ev.data();
        if ((s = launch_eval(h, a)) != ADM_OK) return s;
    } else {
        if (cudaMemcpyAsync(h->d_stage_x, x_host, xb, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ADM_ERR_CUDA;
        s = adm_eval_batch(h, energy, prec, h->d_stage_x, h->d_stage_e, h->d_stage_gn, h->d_stage_grad,
                           h->d_stage_bsr, st);
        if (s != ADM_OK) return s;
    }
    if (energy_per_mesh_host &&
        cudaMemcpyAsync(energy_per_mesh_host, h->d_stage_e, m.n_mesh * sizeof(double), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
        return ADM_ERR_CUDA;
    if (gnorm_host && cudaMemcpyAsync(gnorm_host, h->d_stage_gn, m.n_mesh * sizeof(double),
                                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ADM_ERR_CUDA;
    if (grad_host && cudaMemcpyAsync(grad_host, h->d_stage_grad, xb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ADM_ERR_CUDA;
    if (bsr_vals_host &&
        cudaMemcpyAsync(bsr_vals_host, h->d_stage_bsr, bb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ADM_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status adm_check_bounded_wait(void *stream) { return bounded_wait_check(as_stream(stream)); }

adm_status adm_autotune(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev,
                        int32_t *best_tile_tris, int32_t *best_threads, float *best_ms)
{
    if (!h || !x_dev || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    if (energy == ADM_ARAP2D_RESIDUAL || energy == ADM_MLP_MEMBRANE || energy == ADM_UMBRELLA ||
        !energy_ok(energy, h->m.vdim))
        return ADM_ERR_UNSUPPORTED;
    const int saved_asm = h->assembler, saved_graph = h->use_graph, saved_ring = h->prof_ring;
    h->assembler = 0;
    h->use_graph = 0;
    h->prof_ring = 0;
    const int kind = needs_hinges(energy) ? PAT_SHELL : PAT_TRI;
    adm_status s = needs_hinges(energy) ? ensure_shell(h) : build_pattern(h, PAT_TRI);
    const size_t es = prec == ADM_FP32 ? 4 : 8;
    const int vd = h->m.vdim;
    void *g = nullptr, *H = nullptr;
    double *e = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == ADM_OK && (cudaMalloc(&g, es * h->m.nV * vd) != cudaSuccess ||
                        cudaMalloc(&H, es * pass_nnzb(h, kind) * vd * vd) != cudaSuccess ||
                        cudaMalloc(&e, sizeof(double) * h->m.n_mesh) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        s = ADM_ERR_OOM;
    // (threads per block, units per tile); 128-thread blocks only in FP32,
    // where four of them share an SM at 128 registers
    struct Cand {
        int threads, units;
    };
    std::vector<Cand> cand;
    for (int u : {96, 128, 160, 192, 224}) cand.push_back({256, u});
    if (prec == ADM_FP32 && !h->proj)
        for (int u : {48, 64, 96, 112}) cand.push_back({128, u});
    Cand best{-1, -1};
    float best_t = 1e30f;
    int built_units = -1;
    for (const Cand &c : cand) {
        if (s != ADM_OK) break;
        h->tile_threads = c.threads;
        if (c.units != built_units) {
            h->tile_tris = c.units;
            h->tiles[kind].built = false;
            if ((s = ensure_tiles(h, kind)) != ADM_OK) break;
            built_units = c.units;
        }
        EvalArgs a;
        a.energy = energy;
        a.prec = prec;
        a.vdim = vd;
        a.x = x_dev;
        a.grad = g;
        a.bsr = H;
        a.energy_total = nullptr;
        a.energy_per_mesh = e;
        a.gnorm_per_mesh = nullptr;
        a.stream = st;
        for (int w = 0; w < 2 && s == ADM_OK; ++w) s = launch_eval(h, a);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5 && s == ADM_OK; ++r) s = launch_eval(h, a);
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (s == ADM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            s = ADM_ERR_CUDA;
        if (s == ADM_OK && ms / 5 < best_t) {
            best_t = ms / 5;
            best = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(g);
    cudaFree(H);
    cudaFree(e);
    h->assembler = saved_asm;
    h->use_graph = saved_graph;
    h->prof_ring = saved_ring;
    if (s != ADM_OK) return s;
    h->tile_tris = best.units;
    h->tile_threads = best.threads;
    h->tiles[kind].built = false;
    if ((s = ensure_tiles(h, kind)) != ADM_OK) return s;
    h->tuned[{(int)energy, (int)prec}] = best.units;
    drop_graphs(h);
    if (best_tile_tris) *best_tile_tris = best.units;
    if (best_threads) *best_threads = best.threads;
    if (best_ms) *best_ms = best_t;
    return ADM_OK;
}

adm_status adm_eval_jacobian(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev, void *r_dev,
                             void *jac_vals_dev, void *jtj_bsr_vals_dev, void *stream)
{
    if (!h || !x_dev || !r_dev || (prec != ADM_FP32 && prec != ADM_FP64)) return ADM_ERR_ARG;
    if (energy != ADM_ARAP2D_RESIDUAL || h->m.vdim != 2) return ADM_ERR_UNSUPPORTED;
    adm_status s = build_pattern(h, PAT_TRI);
    if (s != ADM_OK) return s;
    return launch_jacobian(h, prec, x_dev, r_dev, jac_vals_dev, jtj_bsr_vals_dev, as_stream(stream));
}

adm_status adm_profile_read(adm_handle h, float *avg_ms, int32_t *n_launches, int32_t n_stages)
{
    if (!h || !avg_ms || n_stages < 0 || n_stages > ADM_N_STAGES || h->prof_ring <= 0) return ADM_ERR_ARG;
    double sum[ADM_N_STAGES] = {0};
    int cnt[ADM_N_STAGES] = {0};
    for (int i = 0; i < h->prof_count; ++i) {
        int slot = (h->prof_next - 1 - i + h->prof_ring) % h->prof_ring;
        for (int k = 0; k < ADM_N_STAGES; ++k) {
            if (!h->prof_ran[slot * ADM_N_STAGES + k]) continue;
            cudaEvent_t e0 = h->prof_ev[(slot * ADM_N_STAGES + k) * 2], e1 = h->prof_ev[(slot * ADM_N_STAGES + k) * 2 + 1];
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                return ADM_ERR_CUDA;
            sum[k] += ms;
            cnt[k]++;
        }
    }
    for (int k = 0; k < n_stages; ++k) {
        avg_ms[k] = cnt[k] ? (float)(sum[k] / cnt[k]) : 0.0f;
        if (n_launches) n_launches[k] = cnt[k];
    }
    h->prof_count = 0;
    h->prof_next = 0;
    return ADM_OK;
}

adm_status adm_mlp_eval(const float *theta, const float *norm, int64_t n, const float *I, float *out, void *stream)
{
    if (!theta || !norm || n < 0 || (n > 0 && (!I || !out))) return ADM_ERR_ARG;
    return mlp_eval_samples(theta, norm, n, I, out, as_stream(stream));
}

size_t adm_mlp_workspace_size(void) { return mlp_workspace_bytes(); }

adm_status adm_mlp_loss_grad(const float *theta, const float *norm, int64_t n, const float *I, const float *psi,
                             const float *dpsi, float beta, double *loss, float *grad, void *workspace,
                             size_t workspace_bytes, void *stream)
{
    if (!theta || !norm || n <= 0 || !I || !psi || !dpsi || !grad || !workspace) return ADM_ERR_ARG;
    return mlp_loss_grad(theta, norm, n, I, psi, dpsi, beta, loss, grad, workspace, workspace_bytes,
                         as_stream(stream));
}

adm_status adm_mlp_adam(float *theta, float *m, float *v, const float *grad, int64_t step, float lr, float beta1,
                        float beta2, float eps, void *stream)
{
    if (!theta || !m || !v || !grad || step < 1) return ADM_ERR_ARG;
    return mlp_adam(theta, m, v, grad, step, lr, beta1, beta2, eps, as_stream(stream));
}

adm_status adm_mlp_nh_targets(int64_t n, const float *F, double E, double nu, float *I, float *psi, float *dpsi,
                              void *stream)
{
    if (n < 0 || (n > 0 && (!F || !I || !psi || !dpsi))) return ADM_ERR_ARG;
    EnergyParams p;
    p.E = E;
    p.nu = nu;
    return mlp_nh_targets(n, F, p.mu(), p.lambda(), I, psi, dpsi, as_stream(stream));
}

adm_status adm_mlp_attach(adm_handle h, const float *theta, const float *norm)
{
    if (!h || !theta || !norm) return ADM_ERR_ARG;
    adm_status s;
    if (!h->d_mlp_theta) {
        if ((s = dev_alloc(h, &h->d_mlp_theta, ADM_MLP_NPARAM * sizeof(float))) != ADM_OK) return s;
        if ((s = dev_alloc(h, &h->d_mlp_norm, 8 * sizeof(float))) != ADM_OK) return s;
    }
    if (cudaMemcpy(h->d_mlp_theta, theta, ADM_MLP_NPARAM * sizeof(float), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(h->d_mlp_norm, norm, 8 * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return ADM_ERR_CUDA;
    drop_graphs(h);
    return ADM_OK;
}

adm_status adm_get_status(adm_handle h)
{
    if (!h) return ADM_ERR_ARG;
    int st = 0;
    if (cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ADM_ERR_CUDA;
    if (st & ST_TIMEOUT) return ADM_ERR_TIMEOUT;
    if (st & ST_DOMAIN) return ADM_ERR_DOMAIN;
    return ADM_OK;
}

const char *adm_strerror(adm_status s)
{
    switch (s) {
    case ADM_OK: return "ok";
    case ADM_ERR_ARG: return "invalid argument";
    case ADM_ERR_MESH: return "invalid mesh (index range, degenerate rest triangle, non-manifold or "
                              "inconsistently oriented edge)";
    case ADM_ERR_DOMAIN: return "element outside the energy's domain (folded triangle, degenerate hinge, "
                                "non-finite value)";
    case ADM_ERR_CUDA: return "CUDA runtime error";
    case ADM_ERR_TIMEOUT: return "bounded device wait ran out";
    case ADM_ERR_OOM: return "device allocation failed";
    case ADM_ERR_UNSUPPORTED: return "unsupported energy / precision / var_dim combination";
    }
    return "unknown status";
}

void adm_destroy(adm_handle h)
{
    if (!h) return;
    if (h->own_stream) {
        cudaStreamSynchronize(h->own_stream);
        cudaStreamDestroy(h->own_stream);
    }
    drop_graphs(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    for (cudaStream_t cs : h->split_stream)
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
    for (cudaEvent_t e : h->split_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->split_done) cudaEventDestroy(e);
    if (h->split_start) cudaEventDestroy(h->split_start);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    for (void *p : h->owned) cudaFree(p);
    delete h;
}

}  // extern "C"
