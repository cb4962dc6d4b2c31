// internal.h -- host-side structures shared by the C ABI, the mesh builder and
// the kernel launchers of libadm.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "adm.h"

namespace adm {

// stencil sets that own a block pattern
enum PatternKind { PAT_TRI = 0, PAT_SHELL = 1, PAT_RING = 2, PAT_COUNT = 3 };
constexpr int kMaxValence = 12;  // one-ring terms: vertices of higher valence are rejected

// device status bits (latched by kernels with atomicOr)
enum StatusBits { ST_DOMAIN = 1, ST_TIMEOUT = 2 };

struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
};

// mesh as given by the caller plus everything derived from it on the host
struct HostMesh {
    int64_t nV = 0, nT = 0;
    int vdim = 3;
    int n_mesh = 1;
    std::vector<double> V;          // nV * 3 rest positions
    std::vector<int32_t> F;         // nT * 3
    std::vector<int64_t> v_off;     // n_mesh + 1
    std::vector<int64_t> f_off;     // n_mesh + 1
    // hinges (built on demand): canonical (e0, e1, a, b), e0 < e1, sorted
    bool hinges_built = false;
    int hinge_error = 0;
    std::vector<int32_t> H;         // nH * 4
    std::vector<int32_t> H_face;    // face A of every hinge
    std::vector<int64_t> h_off;     // n_mesh + 1 hinge offsets
    // rest data (double)
    std::vector<double> tri_Dinv;   // nT * 4, row-major
    std::vector<double> tri_area;   // nT
    std::vector<double> h_thetabar; // nH
    std::vector<double> h_abar;     // nH, mean rest area of the two faces
    int64_t nH() const { return (int64_t)H.size() / 4; }
    // one-rings (built on demand): ascending edge-adjacent neighbours
    bool rings_built = false;
    std::vector<int32_t> ring_off;  // nV + 1
    std::vector<int32_t> ring;
};

struct Pattern {
    bool built = false;
    std::vector<int32_t> row_ptr, col;
    int32_t *d_row_ptr = nullptr, *d_col = nullptr;
    int64_t nnzb = 0;
    // slot maps: global block of (v_a, v_b) per element, row-major a * nv + b
    int32_t *d_tri_slots = nullptr;    // nT * 9
    int32_t *d_hinge_slots = nullptr;  // nH * 16 (shell pattern only)
    int32_t *d_all_slots = nullptr;    // concatenation exported by adm_slot_map
    int64_t n_all_slots = 0;
    // one-ring pattern only: rings and the ring slot map (mesh_build_ring_slots)
    int32_t *d_ring_off = nullptr, *d_ring = nullptr, *d_ring_slots = nullptr, *d_ring_slot_off = nullptr;
};

// element work split into blocks that never straddle two meshes
struct BlockTable {
    bool built = false;
    int threads = 0;
    int32_t n_blocks = 0;
    int32_t *d_begin = nullptr;      // n_blocks, first element
    int32_t *d_end = nullptr;        // n_blocks, one past last
    std::vector<int32_t> mesh_block_off;  // n_mesh + 1 (host)
    int32_t *d_mesh_block_off = nullptr;  // device copy
};

// per-mesh chunks of the gradient used by the FP64 norm reduction
struct ChunkTable {
    bool built = false;
    int32_t n_chunks = 0;
    int32_t *d_begin = nullptr, *d_end = nullptr;   // in scalar entries
    int32_t *d_mesh_chunk_off = nullptr;            // n_mesh + 1
};

// shared-memory tiles of the tiled assembler (tiles.cpp)
struct TileSet {
    bool built = false;
    int64_t build_id = 0;                // distinct for every build (tiles_build)
    int tile_tris = 0;
    int32_t n_tiles = 0;
    // dynamic shared memory of the tiled kernel, [VD == 3][ADM_FP64 = 0 / ADM_FP32 = 1]:
    // accumulators (VD = 3: 13 per footprint vertex + 9 per pair; VD = 2: 7
    // and 5; x, gradient, padded diagonal, pair blocks) padded to 16 bytes,
    // then the tile's metadata blob
    int64_t smem_bytes[2][2] = {{0, 0}, {0, 0}};
    std::vector<int32_t> hdr;            // 8 per tile: tri begin/count, hinge begin/count,
                                         // footprint begin/count, pairs, code begin
    std::vector<uint16_t> tri_loc;       // 6 per triangle (tile order): 3 local ids, 3 pair slots
    std::vector<uint16_t> hinge_loc;     // 10 per hinge (tile order): 4 local ids, 6 pair slots
    std::vector<int32_t> tri_perm, hinge_perm;  // tile order -> canonical element index
    std::vector<int32_t> foot;           // footprint vertex (global id)
    std::vector<int32_t> row_start;      // BSR block of its row start; bit 31: gradient row shared
    std::vector<int32_t> code_off;       // per footprint row + one sentinel per tile
    std::vector<uint16_t> codes;         // per block of every footprint row
    std::vector<int32_t> zero_blocks;    // shared blocks, zeroed before a pass
    std::vector<int32_t> zero_verts;     // shared gradient rows
    std::vector<int32_t> mesh_tile_off;  // n_mesh + 1
    // mass-spring cloth (tiles_build_cloth, triangle tile sets only): every
    // edge and vertex owned by the lowest-indexed tile whose footprint has it
    bool cloth_built = false;
    std::vector<int32_t> cloth_hdr;      // 4 per tile: edge begin/count, vertex begin/count
    std::vector<uint16_t> edge_loc;      // 3 per edge (tile order): 2 local ids, pair slot
    std::vector<uint16_t> vert_loc;      // 1 per vertex (tile order): local id
    std::vector<double> edge_l2;         // squared rest length per edge (tile order)
    std::vector<double> vert_area3;      // a third of the rest area around each vertex (tile order)
    int32_t *d_cloth_hdr = nullptr;
    uint16_t *d_edge_loc = nullptr, *d_vert_loc = nullptr;
    void *d_edge_l2[2] = {nullptr, nullptr};
    void *d_vert_area3[2] = {nullptr, nullptr};
    std::vector<unsigned char> meta;     // per tile: row starts, row code offsets, codes (16-byte padded)
    std::vector<int64_t> meta_off;       // n_tiles + 1 byte offsets into meta
    // device copies
    int32_t *d_hdr = nullptr, *d_foot = nullptr;
    uint16_t *d_tri_loc = nullptr, *d_hinge_loc = nullptr;
    unsigned char *d_meta = nullptr;
    int64_t *d_meta_off = nullptr;
    int32_t *d_zero_blocks = nullptr, *d_zero_verts = nullptr, *d_mesh_tile_off = nullptr;
    int32_t *d_tri_perm = nullptr;               // tile order -> canonical triangle (learned membrane)
    void *d_tri_rest[2] = {nullptr, nullptr};    // rest data permuted to tile order
    void *d_hinge_rest[2] = {nullptr, nullptr};
};

// vertex-pair interaction terms and the block pattern they extend (dyn.cu;
// Sec. 4.3, Sec. 6.3, Alg. 1)
struct Interactions {
    int kind = -1;                  // pattern kind extended, -1: none
    int64_t n_pairs = 0, n_vf = 0;  // vertex-vertex pairs, vertex-face elements
    int64_t cap_pairs = 0, cap_vf = 0, cap_vf_e = 0, cap_cand = 0, cap_slot = 0;  // buffer capacities (elements)
    int32_t *d_cand = nullptr;      // candidate vertex pairs: the pairs, then 6 per vertex-face element
    int32_t *d_slot = nullptr;      // 2 per candidate: blocks (i,j), (j,i); bit 31: block of the mesh pattern
    int32_t *d_quads = nullptr;     // 4 per vertex-face element: p, a, b, c
    double *d_pair_e = nullptr, *d_vf_e = nullptr;  // energy per term of the last pass
    int32_t *d_rp[2] = {nullptr, nullptr}, *d_col[2] = {nullptr, nullptr};  // double-buffered pattern
    int64_t col_cap[2] = {0, 0};
    int active = 0;
    int64_t nnzb = 0;
    int32_t *d_new = nullptr;       // blocks the mesh pattern lacks (zeroed before every Hessian pass)
    int64_t n_new = 0, cap_new = 0;
    int32_t *d_cnt = nullptr, *d_acc = nullptr, *d_bsum = nullptr;  // scratch of the insertion
    int32_t *d_rp_tmp = nullptr, *d_col_tmp = nullptr;              // pattern with repeated new columns
    int64_t cap_col_tmp = 0;
    int32_t *d_diag_off = nullptr;  // position of v's own block in its mesh-pattern row
    int32_t *d_zero_row = nullptr, *d_zero_off = nullptr;  // shared blocks of the tiles as (row, offset)
    int64_t zero_for_build = -1;    // tile build the (row, offset) list belongs to
    int64_t *d_v_off = nullptr;     // mesh vertex offsets
    double kappa = 0.0, dhat = 0.0, area = 0.0, h = 1.0;
    int64_t n_terms() const { return n_pairs + n_vf; }
};

struct EnergyParams {
    double E = 1.0e5, nu = 0.3, t = 1.0e-3, kb = -1.0, h = 1.0;
    // mass-spring cloth: stiffness, time step, areal density, gravity
    double k = 1.0e4, dt = 1.0 / 60.0, rho = 1.0, g[3] = {0.0, 0.0, -9.81};
    double w = 1.0;  // one-ring (umbrella) term weight
    double mu() const { return E / (2.0 * (1.0 + nu)); }
    double lambda() const { return E * nu / (1.0 - nu * nu); }
    double kbend() const { return kb >= 0.0 ? kb : E * t * t * t / (12.0 * (1.0 - nu * nu)); }
};

// a captured evaluation pass and the arguments it was captured with
struct GraphEntry {
    int energy = 0, prec = 0;
    const void *x = nullptr;
    void *grad = nullptr, *bsr = nullptr;
    double *e_total = nullptr, *e_mesh = nullptr, *gnorm = nullptr;
    const void *v = nullptr;
    void *hv = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace adm

struct adm_ctx {
    int device = 0;
    adm::HostMesh m;
    // device copies of connectivity
    int32_t *d_F = nullptr;
    int32_t *d_H = nullptr;
    // rest data per precision, SoA: triangles 5 fields (d00,d01,d10,d11,area),
    // hinges 2 fields (thetabar, abar / 3)
    void *d_tri_rest[2] = {nullptr, nullptr};
    void *d_hinge_rest[2] = {nullptr, nullptr};
    adm::Pattern pat[adm::PAT_COUNT];
    adm::TileSet tiles[adm::PAT_COUNT];
    // ARAP Jacobian column pattern
    int32_t *d_jac_row_ptr = nullptr, *d_jac_col = nullptr;
    // element block tables (keyed by threads per block)
    adm::BlockTable tri_blocks, hinge_blocks, vert_blocks;
    adm::ChunkTable chunks;
    // scratch for reductions
    double *d_epart = nullptr;      // energy partial per element block
    size_t epart_cap = 0;
    double *d_gpart = nullptr;      // sum of squares partial per gradient chunk
    double *d_emesh = nullptr;      // per-mesh energies when only the total is asked for
    double *d_mesh_energy = nullptr;  // n_mesh
    int *d_status = nullptr;
    std::map<int, adm::EnergyParams> params;
    // options
    int assembler = 0;
    void *d_xhat[2] = {nullptr, nullptr};  // mass-spring inertial target, per precision (null: rest shape)
    adm::Interactions inter;
    int proj = 0;            // per-term Hessian filtering on (adm_set_projection)
    double proj_eps = 0.0;   // value negative local eigenvalues are raised to
    int tile_tris = 0;  // 0: automatic (tile_tris_for)
    int block_threads = 128;
    // host-buffer path
    void *d_stage_x = nullptr, *d_stage_grad = nullptr, *d_stage_bsr = nullptr;
    double *d_stage_e = nullptr, *d_stage_gn = nullptr;
    size_t stage_x_bytes = 0, stage_grad_bytes = 0, stage_bsr_bytes = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t copy_stream = nullptr;         // host-to-device copies of the mesh ranges
    std::vector<cudaEvent_t> split_ev;          // one per mesh range: its x has arrived
    std::vector<int32_t> split_mesh;            // first mesh of every range, n_split + 1
    cudaStream_t split_stream[2] = {nullptr, nullptr};  // the ranges' kernels, alternating
    std::vector<cudaEvent_t> split_done;        // one per mesh range: its kernels have run
    cudaEvent_t split_start = nullptr;          // the pass's stream has reached the ranges
    // CUDA graphs of whole passes (ADM_OPT_GRAPH)
    int use_graph = 0;
    std::vector<adm::GraphEntry> graphs;
    cudaStream_t capture_stream = nullptr;
    // learned membrane: network parameters (FP32 master, used BF16-rounded),
    // input / output standardisation, per-triangle table
    float *d_mlp_theta = nullptr, *d_mlp_norm = nullptr, *d_mlp_table = nullptr;
    // autotuned tile size per (energy, precision)
    std::map<std::pair<int, int>, int> tuned;
    // kernel timing ring: per evaluation and stage, a start and an end event
    int prof_ring = 0, prof_next = 0, prof_count = 0;
    std::vector<cudaEvent_t> prof_ev;          // ring * ADM_N_STAGES * 2
    std::vector<unsigned char> prof_ran;       // ring * ADM_N_STAGES
    std::vector<void *> owned;  // every device allocation, freed by destroy
};

namespace adm {

// mesh.cpp
adm_status mesh_validate(const HostMesh &m);
void mesh_rest_triangles(HostMesh &m);
adm_status mesh_build_hinges(HostMesh &m);
void mesh_build_pattern(const HostMesh &m, bool with_hinges, std::vector<int32_t> &row_ptr,
                        std::vector<int32_t> &col);
adm_status mesh_build_rings(HostMesh &m);
void mesh_build_ring_pattern(const HostMesh &m, std::vector<int32_t> &row_ptr, std::vector<int32_t> &col);
void mesh_build_ring_slots(const HostMesh &m, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                           std::vector<int32_t> &slots, std::vector<int32_t> &slot_off);
void mesh_build_slots(const HostMesh &m, const std::vector<int32_t> &row_ptr,
                      const std::vector<int32_t> &col, bool hinges, std::vector<int32_t> &tri_slots,
                      std::vector<int32_t> &hinge_slots);

// tiles.cpp
adm_status tiles_build(const HostMesh &m, const Pattern &P, bool with_hinges, int tile_tris, TileSet &ts);
// per-tile edge and vertex lists of the mass-spring energy, on a triangle tile set
adm_status tiles_build_cloth(const HostMesh &m, TileSet &ts);
// bytes of a tile's metadata blob, and of its dynamic shared memory
int64_t tile_meta_bytes(int64_t nf, int64_t ncodes);
int64_t tile_smem_bytes(int elem_bytes, int64_t units, int64_t nf, int64_t ncodes);

// kernels.cu
struct EvalArgs {
    int energy;          // adm_energy
    int prec;            // adm_precision
    int vdim;
    const void *x;
    void *grad;          // nullable
    void *bsr;           // nullable
    double *energy_total;      // nullable, device
    double *energy_per_mesh;   // nullable, device
    double *gnorm_per_mesh;    // nullable, device
    cudaStream_t stream;
    const void *v = nullptr;   // matrix-free mode: direction (device, like x)
    void *hv = nullptr;        // matrix-free mode: H v (device, like the gradient)
    // host-fed pass: x arrives in n_split mesh ranges (range k = meshes
    // [split_mesh[k], split_mesh[k + 1]), host array), and the kernels of
    // range k wait for split_ready[k]; 0 = x is resident
    int n_split = 0;
    const int32_t *split_mesh = nullptr;
    const cudaEvent_t *split_ready = nullptr;
};
adm_status launch_eval(adm_ctx *h, const EvalArgs &a);
// a device wait that nothing completes, bounded like the tiled kernel's
// (reduce.cu): ADM_ERR_TIMEOUT once it gives up
adm_status bounded_wait_check(cudaStream_t s);
// contact terms (dyn.cu): replace the vertex-vertex pairs and vertex-face
// elements (p, a, b, c) of pattern `kind` and extend its block pattern on the
// GPU; evaluate the terms of a pass (after the tiled kernel) and add their
// energies (after the reduction)
adm_status interactions_set(adm_ctx *h, int kind, const int32_t *pairs, int64_t n, const int32_t *quads, int64_t nq,
                            double kappa, double dhat, double area, double hstep, cudaStream_t s);
adm_status interactions_eval(adm_ctx *h, const EvalArgs &a, int mode);
adm_status interactions_retile(adm_ctx *h, int kind, cudaStream_t s);  // after a tile rebuild
// per-vertex one-ring terms (ring.cu): the whole pass of ADM_UMBRELLA
adm_status eval_ring(adm_ctx *h, const EvalArgs &a);
adm_status interactions_energy(adm_ctx *h, const EvalArgs &a);
// brackets one stage of one evaluation with events when profiling is on
struct StageTimer {
    adm_ctx *h;
    cudaStream_t s;
    int slot;
    StageTimer(adm_ctx *h_, cudaStream_t s_);
    void begin(int stage);
    void end(int stage);
};
// learned membrane (mlp.cu)
adm_status mlp_eval_samples(const float *th, const float *norm, int64_t n, const float *I, float *out,
                            cudaStream_t s);
size_t mlp_workspace_bytes();
adm_status mlp_loss_grad(const float *th, const float *norm, int64_t n, const float *I, const float *psi,
                         const float *g, float beta, double *loss, float *grad, void *ws, size_t ws_bytes,
                         cudaStream_t s);
adm_status mlp_adam(float *th, float *m, float *v, const float *grad, int64_t step, float lr, float b1, float b2,
                    float eps, cudaStream_t s);
adm_status mlp_nh_targets(int64_t n, const float *F, double mu, double lam, float *I, float *psi, float *dpsi,
                          cudaStream_t s);
adm_status mlp_triangle_table(const float *th, const float *norm, int64_t nT, const int32_t *perm,
                              const int32_t *Fv, const float *rest_tiled, const float *x, float *table,
                              cudaStream_t s);

adm_status launch_jacobian(adm_ctx *h, int prec, const void *x, void *r, void *jv, void *jtj,
                           cudaStream_t stream);

}  // namespace adm
