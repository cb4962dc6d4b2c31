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

// passive, gradient, full Hessian, matrix-free Hessian-vector product
enum Mode { MODE_VALUE = 0, MODE_GRAD = 1, MODE_HESS = 2, MODE_HVP = 3 };

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

// Tiles of the staged-gather assembler (tiles.cpp).
//
// A unit is one triangle plus the mesh edges attached to it (every edge is
// attached to exactly one of its faces): on a shell each attached interior
// edge carries its hinge, on the cloth each attached edge its spring.  The
// attached edges sit in slots s = 0, 1, 2, the edge (t_k, t_k+1) of
// k = (rot + s) mod 3 for a per-unit rotation rot that makes the slots
// consecutive; the hinge of slot s is evaluated in the order (t_k, t_k+1,
// t_k+2, extra), the same hinge (Sec. 7.7) relabelled.  The triangle keeps
// its own vertex order.
//
// A tile is a run of units in Morton order (per mesh).  Every unit writes its
// contributions as "chunks": per unit vertex t_i a vertex chunk (gradient,
// diagonal block upper entries or H v) and per vertex pair a pair chunk (the
// off-diagonal block, oriented from the lower to the higher footprint index);
// an attached hinge adds a vertex chunk and three pair chunks for its extra
// vertex, and adds its other contributions into the unit's own chunks.  The
// chunks of a tile are laid out sorted by target (vertex, then unit order;
// pair, then unit order), so every output entry is the fixed-order sum of one
// contiguous segment: the gather that writes the BSR rows is deterministic
// and needs no atomics.  An output that several tiles produce (a "shared" row
// or block) is stored by the lowest-index of them; each other one stores its
// part in a partial slot of its own, and a fix-up pass adds the slots to the
// output in tile order: no tile ever waits for another.
struct TileSet {
    bool built = false;
    int64_t build_id = 0;                // distinct for every build (tiles_build)
    int tile_units = 0;                  // units per tile at most
    int32_t n_tiles = 0;
    int64_t n_slots = 0, n_vterms = 0;   // attached edges, cloth vertex terms
    // per tile, kHdr int32 (see kHdr* below)
    std::vector<int32_t> hdr;
    // per unit (tile order), 8 uint16: footprint ids of t0 t1 t2; the extra
    // vertex of the hinge in slots 0..2 (0xffff: none; on a cloth tile set the
    // first field is the unit's first vertex term within the tile); flags
    // (number of slots | cloth vertex-term mask << 2 | rot << 5); first slot
    // (within the tile)
    std::vector<uint16_t> unit;
    std::vector<uint16_t> unit_dst;      // per unit 6: chunks of V0 V1 V2 (vertex), P01 P02 P12 (pair)
    std::vector<uint16_t> slot_dst;      // per slot 4: chunks of X (vertex), PX(h0) PX(h1) PX(h2) (pair)
    std::vector<int32_t> tri_perm;       // unit -> canonical triangle
    std::vector<int32_t> tri_verts;      // unit -> its vertices (global ids), 3 per unit
    std::vector<double> tri_rest;        // 5 per unit (Dm^-1 row-major, area)
    std::vector<int32_t> slot_edge;      // slot -> (hinge index) or -1; per slot
    std::vector<int32_t> slot_verts;     // 4 per slot, global ids in evaluation order: t_k, t_k+1, t_k+2,
                                         // the hinge's extra vertex (-1: none)
    std::vector<double> slot_rest;       // 2 per slot: hinge (thetabar, abar/3) or spring (l^2, 0)
    std::vector<double> vterm_rest;      // per cloth vertex term: a third of the rest area around it
    std::vector<int32_t> foot;           // footprint vertices (global ids), sorted, per tile
    std::vector<int32_t> mesh_tile_off;  // n_mesh + 1
    // per tile metadata blob (copied into shared memory): kRowWords int32
    // per footprint row, one code per pair block produced, and the tile's
    // partial slots (global slot indices)
    std::vector<unsigned char> meta;
    std::vector<int64_t> meta_off;       // n_tiles + 1
    std::vector<int32_t> zero_verts;     // vertices no unit touches (zero row and diagonal block)
    std::vector<int32_t> zero_blocks;    // their diagonal blocks
    int64_t max_nvc = 0, max_npc = 0, max_nf = 0, max_meta = 0, max_part = 0;  // largest counts over the tiles
    // fix-up lists of the outputs several tiles produce, 4 int32 per output:
    // row vertex, position of the block in its BSR row (the diagonal block
    // for a vertex output), number of partial slots, first slot.  Vertex
    // outputs (gradient row, diagonal block, H v row) sorted by vertex, pair
    // blocks by block index; slots are allocated in the same order
    std::vector<int32_t> fix_v, fix_p;
    int64_t n_vpart = 0, n_ppart = 0;    // partial slots: vertex (Chunk<MODE_HESS> floats each), pair (VD^2)
    int32_t *d_fix_v = nullptr, *d_fix_p = nullptr;
    void *d_vpart = nullptr, *d_ppart = nullptr;  // partial slots, sized for FP64
    int64_t smem_cache[4][2][2] = {};    // tile_smem_bytes by (mode, VD == 3, FP64), 0: not yet computed
    int32_t *d_hdr = nullptr, *d_foot = nullptr, *d_tri_perm = nullptr, *d_tri_verts = nullptr;
    int32_t *d_slot_verts = nullptr;
    // filtered passes: each term's filtered edge-coordinate result (energy,
    // gradient, packed Hessian), structure of arrays over units and slots,
    // sized for FP64 on first use
    void *d_loc_tri = nullptr, *d_loc_slot = nullptr;
    uint16_t *d_unit = nullptr, *d_unit_dst = nullptr, *d_slot_dst = nullptr;
    unsigned char *d_meta = nullptr;
    int64_t *d_meta_off = nullptr;
    int32_t *d_zero_verts = nullptr, *d_zero_blocks = nullptr, *d_mesh_tile_off = nullptr;
    int32_t *d_sync = nullptr;           // 8 work-queue positions
    void *d_tri_rest[2] = {nullptr, nullptr};  // per precision, SoA 5 x units
    void *d_slot_rest[2] = {nullptr, nullptr}; // per precision, SoA 2 x slots
    void *d_vterm_rest[2] = {nullptr, nullptr};
    bool cloth_built = false;
};
// tile header words
enum TileHdr {
    kHdrUnit = 0, kHdrNUnit, kHdrSlot, kHdrNSlot, kHdrFoot, kHdrNF, kHdrNVC, kHdrNPC, kHdrNCode, kHdrNPart,
    kHdrCodeOff, kHdrPartOff, kHdrVTerm, kHdrNVTerm, kHdr = 16
};
// An output several tiles produce is stored by the lowest-index one; each
// other one writes its part to a partial slot (through the tile's table of
// slots) that the fix-up pass adds in tile order.
// footprint row words: [0] BSR start of the row, [1] number of vertex
// chunks << 24, [2] first vertex chunk, [3] position of the diagonal block in
// the BSR row (15 bits) | partial << 15 | table index << 16 (partial rows).
// pair code (one per pair segment of the tile, 2 words): x = chunk start (13
// bits) | chunk count << 13 (4 bits) | partial A << 17 | partial B << 18 |
// row A << 19 (9 bits); y = position A (9 bits) | row B << 9 | position B
// << 18.  Block A is (lo, hi) in footprint row lo, block B the transpose
// (hi, lo) in row hi; for a partial block, row << 9 | position is its index
// in the tile's slot table.
constexpr int kRowWords = 4;
// footprint rows of one tile at most (the row fields of the pair codes are 9 bits)
constexpr int kMaxFootRows = 512;

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
    int mlp_net = 1;         // network kernel of the learned membrane: 0 mma.sync, 1 tcgen05 (default)
    int tile_threads = 256;  // threads per block of the FP32 tiled kernel (128 or 256)
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

// whether contact terms extend pattern `kind`, and the BSR row pointer
// (device) a pass on it writes through
inline bool pattern_extended(const adm_ctx *h, int kind)
{
    return h->inter.kind == kind && h->inter.d_rp[h->inter.active] != nullptr;
}
inline const int32_t *active_row_ptr(const adm_ctx *h, int kind)
{
    return pattern_extended(h, kind) ? h->inter.d_rp[h->inter.active] : h->pat[kind].d_row_ptr;
}

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
adm_status tiles_build(const HostMesh &m, const Pattern &P, bool with_hinges, int tile_units, TileSet &ts);
// cloth data (spring rest lengths, vertex terms) on a triangle tile set
adm_status tiles_build_cloth(const HostMesh &m, TileSet &ts);
// floats of one chunk: vertex and pair chunks per mode and vertex dimension
#if defined(__CUDACC__)
#define ADM_TILE_HD __host__ __device__ __forceinline__
#else
#define ADM_TILE_HD inline
#endif
ADM_TILE_HD constexpr int chunk_floats(int mode, int vd, bool pair)
{
    return mode == MODE_GRAD ? (pair ? 0 : vd)
           : mode == MODE_HESS ? (pair ? vd * vd : vd + vd * (vd + 1) / 2)
           : mode == MODE_HVP  ? (pair ? 0 : 2 * vd)
                               : 0;
}
// one tile's dynamic shared memory (byte offsets): x of the footprint, v
// (matrix-free mode), vertex chunks, pair chunks, the metadata blob.  The x
// and v regions are sized by nf_cap, the largest footprint of the tile set,
// so that every tile places its chunks after them: the kernel stages the
// next tile's x while the current tile's chunks are still being summed.
struct TileLayout {
    int32_t off_vs, off_sv, off_sp, off_blob, total;
};
ADM_TILE_HD TileLayout tile_layout(int nf_cap, int nvc, int npc, int meta_bytes, int mode, int vd, int eb)
{
    auto a16 = [](int b) { return (b + 15) & ~15; };
    TileLayout L;
    const int xs = nf_cap * vd * eb;
    L.off_vs = a16(xs);
    L.off_sv = a16(L.off_vs + (mode == MODE_HVP ? xs : 0));
    L.off_sp = a16(L.off_sv + nvc * chunk_floats(mode, vd, false) * eb);
    L.off_blob = a16(L.off_sp + npc * chunk_floats(mode, vd, true) * eb);
    L.total = L.off_blob + (mode >= MODE_GRAD ? meta_bytes : 0);
    return L;
}
// tcgen05 operands of the learned membrane's network: the byte offset of
// element (row, k) of a K-major BF16 operand in the canonical layout without
// swizzle (8-row x 16-byte core matrices, row groups 128 bytes apart -- the
// shared-memory descriptor's stride byte offset -- and 8-element K chunks
// lbo bytes apart, its leading byte offset), and the instruction descriptor
// of tcgen05.mma kind::f16 for BF16 A and B, FP32 D, both K-major, an M x N
// tile: D format bits 4-5, A and B formats bits 7-9 and 10-12, N / 8 from
// bit 17, M / 16 from bit 24
ADM_TILE_HD constexpr uint32_t umma_canon(int row, int k, uint32_t lbo)
{
    return (uint32_t)(row >> 3) * 128u + (uint32_t)(k >> 3) * lbo + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}
ADM_TILE_HD constexpr uint32_t umma_idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// dynamic shared memory of the tiled kernel for a tile set, mode and
// precision: the largest tile's layout
int64_t tile_smem_bytes(const TileSet &ts, int mode, int vd, int elem_bytes);

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
// per-triangle table of the learned membrane in unit order: verts = the
// units' rotated vertices (3 per unit), rest_tiled = their rest data (SoA)
adm_status mlp_triangle_table(const float *th, const float *norm, int64_t nT, const int32_t *verts,
                              const float *rest_tiled, const float *x, float *table, int tc_net, int *status,
                              cudaStream_t s);

adm_status launch_jacobian(adm_ctx *h, int prec, const void *x, void *r, void *jv, void *jtj,
                           cudaStream_t stream);

}  // namespace adm
