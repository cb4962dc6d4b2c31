/*
 * adm.h -- C ABI of libadm: per-element forward-mode differentiation of
 * energy terms on triangle meshes and assembly of the global gradient,
 * block-sparse Hessian and sparse Jacobian, on one NVIDIA GB300 (sm_103a).
 *
 * The calls follow the problem statement of "Locality-Aware Automatic
 * Differentiation on the GPU for Mesh-Based Computations" (Sec. 4.1):
 *   F(x) = sum_j f_j(S_j x)                (Eq. 1)
 *   g = sum_j S_j^T grad f_j,  H = sum_j S_j^T Hess f_j S_j   (Eq. 2)
 *   J = sum_j P_j^T J_j S_j                (Eq. 3)
 * with the block pattern of H (and the column pattern of J) fixed from the
 * mesh connectivity at creation time (Sec. 6.1) and every local derivative
 * computed by forward-mode AD in registers (Sec. 5.1, Sec. 6.2).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - No exception crosses the ABI; every call returns an adm_status.
 *  - Argument and mesh errors are detected on the host and returned
 *    synchronously.  Errors found by the kernels (a folded triangle, a
 *    degenerate hinge, a non-finite value) are latched in a device status
 *    word and read with adm_get_status() after the caller has synchronised
 *    the stream; the offending element contributes nothing.
 *  - Evaluation calls are stream-ordered and asynchronous: they enqueue work
 *    on the CUDA stream passed as `stream` (a cudaStream_t; NULL is the
 *    legacy default stream) and return without waiting.
 *  - Ownership: the caller owns every buffer it passes (x, outputs); the
 *    library owns the handle, the pattern arrays it returns, its rest data,
 *    slot maps and work tables.  Pattern pointers stay valid until
 *    adm_destroy().  Evaluation calls allocate no memory except where
 *    stated (the first call of a CUDA graph, the host-buffer call).
 *  - The first evaluation of an energy on a handle builds its tiles and
 *    pattern on the host (synchronous, allocates); make it before capturing
 *    a stream into a CUDA graph.
 *  - Outputs are fully overwritten (no accumulate-into contract).
 *  - Layouts: x and the gradient are vertex-major, x[v * var_dim + d];
 *    BSR values are nnzb blocks of var_dim x var_dim, row-major inside a
 *    block, in the order of the pattern's col array; the pattern stores both
 *    (i, j) and (j, i) (full symmetric storage, as the CSR of Sec. 6.1), and
 *    columns ascend inside every block row.
 *  - Precision: ADM_FP64 buffers are double, ADM_FP32 buffers are float;
 *    energies and gradient norms are always double.
 */
#ifndef ADM_H
#define ADM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adm_ctx *adm_handle; /* opaque, library-owned */

typedef enum {
    ADM_OK = 0,
    ADM_ERR_ARG = -1,         /* bad argument (null pointer, size, enum)        */
    ADM_ERR_MESH = -2,        /* bad mesh: index out of range, degenerate rest
                                 triangle, edge with > 2 faces or inconsistent
                                 orientation where a hinge term needs it       */
    ADM_ERR_DOMAIN = -3,      /* a kernel met an element outside the energy's
                                 domain (folded triangle, degenerate hinge)     */
    ADM_ERR_CUDA = -4,        /* a CUDA runtime call failed                     */
    ADM_ERR_TIMEOUT = -5,     /* a bounded device wait ran out                  */
    ADM_ERR_OOM = -6,         /* device allocation failed                       */
    ADM_ERR_UNSUPPORTED = -7  /* energy / precision / var_dim combination that
                                 this build does not provide                    */
} adm_status;

/* Energy terms.  Stencils: triangle (3 vertices) or hinge = interior edge plus
 * its two opposite vertices (4 vertices, Sec. 7.7). */
typedef enum {
    ADM_SYMDIR2D = 1,         /* area_t (|J|_F^2 + |J^-1|_F^2), UV map, var_dim 2 (Sec. 7.2) */
    ADM_STVK_MEMBRANE = 2,    /* t A (mu |E|^2 + lambda/2 tr(E)^2), var_dim 3       */
    ADM_HINGE_BENDING = 3,    /* k_b (A/3) (theta - theta')^2 h^2, var_dim 3 (Sec. 7.7) */
    ADM_SHELL = 4,            /* ADM_STVK_MEMBRANE + ADM_HINGE_BENDING              */
    ADM_NH_MEMBRANE = 5,      /* Neo-Hookean on the invariants of C (Sec. 7.7)      */
    ADM_MLP_MEMBRANE = 6,     /* learned Neo-Hookean surrogate (adm_mlp_* calls)    */
    ADM_AREA = 7,             /* 1/2 |(x_j - x_i) x (x_k - x_i)| (Sec. 7.6)         */
    ADM_UMBRELLA = 9,         /* per-vertex one-ring term: w/2 |x_v - mean of the
                                 one-ring neighbours of v|^2 (uniform Laplacian
                                 smoothing); block pattern = two-ring of every
                                 vertex; valence <= 12; var_dim 2 or 3       */
    ADM_MASS_SPRING = 8,      /* implicit-Euler cloth (Sec. 7.1): per-vertex
                                 m_v/2 |x_v - xhat_v|^2 - h^2 m_v g.x_v and
                                 per-edge springs h^2 l^2 k/2 (|x_i - x_j|^2 / l^2
                                 - 1)^2; lumped m_v = rho * a third of the rest
                                 area around v; var_dim 3; tiled kernel only  */
    ADM_ARAP2D_RESIDUAL = 16  /* 4 residuals sqrt(A) vec(J - R(J)) per triangle,
                                 var_dim 2 (vector-valued term, Eq. 3)              */
} adm_energy;

typedef enum { ADM_FP64 = 0, ADM_FP32 = 1 } adm_precision;

/* Options for adm_set_option(). */
typedef enum {
    ADM_OPT_ASSEMBLER = 1,    /* 0 = tiled (default): shared-memory tiles,
                                 every contribution staged and each output
                                 summed in a fixed order, no float atomics,
                                 so two passes on the same input give
                                 bit-identical gradients, Hessians and H v;
                                 1 = per-element atomic scatter (the paper's
                                 Sec. 5.5 scheme, kept as a reference path;
                                 its sums depend on thread timing)           */
    ADM_OPT_TILE_TRIS = 2,    /* units (triangles with their attached hinges or
                                 springs) per tile of the tiled assembler,
                                 1..4096; 0 (default): 192, lowered for small
                                 meshes to about nT / 304 (two tiles per SM),
                                 never below 32; tiles are split further until
                                 their shared memory fits */
    ADM_OPT_BLOCK_THREADS = 3,/* threads per block of the element kernels       */
    ADM_OPT_PROFILE = 4,      /* > 0: record CUDA events around every kernel of
                                 each evaluation, on the evaluation's stream,
                                 keeping the last `value` evaluations (a ring);
                                 0: off (default).  Creates events, allocates no
                                 device memory. */
    ADM_OPT_TILE_THREADS = 6, /* threads per block of the tiled kernel in FP32
                                 without filtering: 128 or 256 (0, default:
                                 256); FP64 and filtered passes use 256 */
    ADM_OPT_GRAPH = 5,        /* 1: adm_eval / adm_eval_batch capture their
                                 whole pass (zero-fill, element kernel,
                                 reductions) into a CUDA graph on the first call
                                 with a given (energy, precision, buffers) tuple
                                 and replay it on later calls with the same
                                 tuple (up to 8 tuples are kept); 0: direct
                                 launches (default).  Capture happens on a
                                 library stream, the replay on the caller's
                                 stream.  Changing parameters or options drops
                                 the captured graphs. */
    ADM_OPT_MLP_NET = 7       /* network kernel of the learned membrane
                                 (ADM_MLP_MEMBRANE passes): 1 (default) =
                                 fifth-generation tensor cores (tcgen05.mma,
                                 FP32 accumulators in tensor memory), 128
                                 triangles per MMA tile; 0 = warp-level BF16
                                 tensor-core MMA (mma.sync), one warp per 8
                                 triangles.
                                 Both round weights and activations to BF16
                                 and accumulate in FP32; their outputs differ
                                 by the summation order only. */
} adm_option;

/* Kernel stages reported by adm_profile_read(). */
typedef enum {
    ADM_STAGE_ZERO = 0,       /* zero-fill of outputs (memset)                  */
    ADM_STAGE_TRIANGLES = 1,  /* triangle-term kernel                           */
    ADM_STAGE_HINGES = 2,     /* hinge-term kernel                              */
    ADM_STAGE_GNORM = 3,      /* FP64 gradient-norm partials                    */
    ADM_STAGE_FINALIZE = 4,   /* per-mesh FP64 energy / norm reduction          */
    ADM_STAGE_TILED = 5,      /* fused tiled element + assembly kernel          */
    ADM_STAGE_GRAPH = 6,      /* a whole captured pass replayed (ADM_OPT_GRAPH) */
    ADM_STAGE_MLP = 7,        /* per-triangle network table (learned membrane)  */
    ADM_STAGE_PAIRS = 8,      /* interaction terms over vertex pairs            */
    ADM_N_STAGES = 9
} adm_stage;

/* --- creation ---------------------------------------------------------- */

/* One mesh.  V: nV x 3 rest positions (host, double); F: nF x 3 vertex
 * indices (host, int32, counter-clockwise); var_dim: 3 for positions, 2 for
 * a UV map.  Builds edges, hinges (canonical order: e0 < e1, face A holds
 * e0->e1), rest data, the block patterns and the work tables, and uploads
 * them to the current device.  Synchronous.  Errors: ADM_ERR_ARG,
 * ADM_ERR_MESH, ADM_ERR_OOM, ADM_ERR_CUDA.  On error *out is NULL. */
adm_status adm_create(const double *V, int64_t nV, const int32_t *F, int64_t nF,
                      int32_t var_dim, adm_handle *out);

/* A batch of n_mesh independent meshes concatenated: mesh m owns vertices
 * [v_off[m], v_off[m+1]) and faces [f_off[m], f_off[m+1]); F holds global
 * (batch-wide) vertex indices.  v_off, f_off: n_mesh + 1 entries (host). */
adm_status adm_create_batch(const double *V, const int64_t *v_off, const int32_t *F,
                            const int64_t *f_off, int32_t n_mesh, int32_t var_dim,
                            adm_handle *out);

/* Interaction terms (Sec. 4.3) with the dynamic block pattern they induce
 * (Sec. 6.3, Alg. 1).  Replaces the interaction set of the pattern `energy`
 * uses (membranes and ADM_MASS_SPRING: the triangle pattern; ADM_SHELL and
 * ADM_HINGE_BENDING: the shell pattern; one pattern per handle) with
 *   - n_pairs vertex-vertex terms: pairs, 2 * n_pairs int32 (i, j);
 *   - n_vf vertex-face terms: vf, 4 * n_vf int32 (p, a, b, c), vertex p
 *     against the triangle (a, b, c);
 * (host or device, copied; both counts 0 clear the set).  Every later
 * evaluation of an energy on that pattern adds, per term, the contact
 * barrier of Sec. 7.7, kappa/2 dhat area (s - 1) ln(s) h^2 with s = d / dhat
 * for s < 1 (var_dim 3): d = |x_i - x_j| for a pair, the distance from x_p to
 * the triangle for a vertex-face term (its square written for the corner,
 * edge or interior of the triangle nearest to x_p, decided in the precision
 * of the pass).  A term listed twice counts twice.
 *
 * The block pattern is extended on the GPU: every row keeps its mesh
 * columns, in their order, followed by the columns of the new blocks of the
 * terms (each pair of a term's vertices), ascending and each once; blocks
 * the mesh pattern has add nothing.  adm_pattern then returns the extended
 * pattern (device pointers valid until the next call of this function),
 * whose nnzb sizes the Hessian buffers.  Synchronous on `stream` (reads back
 * the new block count); no pass of this handle may be in flight on another
 * stream meanwhile (the term buffers are rewritten).  Term energies count towards the total and towards
 * the mesh of the term's first vertex (in per-mesh energies their order of
 * summation is not fixed).  The Hessian and matrix-free passes run on the
 * tiled kernel.  Errors: ADM_ERR_ARG (a vertex out of range or repeated
 * within a term, dhat <= 0, a pattern past 2^31 blocks; the set is then
 * cleared), ADM_ERR_UNSUPPORTED (var_dim != 3, a second pattern kind). */
adm_status adm_set_contacts(adm_handle h, adm_energy energy, const int32_t *pairs, int64_t n_pairs,
                            const int32_t *vf, int64_t n_vf, double kappa, double dhat, double area,
                            double h_step, void *stream);

/* adm_set_contacts with vertex-vertex pairs only. */
adm_status adm_set_interactions(adm_handle h, adm_energy energy, const int32_t *pairs, int64_t n_pairs,
                                double kappa, double dhat, double area, double h_step, void *stream);

/* Inertial target xhat of ADM_MASS_SPRING (x^n + h v^n of the time step;
 * host, n_rows * 3 doubles, copied into library memory in both precisions).
 * Until it is set the target is the rest shape.  Errors: ADM_ERR_ARG
 * (NULL, non-finite entries), ADM_ERR_UNSUPPORTED (var_dim != 3). */
adm_status adm_set_inertia_target(adm_handle h, const double *xhat_host);

/* Material parameters of an energy (host array, copied).  Membranes
 * (ADM_STVK_MEMBRANE, ADM_NH_MEMBRANE, ADM_MLP_MEMBRANE): {E, nu, thickness};
 * ADM_HINGE_BENDING: {k_b, h}; ADM_SHELL: {E, nu, thickness, k_b, h};
 * ADM_UMBRELLA: {w};
 * ADM_MASS_SPRING: {k, h, rho, g_x, g_y, g_z} (spring stiffness, time step,
 * areal density, gravity; defaults 1e4, 1/60, 1, (0, 0, -9.81)).
 * Missing trailing values keep their defaults E = 1e5, nu = 0.3,
 * thickness = 1e-3, h = 1, k_b = E t^3 / (12 (1 - nu^2)).  Lame parameters
 * are the plane-stress ones, mu = E / (2 (1 + nu)), lambda = E nu / (1 - nu^2). */
adm_status adm_set_params(adm_handle h, adm_energy energy, const double *p, int32_t np);

adm_status adm_set_option(adm_handle h, adm_option option, int64_t value);

/* --- patterns ------------------------------------------------------------ */

/* Block-sparse (BSR) pattern of the Hessian of `energy`: *block = var_dim,
 * *n_rows = number of vertices, *nnzb = number of blocks, and device
 * pointers to row_ptr (n_rows + 1, int32) and col (nnzb, int32).  Builds the
 * pattern on first use (synchronous, allocates).  Any output may be NULL. */
adm_status adm_pattern(adm_handle h, adm_energy energy, int32_t *block, int64_t *n_rows,
                       int64_t *nnzb, const int32_t **row_ptr_dev, const int32_t **col_dev);

/* CSR pattern of the residual Jacobian of a vector-valued energy
 * (ADM_ARAP2D_RESIDUAL): rows 4t + r (triangle t, residual r), columns
 * v * 2 + d sorted ascending, 6 per row.  Device pointers; any output may
 * be NULL. */
adm_status adm_jac_pattern(adm_handle h, adm_energy energy, int64_t *n_rows, int64_t *n_cols,
                           int64_t *nnz, const int32_t **row_ptr_dev, const int32_t **col_dev);

/* Canonical hinge list (device, nH x 4 int32: e0, e1, a, b) and the slot map
 * of `energy`: for every element in canonical order (triangles in input
 * order, then hinges) and every ordered local vertex pair (a, b), the index
 * of block (v_a, v_b) in the BSR pattern (device int32, n_elem x nv x nv). */
adm_status adm_hinges(adm_handle h, const int32_t **hinges_dev, int64_t *n_hinges);
/* (ADM_ERR_UNSUPPORTED for ADM_UMBRELLA and ADM_MASS_SPRING, which have no
 * per-triangle or per-hinge elements.) */
adm_status adm_slot_map(adm_handle h, adm_energy energy, const int32_t **slots_dev,
                        int64_t *n_entries);

/* --- evaluation -------------------------------------------------------- */

/* Energy, gradient and Hessian of one energy at x (device, n_rows * var_dim
 * of the precision's type).  energy_dev: device double, receives F(x)
 * summed over every mesh of the handle (nullable); grad_dev: device,
 * n_rows * var_dim (nullable); bsr_vals_dev: device, nnzb * var_dim^2
 * (nullable).  With both grad_dev and bsr_vals_dev NULL the call runs the
 * passive (value-only) mode; with bsr_vals_dev NULL the gradient-only mode.
 * Errors: ADM_ERR_ARG, ADM_ERR_UNSUPPORTED, ADM_ERR_CUDA (launch). */
adm_status adm_eval(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev,
                    double *energy_dev, void *grad_dev, void *bsr_vals_dev, void *stream);

/* Hessian filtering (Sec. 7.1, after Teran et al. 2005): with enable = 1,
 * every element term's local Hessian has its negative eigenvalues set to eps
 * (>= 0, finite) before assembly, in adm_eval, adm_eval_batch(_host) and
 * adm_eval_hvp; energies and gradients are unchanged.  For the shell the
 * membrane triangle and the hinge are separate terms.  The filtered passes
 * run on the tiled kernel whatever ADM_OPT_ASSEMBLER says.  Clamping acts on
 * the spectrum of the term as a function of its vertex positions; the three
 * translations, exact zeros of every term here, are left alone.  Errors:
 * ADM_ERR_ARG.  Drops captured graphs when the setting changes.  The first
 * filtered Hessian or H v pass allocates, per tile set, a buffer of every
 * term's filtered result (28 doubles per triangle, 55 per attached edge;
 * 3.8 GB for 4.3M triangles): ADM_ERR_OOM if that fails. */
adm_status adm_set_projection(adm_handle h, int32_t enable, double eps);

/* Matrix-free Hessian-vector product (the paper's matrix-free mode,
 * Sec. 5.5 and Sec. 6.2, which its Newton-CG parameterisation of Sec. 7.2
 * calls once per CG iteration): hv = H(x) v = sum_j S_j^T H_j S_j v, each
 * element's local Hessian applied to its gathered part of v and the products
 * accumulated, without forming the global Hessian.  The same pass gives the
 * energy and, optionally, the gradient.
 *   x_dev, v_dev: device, n_rows * var_dim of the precision's type (v is the
 *                 direction, vertex-major like x);
 *   energy_dev:   device double, F(x) over every mesh (nullable);
 *   grad_dev:     device, n_rows * var_dim (nullable);
 *   hv_dev:       device, n_rows * var_dim, fully overwritten.
 * All buffers are owned by the caller.  Runs on the tiled kernel whatever
 * ADM_OPT_ASSEMBLER says (building its tiles on first use); takes part in
 * ADM_OPT_GRAPH like adm_eval.  Errors: ADM_ERR_ARG (NULL x, v or hv, bad
 * precision), ADM_ERR_UNSUPPORTED (residual energies; the learned membrane
 * without attached weights or in FP64), ADM_ERR_CUDA. */
adm_status adm_eval_hvp(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev,
                        const void *v_dev, double *energy_dev, void *grad_dev, void *hv_dev, void *stream);

/* Batched form: per-mesh energies (device, n_mesh doubles, nullable) and
 * per-mesh gradient 2-norms in FP64 (device, n_mesh doubles, nullable),
 * plus the batch gradient and Hessian as in adm_eval. */
adm_status adm_eval_batch(adm_handle h, adm_energy energy, adm_precision prec,
                          const void *x_dev, double *energy_per_mesh_dev, double *gnorm_dev,
                          void *grad_dev, void *bsr_vals_dev, void *stream);

/* The full derivative pass of adm_eval_batch (energy, gradient, Hessian)
 * with HOST buffers: copies x host->device, evaluates into library-owned
 * device staging buffers, copies back those outputs whose host pointer is
 * not NULL, and returns after the copies completed (synchronous).  Outputs
 * not copied back stay in the staging buffers (for a solver on the device).
 * Staging buffers are allocated on first use (and grown when contact terms
 * extend the pattern); the call uses the library's own stream.  bsr_vals_host
 * holds the nnzb of adm_pattern at the time of the call.  Pinned host
 * buffers make the copies faster. */
adm_status adm_eval_batch_host(adm_handle h, adm_energy energy, adm_precision prec,
                               const void *x_host, double *energy_per_mesh_host,
                               double *gnorm_host, void *grad_host, void *bsr_vals_host);

/* Autotuner of the tiled assembler (the batched evaluation's work split):
 * times the full pass of `energy` at `prec` on x (device) for each candidate
 * pair (threads per block, units per tile) -- 256 threads with {96, 128, 160,
 * 192, 224} units, and in FP32 128 threads (four blocks per SM at 128
 * registers) with {48, 64, 96, 112} units -- keeps the fastest pair for this
 * handle (as ADM_OPT_TILE_THREADS and ADM_OPT_TILE_TRIS) and returns it and
 * its time per pass in ms (any output may be NULL).  Synchronous; allocates
 * temporary output buffers and rebuilds the tiles for every tile size (host
 * work of seconds on a 2M-vertex batch).  Not part of the paper (Sec. 7 uses
 * a fixed patch size of 512 faces). */
adm_status adm_autotune(adm_handle h, adm_energy energy, adm_precision prec, const void *x_dev,
                        int32_t *best_tile_tris, int32_t *best_threads, float *best_ms);

/* Residual r (device, 4 nT), CSR Jacobian values (device, 24 nT, in the
 * order of adm_jac_pattern) and the Gauss-Newton matrix J^T J assembled into
 * the 2 x 2 BSR pattern of the triangle stencil (device, nullable). */
adm_status adm_eval_jacobian(adm_handle h, adm_energy energy, adm_precision prec,
                             const void *x_dev, void *r_dev, void *jac_vals_dev,
                             void *jtj_bsr_vals_dev, void *stream);

/* Average device time (ms) per launch of every stage over the evaluations
 * recorded since profiling was enabled or last read (at most the ring size),
 * and the number of launches of each stage (n_launches may be NULL).  Waits
 * for the recorded events, then clears the ring.  n_stages <= ADM_N_STAGES.
 * ADM_ERR_ARG when profiling is off. */
adm_status adm_profile_read(adm_handle h, float *avg_ms, int32_t *n_launches, int32_t n_stages);

/* FP64 2-norm ||v||_2 of a device vector of n entries (float for ADM_FP32,
 * double for ADM_FP64), written to *norm_dev (device double), enqueued on
 * `stream`.  This is the gradient-norm reduction of adm_eval_batch as a call
 * that allocates nothing and needs no handle; the paper has no counterpart.
 * It is meant for callers that cannot call cudaMalloc where they need the
 * norm: real-time loops whose device memory is fixed in advance (an
 * allocation there can stall or fail mid-loop), plug-ins inside a host
 * framework that owns the device's memory budget, and hosts that route
 * every device allocation through their own pool.
 *  - Scratch: a static device array of 4096 FP64 partial sums (32 KiB) that
 *    every GPU loading the library holds until the process exits; n may be at
 *    most 4096 * 8192 = 33,554,432 entries, larger n returns ADM_ERR_ARG and
 *    launches nothing.
 *  - The first call on a device, with that device current, resolves the
 *    array's device address (cudaGetSymbolAddress) and keeps it for that
 *    device; make that first call before any stream capture.  The kept
 *    address belongs to the device's primary context: do not use this call
 *    after a cudaDeviceReset of that device, nor from another context on it.
 *  - All calls share the one array and it keeps the last call's partials:
 *    calls whose work overlaps on the GPU (different streams, no ordering)
 *    race on it.  Calls ordered on one stream are safe; nothing needs
 *    clearing between them.
 *  - No cudaMalloc, cudaFree or allocating library routine is called. */
adm_status adm_grad_norm_noalloc(const void *v_dev, int64_t n, adm_precision prec, double *norm_dev,
                                 void *stream);

/* Failure-detection check of the device waits.  Every wait in this
 * library's kernels is bounded: the tiled kernel waits for the bulk copy of
 * a tile's metadata for about a second at most, then latches ADM_ERR_TIMEOUT
 * in the status word and skips its write-out, leaving the context usable.
 * This call runs that same bounded wait, in one thread, on a shared-memory
 * barrier that nothing completes, and returns ADM_ERR_TIMEOUT when the wait
 * gave up as it must (about a second; synchronous on `stream`).  Any other
 * result is ADM_ERR_CUDA.  The handle-free call touches no caller memory. */
adm_status adm_check_bounded_wait(void *stream);

/* --- learned membrane energy ------------------------------------------- */
/* A per-triangle MLP surrogate of the Neo-Hookean membrane density on the
 * invariants (I1, I2, I3) of C3 = diag(F^T F, 1): u = (I - m_I)/s_I,
 * a1 = silu(W1 u + b1), a2 = silu(W2 a1 + b2), y = w3.a2 + b3,
 * psi = s_psi y + m_psi, hidden width 64.  Not in the paper (it stands in for
 * an analytic density of Sec. 7.7).  theta: ADM_MLP_NPARAM floats in the order
 * W1 (64x3 row-major), b1 (64), W2 (64x64 row-major, row = output unit), b2
 * (64), w3 (64), b3; the kernels use them rounded to BF16, contract on the
 * tensor cores with FP32 accumulation.  norm: 8 floats
 * {m_I1, m_I2, m_I3, s_I1, s_I2, s_I3, m_psi, s_psi}.  All pointers are
 * device pointers; all calls are stream-ordered. */
#define ADM_MLP_NPARAM 4481

/* Network on n invariant samples I (n x 3): out (n x 10) = psi, dpsi/dI (3),
 * upper Hessian in I (I1I1, I1I2, I2I2, I1I3, I2I3, I3I3), by forward mode
 * through the network. */
adm_status adm_mlp_eval(const float *theta, const float *norm, int64_t n, const float *I, float *out,
                        void *stream);

/* Bytes of the workspace adm_mlp_loss_grad needs (per-warp gradient partials). */
size_t adm_mlp_workspace_size(void);

/* Sobolev loss on standardised quantities,
 *   L = mean (y - (psi - m_psi)/s_psi)^2
 *     + beta mean sum_k (dy/du_k - dpsi/dI_k s_k / s_psi)^2,
 * over n samples (I: n x 3, psi: n, dpsi: n x 3) and its gradient in theta
 * (device, ADM_MLP_NPARAM floats); loss: device double (nullable).  The sum
 * over samples is deterministic. */
adm_status adm_mlp_loss_grad(const float *theta, const float *norm, int64_t n, const float *I,
                             const float *psi, const float *dpsi, float beta, double *loss, float *grad,
                             void *workspace, size_t workspace_bytes, void *stream);

/* One Adam step on theta with moments m, v (all ADM_MLP_NPARAM floats);
 * step counts from 1. */
adm_status adm_mlp_adam(float *theta, float *m, float *v, const float *grad, int64_t step, float lr,
                        float beta1, float beta2, float eps, void *stream);

/* The analytic Neo-Hookean density (the ADM_NH_MEMBRANE density, plane-stress
 * Lame parameters of E, nu) on n deformation samples F (n x 3 x 2 row-major):
 * invariants I (n x 3), psi (n), dpsi/dI (n x 3). */
adm_status adm_mlp_nh_targets(int64_t n, const float *F, double E, double nu, float *I, float *psi,
                              float *dpsi, void *stream);

/* Network used by ADM_MLP_MEMBRANE on this handle (copied; synchronous,
 * allocates on first use).  ADM_MLP_MEMBRANE then evaluates
 * f = thickness * A_rest * psi(I(C)) with FP32 local AD and the tiled
 * assembler (a per-triangle network pass, stage ADM_STAGE_MLP, precedes the
 * element kernel); FP64 and the atomic assembler return ADM_ERR_UNSUPPORTED. */
adm_status adm_mlp_attach(adm_handle h, const float *theta, const float *norm);

/* Device status word of the last evaluation on this handle: ADM_OK,
 * ADM_ERR_DOMAIN or ADM_ERR_TIMEOUT.  Call after synchronising the stream of
 * that evaluation; this call itself blocks until the status is read. */
adm_status adm_get_status(adm_handle h);

const char *adm_strerror(adm_status s);

/* Frees every device and host allocation of the handle (synchronous). */
void adm_destroy(adm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* ADM_H */
