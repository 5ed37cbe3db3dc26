/*
 * gipc_mas_pcg.h -- C ABI of the GB300 Newton-step linear solver.
 *
 * The library solves the Newton system P d = -grad E of implicit IPC
 * (Sec. 3.2, Eq. tailor): it assembles the block-sparse Hessian from
 * duplicate 3x3 blocks (Sec. 5.2), builds the connectivity-enhanced
 * multilevel additive Schwarz (MAS) preconditioner (Sec. 3, supplement
 * Sec. 2) and runs PCG (Sec. 3.2) -- all on one GPU.
 *
 * Conventions shared by every call
 *   - Return value: GS_OK (0) or a negative GS_ERR_* status.  On error no
 *     output handle is created and outputs may be partially written.
 *   - "device" pointers are CUDA device pointers on the context's device;
 *     "host" pointers are ordinary host memory.  The caller owns every
 *     buffer it passes; the library owns gs_mat / gs_mas handles until the
 *     matching *_destroy call.
 *   - All work is issued on the context's stream.  Calls that return sizes
 *     or statuses synchronise that stream before returning.
 *   - Threads: one context per host thread at a time.  A gs_mat or gs_mas
 *     may move between contexts but is used by one at a time: the row SpMV
 *     builds its transposed references and row order into the matrix on
 *     first use, and rebuilds the order when a context with another
 *     GS_TUNE_SPMV_WINDOW uses it.
 *   - Indices are int32; block values are float64, each 3x3 block stored
 *     row-major (9 consecutive doubles).
 *   - Vectors hold 3 doubles per block row (x, y, z).  Several right-hand
 *     sides are stored one after another: entry c of block row i of RHS k
 *     is v[k * 3 * n + 3 * i + c].
 */
#ifndef GIPC_MAS_PCG_H
#define GIPC_MAS_PCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define GS_OK 0
#define GS_ERR_INVALID -1     /* bad argument: null pointer, size or index out of range */
#define GS_ERR_CUDA -2        /* a CUDA runtime call failed (message: gs_last_error) */
#define GS_ERR_NOT_SPD -3     /* non-positive pivot in a domain Cholesky, or p.Ap <= 0 */
#define GS_ERR_MAXITER -4     /* PCG stopped at max_iter before reaching tol; x is written */
#define GS_ERR_NONFINITE -5   /* NaN or Inf met in a reduction */
#define GS_ERR_UNSUPPORTED -6 /* option outside the supported set (e.g. domain size > 32) */
#define GS_ERR_TIMEOUT -7     /* a bounded wait inside a kernel gave up (no hang: the kernel returned) */

typedef struct gs_ctx_s* gs_ctx;
typedef struct gs_mat_s* gs_mat;
typedef struct gs_mas_s* gs_mas;

/* Human-readable name of a status code (static string). */
const char* gs_status_string(int status);
/* Last error message recorded on this thread (static buffer, never null). */
const char* gs_last_error(void);

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device`, issuing work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is
 * borrowed, not owned.  Work buffers are allocated lazily from the
 * device's stream-ordered memory pool and reused across calls. */
int gs_create(gs_ctx* out, int device, void* stream);
int gs_set_stream(gs_ctx ctx, void* stream);
int gs_destroy(gs_ctx ctx);

/* ---------------------------------------------------------------- assembly */
/* Global Hessian assembly by hash-key reduction (Sec. 5.2, Alg.
 * FastHashReduction and Alg. FastSegmentReduction).
 *
 * rows, cols: device int32[n_blocks], block row / column of every input
 *   block, each in [0, n_block_rows).
 * blocks: device double[n_blocks * 9], row-major 3x3 blocks.
 * The inputs describe the full symmetric matrix: an input with
 * row <= col is accumulated, an input with row > col is not consumed (its
 * transpose is the block at (col, row)).  Duplicates are summed.
 * Result (*out): the distinct keys in ascending (row, col) order with
 * their summed blocks -- the paper's Sorted Symmetric Block Coordinates
 * (Sec. 5.3) -- plus a block-row pointer.
 * Errors: GS_ERR_INVALID for n_block_rows <= 0, n_blocks < 0, a null
 * pointer with n_blocks > 0, or any index outside [0, n_block_rows). */
int gs_assemble(gs_ctx ctx, int32_t n_block_rows, const int32_t* rows, const int32_t* cols,
                const double* blocks, int64_t n_blocks, gs_mat* out);

/* Two-level assembly of coupled FEM / affine-body (ABD) blocks (Sec. 5.1,
 * Sec. 5.2 "unifying four block types").
 * Inputs are 3x3 blocks in full-space node numbering (n_nodes nodes),
 * with the same row <= col convention as gs_assemble.  An index
 * n_nodes + 4b + a (a = 0..3) names body b's own reduced block row a: a
 * body's 12 x 12 Hessian (inertia, orthogonality potential) enters as its
 * 3x3 sub-blocks there (the ABD-ABD type of Sec. 5.2) with weight 1.
 * body_of_node: device int32[n_nodes], -1 for a FEM vertex, else the affine
 *   body index in [0, n_bodies).  FEM vertices must be nodes 0..n_fem-1.
 * xbar: device double[n_nodes * 3], rest coordinates of body nodes (read
 *   for nodes with body_of_node >= 0).
 * Level 1 reduces blocks per node pair; level 2 maps each reduced pair
 * through the Jacobians J = [I, xbar_1 I, xbar_2 I, xbar_3 I] (Sec. 3.1),
 * i.e. sub-block (a, b) = w_a(r) w_b(c) C with w = [1, xbar], and reduces
 * again.  Result block rows: FEM vertex v -> v; body b -> the four block
 * rows n_fem + 4b + {0,1,2,3} (q = [p; a_1; a_2; a_3], a_k the columns of A).
 * Errors: as gs_assemble (indices checked against n_nodes + 4 n_bodies),
 * plus GS_ERR_INVALID for a body index out of range or a body node
 * numbered below n_fem. */
int gs_assemble_abd(gs_ctx ctx, int32_t n_nodes, int32_t n_fem, int32_t n_bodies,
                    const int32_t* body_of_node, const double* xbar, const int32_t* rows,
                    const int32_t* cols, const double* blocks, int64_t n_blocks, gs_mat* out);

/* Size of an assembled matrix: block rows and stored (diagonal + upper) blocks. */
int gs_mat_info(gs_mat mat, int32_t* n_block_rows, int64_t* nnzb_upper);
/* Copy the stored blocks out: device int32[nnzb] rid, cid and double[nnzb*9]
 * au, in ascending (row, col) order.  Any output may be NULL (skipped). */
int gs_mat_export(gs_ctx ctx, gs_mat mat, int32_t* rid, int32_t* cid, double* au);
int gs_mat_destroy(gs_mat mat);

/* ---------------------------------------------------------------- SpMV */
#define GS_SPMV_SRBK 0 /* Alg. SRBK: upper blocks, warp segmented reduce + transposed atomics */
#define GS_SPMV_ROW 1  /* row-gather over the upper blocks and their transposes; no atomics,
                          bit-reproducible */
#define GS_SPMV_ROW_FF 2 /* the row-gather product in float-float arithmetic on the FP32 units:
                            A (scaled by powers of two per block row, once per matrix) and x
                            (scaled per RHS) split into pairs of floats, products and sums by
                            error-free transformations (exact product by FMA, Knuth's
                            two-sum).  Error per entry at most ((3m+1)(m+4) + 6) u^2 (|A||x|)_i,
                            u = 2^-24, m = 3 x the row's stored blocks of both triangles
                            (1.9e-11 for a 13-block row; FP64 sums are within m 2^-53);
                            terms below 2^-100 of the row's largest lose their low part.
                            Bit-reproducible; same launch shapes as GS_SPMV_ROW */

/* y = A x for nrhs right-hand sides (Sec. 5.3), A the full symmetric matrix
 * whose diagonal and upper blocks `mat` stores.  x, y: device
 * double[nrhs * 3n], must not overlap.  Errors: GS_ERR_INVALID. */
int gs_spmv(gs_ctx ctx, gs_mat mat, const double* x, double* y, int32_t nrhs, int32_t variant);

/* ---------------------------------------------------------------- partition */
/* Level-0 domain partition (Sec. 3.2, Eq. num_subdomains, supplement
 * Algorithm 1).  Runs on the host, once per mesh, like the paper's METIS
 * pre-processing.  Rule (deterministic; METIS is replaced): recursive
 * coordinate bisection of the rest positions -- split a set needing
 * P = ceil(size / N) > 1 parts along the coordinate of largest extent
 * (ties: x, then y, then z), ordering by (coordinate, node index) and
 * putting the first N * ceil(P / 2) nodes left; leaves are parts numbered
 * left to right, so M = ceil(n_nodes / N) and only the last part is short.
 * Node v gets slot map[v] = N * part + rank of v in its part (ascending
 * node index); slots without a node are padding.
 * X: host double[n_nodes * 3].  map: host int32[n_nodes] (output).
 * n_domains: host, receives M.  Errors: GS_ERR_INVALID. */
int gs_partition(int32_t n_nodes, const double* X, int32_t domain_size, int32_t* map,
                 int32_t* n_domains);

/* Partition of several independent meshes at once (host): mesh s owns nodes
 * [node_off[s], node_off[s+1]) and is partitioned by gs_partition on its
 * own, its slots following those of mesh s-1, so no domain mixes meshes.
 * node_off: host int32[n_sys + 1], node_off[0] = 0, ascending.  X, map,
 * n_domains as gs_partition over all nodes.  Errors: GS_ERR_INVALID. */
int gs_partition_batch(int32_t n_sys, const int32_t* node_off, const double* X, int32_t domain_size, int32_t* map,
                       int32_t* n_domains);

/* The level-0 partition computed on the device (the paper runs METIS on the
 * host, Sec. 3.2; these rules are deterministic and bit for bit the host's).
 * rule GS_PART_RCB: the recursive coordinate bisection of gs_partition.
 * GS_PART_RCB_COMPONENTS: the same bisection inside each connected component
 *   of the mesh graph (components numbered by their smallest node), so no
 *   part mixes two bodies; needs adj_ptr / adj.  On a connected mesh it
 *   equals GS_PART_RCB.
 * GS_PART_MORTON: N consecutive nodes in Morton order (each coordinate cut
 *   to 10 bits over the bounding box, q = min(floor((x - lo) / (hi - lo)
 *   * 1024), 1023), 0 on a flat axis; bits interleaved x, y, z from the
 *   lowest; ties by node index): the level-0 subdomains of the earlier MAS
 *   the paper compares against (Sec. 3.1), for comparisons.
 * Slots as gs_partition: map[v] = N * part + rank of v among its part's
 * nodes in ascending index.
 * X: device double[n * 3]; adj_ptr, adj: device int32 CSR of the mesh graph
 * (may be NULL except for GS_PART_RCB_COMPONENTS); map: device int32[n];
 * n_domains: host, receives the part count.  Uses the context's stream and
 * allocates working memory from its pool.  Errors: GS_ERR_INVALID (a
 * non-finite position, a neighbour out of range, bad arguments). */
#define GS_PART_RCB 0
#define GS_PART_RCB_COMPONENTS 1
#define GS_PART_MORTON 2
int gs_partition_device(gs_ctx ctx, int32_t n, const double* X, const int32_t* adj_ptr, const int32_t* adj,
                        int32_t domain_size, int32_t rule, int32_t* map, int32_t* n_domains);

/* ---------------------------------------------------------------- MAS */
#define GS_PREC_FP64 0 /* domain inverses stored and applied in FP64 */
#define GS_PREC_FP32 1 /* inverses rounded to FP32, applied with FP32 accumulation */
#define GS_PREC_BF16 2 /* level 0: the inverse Cholesky factor W (M_d^-1 = W^T W) rounded to BF16
                          (via FP32, nearest even), applied as W^T (W r) with FP32 accumulation, on
                          the tensor cores when 3N is a multiple of 16 and nrhs <= 8; coarse levels
                          as GS_PREC_FP32.  Rounding the factor, not the inverse, keeps the
                          preconditioner positive semi-definite. */

typedef struct gs_mas_opts {
  int32_t domain_size; /* N: nodes per domain, 1..32 (paper: 16 or 32, Sec. 3.2) */
  int32_t max_levels;  /* upper bound on the number of levels, >= 1 */
  int32_t precision;   /* GS_PREC_* of the stored inverses */
} gs_mas_opts;

/* Build the connectivity-enhanced MAS preconditioner of `mat` on the
 * device (Sec. 3.3, Alg. 1; supplement Algorithms 2-5, Eq. 4-6).
 * map: device int32[n], the level-0 slot of every node (gs_partition);
 *   n_domains0 level-0 domains of domain_size slots each.
 * adj_ptr, adj: device int32 CSR of the mesh node graph (n + 1 entries,
 *   then adj_ptr[n] neighbours); contacts: device int32[2 * n_contacts]
 *   node pairs (may be NULL when n_contacts == 0).  Edges of both define
 *   connectivity at every level.
 * Levels: level l+1's supernodes are the connected components of level
 * l's items inside each domain, numbered domain by domain and by smallest
 * lane; a level is added while fewer than max_levels exist, level l has
 * more than one domain and some items merged.  Level matrices are the
 * Galerkin products S_d C_l A C_l^T S_d^T; each domain's real part is
 * inverted through a Cholesky factorisation.
 * Errors: GS_ERR_INVALID, GS_ERR_UNSUPPORTED (domain_size > 32),
 * GS_ERR_NOT_SPD (a domain pivot <= 0; no handle is returned). */
int gs_build_mas(gs_ctx ctx, gs_mat mat, const int32_t* map, int32_t n_domains0,
                 const int32_t* adj_ptr, const int32_t* adj, const int32_t* contacts,
                 int64_t n_contacts, const gs_mas_opts* opts, gs_mas* out);
/* The same build from the mesh itself: the level-0 partition of the node
 * positions X (device double[n * 3]) by `part_rule` (GS_PART_*) on the
 * device (gs_partition_device), then gs_build_mas.  The call the paper's
 * build_mas(BSR, mesh connectivity) names. */
int gs_build_mas_mesh(gs_ctx ctx, gs_mat mat, const double* X, int32_t part_rule, const int32_t* adj_ptr,
                      const int32_t* adj, const int32_t* contacts, int64_t n_contacts, const gs_mas_opts* opts,
                      gs_mas* out);

/* Level count and item counts: n_items[l] for l < *n_levels (n_items may be
 * NULL; it must hold max_levels entries).  Level 0 counts padded slots. */
int gs_mas_info(gs_mas mas, int32_t* n_levels, int32_t* n_items);
/* coarse: device int32[n], the item of every node at `level` (level 0: map). */
int gs_mas_export_coarse(gs_ctx ctx, gs_mas mas, int32_t level, int32_t* coarse);
/* inv: device double[n_domains(level) * (3N)^2], each domain's inverse,
 * row-major 3N x 3N, padded rows/columns zero (FP64 copy). */
int gs_mas_export_inverse(gs_ctx ctx, gs_mas mas, int32_t level, double* inv);
/* z = M^{-1} r = sum_l C_l^T M_l^{-1} C_l r (supplement Eq. 6) for nrhs
 * right-hand sides; r, z device double[nrhs * 3n], not overlapping. */
int gs_mas_apply(gs_ctx ctx, gs_mas mas, const double* r, double* z, int32_t nrhs);
/* The same apply with no device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * once they are running -- an application that gives the library a fixed
 * memory budget at start-up, where a later cudaMalloc could fail under the
 * cap or stall every stream on the device while memory is mapped.  The
 * coarse-level scratch that gs_mas_apply takes from the memory pool lives
 * here in a fixed 4 MiB array compiled into the library, held by every GPU
 * that loads it until the process exits.
 * Arguments and result: as gs_mas_apply.  Limit: 2 * nrhs * 3 * (items of
 * all levels >= 1, domains padded to N) doubles must not exceed 524,288;
 * otherwise GS_ERR_INVALID with a message naming the sizes.
 * The first call on each context looks the array's address up (with that
 * context's device current) and keeps it in the context; make it before any
 * stream capture begins.  A context created after a device reset looks the
 * address up again.
 * Calls share the array and clear its restricted part on entry; calls whose
 * work overlaps on the GPU race on it. */
int gs_mas_apply_noalloc(gs_ctx ctx, gs_mas mas, const double* r, double* z, int32_t nrhs);
int gs_mas_destroy(gs_mas mas);

/* ---------------------------------------------------------------- PCG */
/* Preconditioned conjugate gradients (Sec. 3.2): x0 = 0, independent
 * recurrences per right-hand side, stopping RHS k when its recurrence
 * residual satisfies ||r||_2 <= tol * ||b_k||_2 (b_k = 0 gives x_k = 0 and
 * 0 iterations) or at max_iter iterations (iteration = one SpMV).
 * b, x: device double[nrhs * 3n].  iters: host int32[nrhs], rel_res: host
 * double[nrhs] (recurrence residual ratio at exit); either may be NULL.
 * spmv_variant: GS_SPMV_*.
 * Returns GS_OK, GS_ERR_MAXITER (some RHS did not converge; x holds the
 * last iterate), GS_ERR_NOT_SPD (p.Ap <= 0), GS_ERR_NONFINITE,
 * GS_ERR_INVALID. */
int gs_pcg_solve(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* b, int32_t nrhs, double tol,
                 int32_t max_iter, int32_t spmv_variant, double* x, int32_t* iters,
                 double* rel_res);

/* Mixed-precision solve: one FP32 MAS-PCG recurrence with FP64 reliable
 * updates (the paper solves in FP64 throughout; this is the library's
 * precision form).  The recurrence runs on an FP32 copy of the blocks, the
 * FP32 (or, for a GS_PREC_BF16 MAS, the BF16-factored) preconditioner and
 * FP32 vectors, with the p.Ap and r.z reductions and alpha, beta in FP64.
 * Once RHS k's FP32 residual has fallen by inner_tol since its last
 * correction, x_k += d_k in FP64, r_k = b_k - A x_k is recomputed with the
 * FP64 SpMV and the recurrence continues from it (search direction kept).
 * RHS k stops once that true residual satisfies ||r_k|| <= tol ||b_k||, the
 * same test as gs_pcg_solve.
 * b, x: device double[nrhs * 3n], RHS-major as everywhere; nrhs 1..8.
 * max_iter bounds the inner iterations summed over outer steps.
 * iters: host int32[nrhs], inner iterations (FP32 SpMVs) per RHS; rel_res:
 * host double[nrhs], final true residual ratio; outer_iters: host, number
 * of reliable updates.  Any of the three may be NULL.  The FP32 copies of
 * the blocks and inverses are made on first use and kept with the handles.
 * Returns as gs_pcg_solve. */
int gs_pcg_solve_mixed(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* b, int32_t nrhs, double tol,
                       int32_t max_iter, double inner_tol, double* x, int32_t* iters, double* rel_res,
                       int32_t* outer_iters);

/* Batched solve of independent systems, one right-hand side each (the
 * paper solves one system at a time; this is the library's batching form).
 * `mat` holds the systems as the diagonal blocks of one block-diagonal
 * matrix -- system s owns block rows [node_off[s], node_off[s+1]) -- and
 * `mas` is built on it from a gs_partition_batch map, so every SpMV and MAS
 * apply serves all systems in one launch, while each system keeps its own
 * PCG recurrence: its own dot products, alpha, beta and stopping test
 * ||r_s|| <= tol ||b_s||.  use_graph != 0 runs the whole iteration loop as
 * one CUDA graph launch (a conditional WHILE node; the loop ends when every
 * system converged or after max_iter iterations); otherwise the host polls
 * a convergence flag every 8 iterations.
 * node_off: host int32[n_sys + 1]; b, x: device double[3n]; iters: host
 * int32[n_sys]; rel_res: host double[n_sys] (either may be NULL).
 * Returns as gs_pcg_solve. */
int gs_pcg_solve_batch(gs_ctx ctx, gs_mat mat, gs_mas mas, int32_t n_sys, const int32_t* node_off, const double* b,
                       double tol, int32_t max_iter, int32_t use_graph, double* x, int32_t* iters, double* rel_res);

/* ---------------------------------------------------------------- adjoint */
/* Gradients through x = A^{-1} b for a loss L(x) (the paper solves only
 * forward; this is the library's differentiation form).
 * x: device double[nrhs * 3n], the forward solution; g: dL/dx, same layout.
 * lam: output dL/db = A^{-1} g, solved with the same preconditioner to tol
 *   (mixed != 0: by gs_pcg_solve_mixed, else by gs_pcg_solve).
 * dLdH: optional output double[nnzb * 9], the gradient with respect to each
 *   stored block of `mat` (row-major 3x3): -sum_k (lam_r x_c^T + x_r lam_c^T)
 *   for an off-diagonal block (it also sits transposed at (c, r)) and
 *   -sum_k lam_r x_r^T for a diagonal block.
 * dLdinput: optional output double[n_blocks * 9] for the triplets given to
 *   gs_assemble: each input receives the gradient of the stored block it was
 *   summed into, 0 for inputs below the diagonal (needs dLdH).
 * iters: optional host int32[nrhs], iterations of the adjoint solve.
 * Returns as gs_pcg_solve. */
int gs_adjoint(gs_ctx ctx, gs_mat mat, gs_mas mas, const double* x, const double* g, int32_t nrhs, double tol,
               int32_t max_iter, int32_t mixed, double* lam, double* dLdH, double* dLdinput, int32_t* iters);

/* ---------------------------------------------------------------- tuning */
/* Launch shapes a context uses, set by the autotuner (or by hand).  Values
 * outside the listed set return GS_ERR_INVALID.  Results do not depend on
 * the choice except through the order of floating-point sums. */
#define GS_TUNE_SPMV_LANES 0      /* lanes per block row of the FP64 row SpMV: 1, 2 (default), 4, 8 */
#define GS_TUNE_SPMV32_LANES 1    /* lanes per block row of the FP32 SpMV of the mixed solve: 2 (default), 4 */
#define GS_TUNE_APPLY_RHS 2       /* right-hand sides per thread in the level-0 MAS product: 2, 4 (default), 8 */
#define GS_TUNE_BATCH_CHUNK 3     /* vector entries per work item of the batched reductions: 1024..16384 (4096) */
#define GS_TUNE_BF16_TC 4         /* BF16 level-0 apply on the tensor cores (1, default) or on FP32 cores (0);
                                     the tensor-core form needs 3N a multiple of 16 (N = 16, 32) and nrhs <= 8 */
#define GS_TUNE_F64_TC 5          /* FP64 MAS apply on the BF16 tensor cores by exact digit splitting (FP64
                                     accuracy): 4 (default) from 7 BF16 digit matrices per inverse (3.5x
                                     the bytes of the packed FP64 lower triangle), one CTA of 256 threads
                                     per domain (two threads per row of the epilogue, four RHS each); 1 the
                                     same digits, 128 threads per domain; 2 the same digits, one persistent
                                     warp-specialised CTA per SM for level 0; 3
                                     from each symmetric inverse's block lower triangle, scaled
                                     symmetrically and stored as 8 base-128 digit bytes per entry (1.07x),
                                     expanded to BF16 in shared memory (fewer bytes, more instructions); 0
                                     on the FP64 cores.  The digit storage is made when a preconditioner is built or
                                     refreshed, for the value set then; applying it with a value whose
                                     storage was not made uses the FP64 cores.  Needs N = 16 or 32 and
                                     nrhs <= 8 */
#define GS_TUNE_SPMV_WINDOW 6     /* row order of the row SpMVs: longest rows first within windows of this
                                     many consecutive rows (256..65536, a power of 2; default 1024), so that
                                     the rows in flight stay neighbours and their gathers hit L2; 0: over
                                     all rows */
#define GS_TUNE_SPMV_WS 7         /* FP64 row SpMV: 1 (default) a persistent grid (two blocks per SM) whose
                                     warps take the next rows of the order from a counter; 0 one thread
                                     group per row */
#define GS_TUNE_SPMV_FF_RHS 8     /* float-float SpMV (GS_SPMV_ROW_FF): right-hand sides per thread and pass,
                                     8 (default; the GS_TUNE_SPMV_LANES lanes of a row share its blocks), or
                                     4 / 2 / 1 (each of nrhs / value lanes walks all the row's blocks for its own
                                     right-hand sides; fewer registers, more resident warps) */
#define GS_TUNE_COUNT 9           /* number of parameters */
int gs_tune_set(gs_ctx ctx, int32_t param, int32_t value);
int gs_tune_get(gs_ctx ctx, int32_t param, int32_t* value);

/* ---------------------------------------------------------------- microbenchmarks */
/* Measurement only; not part of the solve.
 *
 * gs_micro_segment_reduce: reduce nb 3x3 blocks (device double[nb * 9]) whose
 * device uint64 keys are sorted ascending (each key < 2^62) into one block per
 * distinct key, written to out (device double[nb * 9], first *n_unique used).
 * method 0 = the paper's FastHashReduction (run flags, exclusive scan, warp
 * head-segmented reduction; Sec. 5.2), method 1 = the CUB library's
 * DeviceReduce::ReduceByKey, the baseline the paper compares against.
 * *ms: device time of the reduction (events on the context's stream; for
 * method 0 excluding the readback of the unique count between its phases).
 *
 * gs_micro_bsr_spmv_cusparse: y = A x with the cuSPARSE library's BSR SpMV on
 * the FULL matrix (both triangles; 3x3 row-major blocks; device CSR-of-blocks
 * row_ptr[n + 1], col_ind[nnzb], vals[nnzb * 9]; x, y device double[3n]),
 * repeated `reps` times; *ms = mean time per call.  The baseline for the
 * paper's symmetric storage (Sec. 5.3).
 * Errors: GS_ERR_INVALID for bad arguments, GS_ERR_CUDA for library failures. */
int gs_micro_segment_reduce(gs_ctx ctx, int64_t nb, const uint64_t* keys, const double* blocks, int32_t method,
                            double* out, int64_t* n_unique, float* ms);
int gs_micro_bsr_spmv_cusparse(gs_ctx ctx, int32_t n, int32_t nnzb, const int32_t* row_ptr, const int32_t* col_ind,
                               const double* vals, const double* x, double* y, int32_t reps, float* ms);

/* ---------------------------------------------------------------- elastic bodies and Newton */
/* A tet mesh body on the device with the stable Neo-Hookean energy
 * (Sec. 3.1 names the elastic energies the Hessian is assembled from; the
 * form used is Smith, de Goes and Kim 2018 without the log term):
 *   Psi(F) = mu/2 (|F|^2 - 3) + lam/2 (det F - alpha)^2, alpha = 1 + mu/lam,
 * mu = 4/3 mu_L, lam = lam_L + 5/6 mu_L from Young's modulus E and Poisson's
 * ratio nu.  The incremental potential of one implicit-Euler step is
 *   E(x) = sum_t vol_t Psi(F_t) + sum_v m_v/(2 dt^2) |x_v - xt_v|^2
 *        + sum_springs 1/2 (x_i - x_j - r)^T K (x_i - x_j - r),
 * m_v = rho (sum of the adjacent rest volumes) / 4.  Its Hessian is the
 * element Hessians, each projected to positive semi-definite by the analytic
 * eigensystem of the F-Hessian (negative eigenvalues set to 0), plus
 * M / dt^2 and the spring blocks [K, -K; -K, K].
 * Assembly follows the paper's hash-key reduction (Sec. 5.1-5.2) with the
 * pattern fixed: element keys are sorted once when the body is created,
 * spring keys whenever the springs change, and every later assembly only
 * writes values and reduces them in the stored order. */
typedef struct gs_fem_s* gs_fem;

/* X: device double[n_vertices * 3] rest positions (copied); tets: device
 * int32[n_tets * 4], four distinct vertices each (copied).  rho: density,
 * dt: time step.  Errors: GS_ERR_INVALID (sizes, E <= 0, nu outside
 * [0, 0.5), rho or dt <= 0, an index out of range or repeated in a tet),
 * GS_ERR_NONFINITE (a rest tet of zero volume). */
int gs_fem_create(gs_ctx ctx, int32_t n_vertices, int64_t n_tets, const double* X, const int32_t* tets,
                  double E, double nu, double rho, double dt, gs_fem* out);
/* Replace the body's springs (contact pairs in the synthetic scenes): pairs
 * device int32[2 n] of distinct vertices, K device double[9 n] symmetric
 * PSD 3x3 stiffness (row-major), rest device double[3 n] rest offsets
 * x_i - x_j.  Copied.  Only these keys are sorted; they are merged into the
 * element pattern.  n = 0 removes them.  Matrices assembled before the call
 * can no longer be refilled.  Errors: GS_ERR_INVALID. */
int gs_fem_set_springs(gs_ctx ctx, gs_fem fem, const int32_t* pairs, const double* K, const double* rest,
                       int64_t n);
/* Stored blocks of the merged pattern and of the element part alone; the
 * Lame parameters (mu, lam) used.  Outputs host, each may be NULL. */
int gs_fem_info(gs_fem fem, int64_t* n_stored, int64_t* n_element_stored, double* lame_mu, double* lame_lambda);
/* Rest data: w device double[n_tets * 12] (F = sum_a x_a w_a^T, w[t][a][j]),
 * vol device double[n_tets], mass device double[n_vertices]; each may be NULL. */
int gs_fem_export_rest(gs_ctx ctx, gs_fem fem, double* w, double* vol, double* mass);
/* E(x) (host double) and, if grad is not NULL, its gradient (device
 * double[3 n_vertices]) at x (device double[3 n_vertices]); xt the
 * predicted positions, same layout.  Sums in a fixed order (bit-reproducible). */
int gs_fem_energy(gs_ctx ctx, gs_fem fem, const double* x, const double* xt, double* energy, double* grad);
/* The Hessian as upper triplets: 10 per tet in the pair order (0,0) (0,1)
 * (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3), each at (min, max) of its
 * two vertices (transposed when the first is the larger); then one
 * m_v / dt^2 I per vertex; then 3 per spring: (i, i) K, (j, j) K,
 * (min, max) -K.  rows, cols device int32, blocks device double[9 each]
 * (row-major), 10 n_tets + n_vertices + 3 n_springs entries; rows and cols
 * may be NULL. */
int gs_fem_triplets(gs_ctx ctx, gs_fem fem, const double* x, int32_t* rows, int32_t* cols, double* blocks);
/* A new matrix (gs_mat_destroy) holding the Hessian at x in the body's
 * pattern. */
int gs_fem_assemble(gs_ctx ctx, gs_fem fem, const double* x, gs_mat* out);
/* New values at x into a matrix made by gs_fem_assemble of the same body
 * since its springs last changed (the numeric phase: no sort).
 * Errors: GS_ERR_INVALID for a matrix of another pattern. */
int gs_fem_refill(gs_ctx ctx, gs_fem fem, const double* x, gs_mat mat);
int gs_fem_destroy(gs_fem fem);

/* New level matrices and inverses for `mat` (same nodes) in an existing
 * preconditioner: the numeric part of gs_build_mas, keeping the partition
 * and the levels (they depend only on the graph and the contacts).
 * Errors: as gs_build_mas; GS_ERR_INVALID for a matrix of another size. */
int gs_mas_refresh(gs_ctx ctx, gs_mas mas, gs_mat mat);

/* ---------------------------------------------------------------- assembly primitives
 * The two device primitives of the hash assembly (Sec. 5.2, Alg.
 * FastHashReduction), exposed for tests and measurement; gs_assemble and
 * gs_assemble_abd call them internally.
 *
 * gs_prim_sort_pairs: keys_out / vals_out (device uint64[n] / uint32[n])
 * receive the pairs of keys_in / vals_in sorted by the key bits
 * [0, end_bit), 1 <= end_bit <= 64, stable (equal keys keep their input
 * order); a least-significant-digit radix sort with 8-bit digits.  The inputs
 * are not modified and must not be the outputs.  Uses the context's scratch.
 * gs_prim_exclusive_scan: out[i] = in[0] + ... + in[i-1] (device int32[n],
 * n < 2^31, in == out allowed).  Both run on the context's stream and return
 * without synchronising.  Errors: GS_ERR_INVALID (null pointers, sizes,
 * end_bit, aliasing), GS_ERR_CUDA. */
int gs_prim_sort_pairs(gs_ctx ctx, const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                       uint32_t* vals_out, int64_t n, int32_t end_bit);
int gs_prim_exclusive_scan(gs_ctx ctx, const int32_t* in, int32_t* out, int64_t n);

/* ---------------------------------------------------------------- stiff cloth
 * Element Hessians of a triangle sheet on the device (the stiff-cloth
 * scenes; Sec. 4 for the strain limit): per triangle, with F = sum_a x_a w_a^T
 * from the in-plane rest edge matrix and a_t = rest area * thickness, the
 * membrane Hessian a_t (Baraff-Witkin stretching lam (|f_d| - 1)^2 per
 * direction with its negative eigenvalue clamped, the cubic strain limit
 * E max(|f_d| - 1, 0)^3 with the analytic PSD Hessian of Eq. Stretch_Hessian,
 * Gauss-Newton shearing 0.3 lam (f_0 . f_1)^2) pulled back to the vertex
 * blocks; per interior edge (hinge) the Gauss-Newton bending Hessian
 * 2 k_b grad(theta) grad(theta)^T of the dihedral angle, k_b = E t^3 / 12
 * |e_rest|^2 / (A_1 + A_2); lumped masses rho t A / 3 per triangle corner as
 * m / dt^2 I. */
typedef struct gs_cloth_s* gs_cloth;

/* X: device double[n_vertices * 3] rest positions (only x and y are used: the
 * sheet rests in the plane z = 0); tris: device int32[n_tris * 3]; hinges:
 * device int32[n_hinges * 4] = (e_0, e_1, o_1, o_2), the shared edge and the
 * opposite vertex of each of its two triangles.  Copied.  Errors:
 * GS_ERR_INVALID (sizes, E or lam < 0, thickness, rho or dt <= 0, an index out
 * of range or repeated in a triangle), GS_ERR_NONFINITE (a degenerate rest
 * triangle or hinge). */
int gs_cloth_create(gs_ctx ctx, int32_t n_vertices, const double* X, int64_t n_tris, const int32_t* tris,
                    int64_t n_hinges, const int32_t* hinges, double E, double lam, double thickness, double rho,
                    double dt, gs_cloth* out);
/* The Hessian at x (device double[3 n_vertices]) as upper triplets: 6 per
 * triangle in the pair order (0,0) (0,1) (0,2) (1,1) (1,2) (2,2), then 10 per
 * hinge in the pair order of (e_0, e_1, o_1, o_2) with a <= b, each at (min,
 * max) of its two vertices (transposed when the first is the larger), then one
 * mass block per vertex; rows, cols device int32 (each may be NULL), blocks
 * device double[9 each] (row-major); gs_cloth_info gives the count.
 * Asynchronous on the context's stream: the call returns once the kernels are
 * queued.  Errors: GS_ERR_INVALID (a null argument, a cloth of another
 * context).  The values are not checked: a deformed triangle with a
 * zero-length edge direction, or a hinge whose triangle collapsed, gives
 * non-finite blocks, which gs_build_mas reports as GS_ERR_NOT_SPD and
 * gs_pcg_solve as GS_ERR_NONFINITE. */
int gs_cloth_triplets(gs_ctx ctx, gs_cloth c, const double* x, int32_t* rows, int32_t* cols, double* blocks);
int gs_cloth_info(gs_cloth c, int64_t* n_triplets);
int gs_cloth_destroy(gs_cloth c);

typedef struct gs_newton_opts {
  double tol;            /* stop when max_i |d_i| <= tol * dt (the step's velocity is small) */
  int32_t max_newton;    /* steps at most */
  double pcg_tol;        /* relative residual of each linear solve */
  int32_t pcg_max_iter;
  int32_t spmv_variant;  /* GS_SPMV_* */
  int32_t domain_size;   /* MAS options */
  int32_t max_levels;
  int32_t precision;     /* GS_PREC_* */
  int32_t part_rule;     /* GS_PART_* level-0 partition of the rest positions */
  double armijo;         /* c in E(x + a d) <= E(x) + c a g.d, 0 <= c < 1 */
  int32_t max_halvings;  /* line-search halvings per step at most (the last step is taken) */
} gs_newton_opts;

typedef struct gs_newton_stats {
  int32_t iterations;      /* steps taken */
  int32_t pcg_iterations;  /* summed over the solves */
  int32_t halvings;        /* line-search halvings, summed */
  int32_t converged;       /* 1 when the last direction met tol */
  double energy0, energy;  /* E at the start and at the returned x */
  double step_inf;         /* max |d| of the last direction */
  double ms[6];            /* CUDA-event time: energy + gradient, Hessian + assembly, MAS build / refresh,
                              PCG, line search, total */
} gs_newton_stats;

/* Newton's method on the incremental potential (Fig. framework; supplement
 * Eq. 1): per step the gradient, the projected Hessian refilled into the
 * fixed pattern, the MAS built once (partition of the rest positions by
 * part_rule, adjacency adj_ptr / adj as in gs_build_mas, springs as
 * contacts) and refreshed after, d = -H^-1 g by MAS-PCG (an unconverged
 * solve still gives a descent direction and is used), a stop when
 * max |d| <= tol dt, and backtracking from a = 1 by halving until the
 * Armijo condition holds.  x: device double[3 n_vertices], the start,
 * overwritten by the result; xt: predicted positions.  energies: host
 * double[max_newton + 1] or NULL, E at every iterate.
 * Returns GS_OK when converged, GS_ERR_MAXITER after max_newton steps
 * (x holds the last iterate), GS_ERR_NOT_SPD if g.d >= 0, or the status
 * of a failed assembly, build or solve. */
int gs_fem_newton(gs_ctx ctx, gs_fem fem, const double* xt, double* x, const int32_t* adj_ptr,
                  const int32_t* adj, const gs_newton_opts* opts, gs_newton_stats* stats, double* energies);

/* ---------------------------------------------------------------- measurement */
/* Kernel classes the library counts (and optionally times) per context.
 * The split follows the paper's cost model T = T_ga + T_pa + N_pcg T_pcg
 * with T_pcg = T_spmv + T_ap + T_dot + T_axpby (supplement Eq. 1-2). */
#define GS_K_ASSEMBLE 0         /* key encode, run flags, segment reduction, row pointers */
#define GS_K_LIBPRIM 1          /* radix sort / scan primitives from the CUDA toolkit (CUB) */
#define GS_K_SPMV 2             /* symmetric SpMV */
#define GS_K_MAS_LEVELS 3       /* connectivity masks, expansion, numbering, coarse tables */
#define GS_K_MAS_MATRICES 4     /* level-matrix scatter and per-domain reduction */
#define GS_K_MAS_INVERT 5       /* per-domain Cholesky inverses */
#define GS_K_MAS_APPLY_L0 6     /* level-0 dense products fused with the prolongation */
#define GS_K_MAS_APPLY_COARSE 7 /* restriction and coarse-level dense products */
#define GS_K_PCG_VECTOR 8       /* dot products and vector updates */
#define GS_K_OTHER 9            /* validation and setup kernels */
#define GS_K_ELEMENT 10         /* element Hessians, forces, energies and rest shapes (gs_fem_*) */
#define GS_K_COUNT 11

/* Start counting kernel launches per class on `ctx`; classes whose bit is
 * set in `timed_classes` are also bracketed by CUDA events on the context
 * stream (adds two event records per such launch). */
int gs_profile_begin(gs_ctx ctx, uint32_t timed_classes);
/* Stop, synchronise the stream and report per class: launches (host
 * int64[GS_K_COUNT]) and summed event time in ms (host double[GS_K_COUNT],
 * 0 for untimed classes).  Either output may be NULL. */
int gs_profile_end(gs_ctx ctx, int64_t* launches, double* ms);

/* Device allocations the library has made on `ctx` so far (stream-ordered
 * pool allocations of matrices, preconditioners and scratch; gs_create's own
 * 256-byte flag word is not counted): their number and total bytes.  Either
 * output may be NULL.  Lets a caller check that a call allocated nothing. */
int gs_ctx_alloc_stats(gs_ctx ctx, int64_t* n_allocs, int64_t* bytes);

/* Testing aid: OR `flags` into the context's device error word, as a kernel
 * whose check failed would (bits: 1 index out of range, 2 not positive
 * definite, 4 non-finite, 8 a bounded wait gave up).  The next call that
 * reads the word reports the matching status and clears it.  It stands in
 * for a device-side failure without making one.  GS_ERR_INVALID for unknown
 * bits. */
int gs_debug_raise_flags(gs_ctx ctx, int32_t flags);

#ifdef __cplusplus
}
#endif

#endif /* GIPC_MAS_PCG_H */
