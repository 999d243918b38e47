/*
 * gbpcg.h -- C ABI of libgbpcg.so, a GB300 (sm_103a) implementation of the
 * Jacobi-preconditioned conjugate-gradient hot path studied in arxiv
 * 2603.23343 ("Numerical Kernels on a Spatial Accelerator: A Study of
 * Tenstorrent Wormhole").
 *
 * Problem (Sec. VII): solve A x = b where A is the matrix-free seven-point
 * finite-difference operator of Sec. VI with zero Dirichlet boundaries on the
 * unit cube, preconditioned by Jacobi (element-wise scaling by the inverse
 * diagonal).  The three kernels the paper composes are exposed on their own:
 * element-wise axpy (Sec. IV), the global dot-product reduction (Sec. V) and
 * the stencil (Sec. VI).
 *
 * Conventions shared by every entry point
 *   - Grids: nx*ny*nz interior points, x fastest, index (k*ny + j)*nx + i,
 *     spacing h_d = 1/(n_d + 1).  Constant coefficient:
 *       (A u)_c = sum_d (2 u_c - u_{c-e_d} - u_{c+e_d}) / h_d^2
 *     Block coefficient k (constant on kbx*kby*kbz blocks):
 *       (A u)_c = sum_d sum_{+-} k_f (u_c - u_nb) / h_d^2,
 *     k_f = harmonic mean of the two cells' k on interior faces, the cell's
 *     own k on boundary faces.  Points outside the grid hold u = 0.
 *   - Memory: every pointer is a plain address owned by the caller; the
 *     library never frees caller memory and allocates no device memory in
 *     these calls (scratch comes from caller-provided workspaces).  Device
 *     arrays must be 16-byte aligned for the fast (TMA) path; any alignment
 *     works, more slowly, otherwise.
 *   - Streams: work is enqueued on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  Only gbpcg_pcg_solve* synchronise the stream,
 *     once at the end, to fill the host-side result.
 *   - Errors: functions return a gbpcg_status.  Invalid arguments return
 *     GBPCG_ERR_ARG before anything is launched; CUDA failures return
 *     GBPCG_ERR_CUDA.  gbpcg_last_error() gives a message for the calling
 *     thread's last failure.
 */
#ifndef GBPCG_H
#define GBPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *gbpcg_stream; /* identical to cudaStream_t */

typedef enum {
    GBPCG_OK = 0,
    GBPCG_ERR_ARG = 1,         /* bad shape, NULL pointer, small workspace, bad dtype */
    GBPCG_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    GBPCG_NOT_CONVERGED = 3,   /* maxit reached before the tolerance */
    GBPCG_BREAKDOWN = 4,       /* p.Ap <= 0 or a non-finite scalar */
    GBPCG_TIMEOUT = 5,         /* a bounded device wait gave up */
    GBPCG_FALLBACK_USED = 6    /* learned preconditioner rejected; Jacobi finished */
} gbpcg_status;

typedef enum {
    GBPCG_F32 = 0,
    GBPCG_BF16 = 1,
    GBPCG_F16 = 2,
    GBPCG_F64 = 3
} gbpcg_dtype;

typedef enum {
    GBPCG_PRECOND_JACOBI = 0,
    GBPCG_PRECOND_LEARNED = 1, /* gbpcg_fcg_solve only */
    GBPCG_PRECOND_MG = 2       /* gbpcg_mg_pcg_solve only */
} gbpcg_precond;

/* Grid and operator.  k_block == NULL selects the constant-coefficient
 * (Poisson) operator; otherwise it is a DEVICE array of float, one value per
 * block, shape (ceil(nz/kbz), ceil(ny/kby), ceil(nx/kbx)) row-major. */
typedef struct gbpcg_grid {
    int32_t nx, ny, nz;
    const float *k_block;
    int32_t kbx, kby, kbz;
} gbpcg_grid;

/* Flags of gbpcg_opts.flags */
#define GBPCG_FLAG_HOST_IO 1u /* b and x may be host pointers; staged through the workspace */
#define GBPCG_FLAG_PROFILE 2u /* launch the iteration kernels one by one (no graph), each
                                 bracketed by CUDA events; fills gbpcg_result.pass_ms (BF16 /
                                 F16 storage: the inner solves' passes, summed over the steps) */
#define GBPCG_FLAG_AUTOTUNE 4u /* batched solves: pick each shape's tile configuration by timing
                                  (cached per shape in the process); the workspace grows by a
                                  scratch x per problem */
#define GBPCG_FLAG_HOST_LOOP 8u /* the paper's FP32 variant reads the residual norm back to the
                                   host every iteration (Sec. VII): the fused kernels launched one
                                   iteration at a time, the host reading the device's stop flag
                                   after each (FP32 storage; results equal the graph's bit for
                                   bit) */
#define GBPCG_FLAG_BATCH_GRAPH 32u /* batched solves: one CUDA graph with a branch per problem
                                      instead of the single persistent kernel */
#define GBPCG_FLAG_SPLIT 16u /* the paper's FP32 split-kernel solver (Sec. VII) and its H100
                                comparator's structure: one kernel per operation (stencil, dot,
                                axpy, element-wise Jacobi scaling, p update), alpha and beta formed
                                on the host from dot products read back every iteration.  FP32
                                device b and x, constant coefficient, no residual replacement;
                                rel_res_true is not evaluated (0) */

typedef struct gbpcg_opts {
    double tol;            /* stop when ||r_k||_2 / ||b||_2 <= tol (recursive residual) */
    int32_t maxit;         /* iteration cap (number of A.p products) */
    int32_t precond;       /* gbpcg_precond */
    int32_t storage;       /* gbpcg_dtype of the iteration vectors: F32, or BF16 / F16 for
                              mixed precision with FP64 iterative refinement */
    int32_t io_dtype;      /* gbpcg_dtype of b and x: F32 or F64 (F64 required with 16-bit storage) */
    uint32_t flags;        /* GBPCG_FLAG_* */
    int32_t tile_cfg;      /* 0: automatic; else (a + 1) | (b + 1) << 8 picks the tile
                              configuration of pass A / pass B (see gbpcg_tile_config) */
    void *workspace;       /* device scratch owned by the caller */
    size_t workspace_bytes;
    double inner_tol;      /* refinement (16-bit storage): relative tolerance of each inner solve;
                              0 selects the default, 0.1 for BF16 and 1e-2 for F16 */
    int32_t max_outer;     /* refinement: maximum outer FP64 steps */
    int32_t fcg_m;         /* gbpcg_fcg_solve: each search direction is A-orthogonalised against the
                              last fcg_m ones (1 .. 32; 0 selects 24); ignored elsewhere */
} gbpcg_opts;

typedef struct gbpcg_result {
    int32_t iters;             /* iterations taken */
    int32_t status;            /* gbpcg_status of the solve */
    double rel_res_recursive;  /* ||r||/||b|| of the recursively updated residual */
    double rel_res_true;       /* ||b - A x||/||b|| recomputed in FP64 on the GPU */
    double time_ms;            /* device time of the solve (CUDA events) */
    double pass_ms[2];         /* GBPCG_FLAG_PROFILE: summed time of the pass-A / pass-B launches */
    int32_t pass_launches[2];  /* GBPCG_FLAG_PROFILE: number of timed launches of each pass */
    int32_t replacements;      /* residual replacements (x flushed, r = b - A x in FP64) */
    int32_t refine_steps;      /* outer refinement steps (16-bit storage), else 0 */
    int32_t pass_ctas[2];      /* GBPCG_FLAG_PROFILE: CTAs per launch of pass A / pass B (tiles x z
                                  chunks, pass B's chunks possibly cut into parts) */
} gbpcg_result;

/* Library version string, e.g. "gbpcg 0.1 sm_103a". */
const char *gbpcg_version(void);

/* Message describing the calling thread's last failure ("" if none). */
const char *gbpcg_last_error(void);

/* Bytes of scratch gbpcg_dot needs (a small constant; at least 256-byte
 * aligned device memory is expected). */
size_t gbpcg_dot_workspace_size(void);

/*
 * q = A p  (Sec. VI: seven-point stencil, zero Dirichlet; Sec. VII: the
 * operator of the solver).  p and q are DEVICE arrays of nx*ny*nz elements of
 * `dtype` (F32, BF16, F16: arithmetic in FP32; F64: arithmetic in FP64);
 * they must not overlap.  Values outside the grid are zero.
 */
int gbpcg_stencil_apply(const gbpcg_grid *grid, int32_t dtype, const void *p, void *q,
                        gbpcg_stream stream);

/*
 * *result = sum_i x_i y_i  (Sec. V: element-wise product, local sums, one
 * global reduction).  x, y: DEVICE arrays of n elements of dtype (F32, BF16,
 * F16, F64); result: DEVICE double.  Per-thread sums are FP32 (FP64 for F64
 * input); block and grid sums are FP64 and taken in a fixed order, so the
 * result is bitwise reproducible.  workspace: DEVICE scratch of at least
 * gbpcg_dot_workspace_size() bytes; concurrent calls need distinct
 * workspaces.  n = 0 writes 0.
 */
int gbpcg_dot(int64_t n, int32_t dtype, const void *x, const void *y, double *result,
              void *workspace, size_t workspace_bytes, gbpcg_stream stream);

/*
 * *result = sum_i x_i y_i, like gbpcg_dot, without any memory from the
 * caller or the allocator.  (The paper has no counterpart; this exists for
 * callers that cannot allocate device memory: code running while a stream is
 * being captured into a CUDA graph, where cudaMalloc is not allowed; code
 * that runs under another framework's memory pool and must not create
 * allocations of its own; and latency-critical loops that cannot afford the
 * device synchronisation cudaMalloc/cudaFree may cause.)
 *
 * Its scratch is a static 128 KiB device array inside the library, present on
 * every GPU that loads it until the process exits.  The first call on a
 * device looks up that array's device address and keeps it for the life of
 * the process, so make that first call outside any stream capture; the kept
 * address does not survive cudaDeviceReset on that device (do not call this
 * function on a device after resetting it).  n is limited to 2^30 elements; larger n
 * returns GBPCG_ERR_ARG.  All calls share the one array: calls that may
 * overlap on the GPU (different streams, or different host threads without
 * ordering) race and must be serialised by the caller.  x, y: DEVICE arrays
 * of n elements of dtype; result: DEVICE double; n = 0 writes 0.
 */
int gbpcg_dot_noalloc(int64_t n, int32_t dtype, const void *x, const void *y, double *result,
                      gbpcg_stream stream);

/*
 * Reduction variants of the dot product (Sec. V compares reducing each tile
 * to a scalar before sending, Method 1, with sending whole tiles and reducing
 * at the root, Method 2, and two routes of the partial sums through the
 * network).  *result = sum_i x_i y_i with FP32 per-thread sums of four
 * products added into FP64, then:
 *   0  one partial per CTA, the last CTA to arrive adds them in block order
 *      (gbpcg_dot's scheme; Method 1)
 *   1  one partial per warp (8 per CTA), the last CTA adds them (Method 2)
 *   2  one partial per CTA, added by a second kernel launch
 *   3  one partial per CTA, FP64 atomicAdd into one accumulator (order not
 *      fixed: the result may differ in the last bits from run to run)
 *   4  one partial per CTA; the last CTA of each group of 32 adds its group,
 *      the last group to finish adds the group totals (a two-level tree)
 * x, y: DEVICE FP32, 16-byte aligned, n >= 1; result: DEVICE double;
 * workspace: DEVICE, gbpcg_dot_variant_workspace_size() bytes, 256-byte
 * aligned.  Variants 0, 1, 2 and 4 are bitwise reproducible.
 */
size_t gbpcg_dot_variant_workspace_size(void);
int gbpcg_dot_variant(int32_t variant, int64_t n, const float *x, const float *y, double *result,
                      void *workspace, size_t workspace_bytes, gbpcg_stream stream);

/*
 * Boundary-handling variants of q = A p (Sec. VI-C measures the cost of
 * setting the boundary halo to zero by hand), constant coefficient, FP32
 * DEVICE p and q:
 *   0  TMA boxes, the out-of-grid part zero-filled by the TMA unit (the
 *      library's stencil; needs 16-byte aligned arrays, nx a multiple of 4)
 *   1  boxes copied with plain loads, each element bounds-checked and set to
 *      zero outside the grid
 *   2  TMA boxes, then the out-of-grid part of every box that touches the
 *      boundary set to zero again by the threads (explicit zero fill)
 * All three give the same q bit for bit.
 */
int gbpcg_stencil_apply_variant(const gbpcg_grid *grid, int32_t variant, const float *p, float *q,
                                gbpcg_stream stream);

/*
 * y = alpha x + y  (Sec. IV: element-wise arithmetic).  x, y: DEVICE arrays of
 * n elements of dtype (F32, BF16, F16: FP32 arithmetic; F64); in place on y.
 */
int gbpcg_axpy(int64_t n, int32_t dtype, double alpha, const void *x, void *y,
               gbpcg_stream stream);

/* Tile configuration `index` (0 .. count-1) of the solver's data passes: tile
 * width tx and height ty in grid points, pipeline stages.  Returns
 * GBPCG_ERR_ARG past the last configuration (the way to count them).  Used
 * by autotuners together with gbpcg_opts.tile_cfg. */
int gbpcg_tile_config(int32_t index, int32_t *tx, int32_t *ty, int32_t *stages);

/* Bytes of workspace gbpcg_pcg_solve needs for this grid and options. */
int gbpcg_workspace_size(const gbpcg_grid *grid, const gbpcg_opts *opts, size_t *bytes);

/*
 * Jacobi-preconditioned CG (Sec. VII) for A x = b, with FP32 vectors and
 * FP64 scalars.  Updates are accumulated in a correction vector and, at every
 * two decades of residual reduction and at recursive convergence, flushed into x
 * while the residual is replaced by b - A x computed in FP64 (reliable
 * updates), so the returned x meets the tolerance in its true residual.
 * The FP32 vectors work on s b and s x, s a power of two that brings max |b|
 * near 1 when it is far from 1: any scale of b that FP64 can hold converges
 * alike (a solve of 2^k b returns 2^k times the solution of b, bit for bit).
 *
 * Mixed precision (opts->storage BF16 or F16, FP64 b and x): iterative
 * refinement.  Each outer step computes r = b - A x in FP64 and stops when
 * ||r||/||b|| <= tol; otherwise it solves the scaled correction equation
 * with 16-bit vectors and FP32 arithmetic to opts->inner_tol (at most maxit
 * iterations) and adds the correction to x in FP64; at most opts->max_outer
 * steps.  result->iters counts all inner iterations.
 *
 * b (read) and x (initial
 * guess in, solution out) hold nx*ny*nz elements of opts->io_dtype; they are
 * DEVICE pointers, or HOST pointers when opts->flags has GBPCG_FLAG_HOST_IO
 * (then they are copied through the workspace inside the call).  The whole
 * iteration runs on the device inside one CUDA graph (no per-iteration host
 * round trip; compare the paper's FP32 variant, which reads the norm back
 * every iteration).  Stops when ||r||/||b|| <= tol or after maxit
 * iterations; b = 0 gives x = 0.  Fills *result (host memory) and returns
 * its status.  Synchronises `stream` once at the end.
 */
int gbpcg_pcg_solve(const gbpcg_grid *grid, const void *b, void *x, const gbpcg_opts *opts,
                    gbpcg_result *result, gbpcg_stream stream);

/*
 * Many independent problems, each the Jacobi-PCG solve of gbpcg_pcg_solve
 * (Sec. VII), in one launch.  grids[i], b[i], x[i] (DEVICE pointers,
 * opts->io_dtype) describe problem i; storage is F32; results[i] receives
 * problem i's outcome (time_ms is the batch's).  The workspace
 * (gbpcg_workspace_size_batched) holds every problem's scratch.  Returns
 * GBPCG_OK when all problems converged, else the first other status.
 *
 * Up to 4096 constant-coefficient grids with nx a multiple of 4 (and at most
 * 4096 tiles each) run as ONE persistent
 * kernel (a cooperative launch of as many CTAs as the GPU holds, inside a
 * cached one-node CUDA graph): every problem runs its own sequence of phases
 * (pass A, pass B, and a flush and an FP64 residual for each residual
 * replacement), any CTA claiming any available work item (a tile of z
 * planes, or a run of rows) of any unfinished problem; the CTA that
 * completes a phase takes the problem's scalar step and opens its next
 * phase.  Setup and finalize are phases of all problems at once between
 * grid barriers.  Every wait is bounded: if one gives up, the unfinished
 * problems report GBPCG_TIMEOUT.  result.pass_launches = {1, phases run
 * over all problems (2 per iteration and 2 per replacement)},
 * pass_ctas[0] = the tile configuration (0: 64x16, 1: 128x8, 2: 32x32):
 * opts->tile_cfg = c + 1 selects configuration c, else
 * GBPCG_FLAG_AUTOTUNE times the three and keeps the fastest per set of
 * shapes, else 64x16.  Otherwise (block coefficients, or GBPCG_FLAG_BATCH_GRAPH) each
 * problem's whole solve is a branch of one CUDA graph with its own
 * device-driven loop, tiles per shape from the autotuner.
 */
int gbpcg_workspace_size_batched(int32_t nprob, const gbpcg_grid *grids, const gbpcg_opts *opts,
                                 size_t *bytes);
int gbpcg_pcg_solve_batched(int32_t nprob, const gbpcg_grid *grids, const void *const *b, void *const *x,
                            const gbpcg_opts *opts, gbpcg_result *results, gbpcg_stream stream);

/* ------------------------------------------------------------------------
 * General sparse matrices in Sliced-ELL form (SELL-32): the format the
 * paper's H100 comparator stores the seven-point operator in (Sec. VII-A,
 * cuSPARSE Sliced ELL), and the "more general sparse matrix
 * representations" its conclusion names.  Rows are grouped in slices of 32
 * consecutive rows; slice s holds w_s = (slice_ptr[s+1] - slice_ptr[s]) / 32
 * entries per row, w_s the slice's longest row, stored column-major within
 * the slice: entry j of row 32 s + l is at slice_ptr[s] + 32 j + l.  Rows
 * shorter than w_s are padded with value 0 and their own row as column.
 * slice_ptr has ceil(n / 32) + 1 entries (slice_ptr[0] = 0); col are 32-bit
 * column indices; inv_diag is the Jacobi preconditioner D^-1.  All arrays
 * are DEVICE arrays owned by the caller.
 * ---------------------------------------------------------------------- */
typedef struct gbpcg_sell {
    int64_t n;                  /* rows = columns, 1 .. 2^31 - 1 */
    int32_t slice;              /* rows per slice: 32 */
    const int64_t *slice_ptr;   /* ceil(n / 32) + 1 */
    const int32_t *col;         /* slice_ptr[last] entries */
    const float *val;           /* slice_ptr[last] entries */
    const float *inv_diag;      /* n */
} gbpcg_sell;

/* SELL layout of the seven-point operator of `grid` (the matrix of
 * gbpcg_stencil_apply, block coefficients included): *nnz_stored receives
 * the stored entries (padding included); slice_ptr (DEVICE, may be NULL for
 * a size query) receives the slice offsets.  Computed on the host;
 * synchronises `stream` when it copies slice_ptr. */
int gbpcg_sell_stencil_layout(const gbpcg_grid *grid, int64_t *slice_ptr, int64_t *nnz_stored,
                              gbpcg_stream stream);
/* Fills col, val, inv_diag (DEVICE) of that operator: each row's entries in
 * column order (z-1, y-1, x-1, centre, x+1, y+1, z+1), absent neighbours
 * skipped; the same FP32 face weights as the stencil kernels. */
int gbpcg_sell_from_stencil(const gbpcg_grid *grid, const int64_t *slice_ptr, int32_t *col, float *val,
                            float *inv_diag, gbpcg_stream stream);
/* SELL layout of a CSR matrix (row_ptr: DEVICE, n + 1 entries): as
 * gbpcg_sell_stencil_layout.  Reads row_ptr back to the host; synchronises. */
int gbpcg_sell_csr_layout(int64_t n, const int64_t *row_ptr, int64_t *slice_ptr, int64_t *nnz_stored,
                          gbpcg_stream stream);
/* CSR (DEVICE row_ptr, csr_col, csr_val) -> SELL col, val and inv_diag (1 /
 * the diagonal entry; 0 for a row without a non-zero diagonal). */
int gbpcg_sell_from_csr(int64_t n, const int64_t *row_ptr, const int32_t *csr_col, const float *csr_val,
                        const int64_t *slice_ptr, int32_t *col, float *val, float *inv_diag, gbpcg_stream stream);
/* y = A x, FP32 (DEVICE x, y of n elements, distinct). */
int gbpcg_sell_spmv(const gbpcg_sell *matrix, const float *x, float *y, gbpcg_stream stream);
/* Bytes of workspace gbpcg_sell_pcg_solve needs. */
int gbpcg_sell_workspace_size(const gbpcg_sell *matrix, size_t *bytes);
/*
 * Jacobi-PCG (Sec. VII's iteration) for A x = b with A in SELL form, A
 * symmetric positive definite.  b (read), x (initial guess in, solution
 * out): DEVICE FP64 arrays of n elements; opts: io_dtype F64, storage F32,
 * Jacobi, no flags, tol and maxit as for gbpcg_pcg_solve, workspace of
 * gbpcg_sell_workspace_size bytes (256-byte aligned).  Per iteration three
 * kernels (q = A p with p.q; x += alpha p in FP64, r -= alpha q with r.r and
 * r.z; p = D^-1 r + beta p), the scalars on the device, the loop one CUDA
 * graph.  The residual is replaced by b - A x computed in FP64 when it has
 * dropped two decades since the last replacement and when it meets the
 * tolerance, so convergence is decided on a true residual.  Fills *result
 * (rel_res_true: FP64 ||b - A x|| / ||b||); synchronises `stream`.
 */
int gbpcg_sell_pcg_solve(const gbpcg_sell *matrix, const double *b, double *x, const gbpcg_opts *opts,
                         gbpcg_result *result, gbpcg_stream stream);

/*
 * Autotuner (no counterpart in the paper; the paper hard-codes its tile
 * layout, Sec. VI-A): times every tile configuration that fits the grid
 * over a short solve of A x = b from x = 0 (x kept in workspace scratch, b
 * only read), stores the fastest in the process-wide cache used by
 * GBPCG_FLAG_AUTOTUNE and returns it as a gbpcg_opts.tile_cfg code, with the
 * mean time of one iteration in *us_per_iter (may be NULL).  The workspace
 * must be gbpcg_workspace_size() of opts with GBPCG_FLAG_AUTOTUNE set.
 * gbpcg_autotune_record seeds the cache with a code found earlier (e.g. read
 * back from a file).
 */
int gbpcg_autotune(const gbpcg_grid *grid, const gbpcg_opts *opts, const void *b, int32_t *tile_cfg,
                   double *us_per_iter, gbpcg_stream stream);
int gbpcg_autotune_record(const gbpcg_grid *grid, const gbpcg_opts *opts, int32_t tile_cfg);

/* ------------------------------------------------------------------------
 * Geometric multigrid preconditioner (the paper's conclusion names multigrid
 * solvers as future work; it gives no design).  Aggregation hierarchy: coarse
 * cell I owns the 2 x 2 x 2 fine cells 2I + {0,1}^3, P copies a coarse value
 * to them, the coarse operator is the Galerkin product P^T A P (again a
 * seven-point operator: a coarse face carries the sum of the four fine face
 * weights across it).  Levels are added while every size is even and stays
 * >= 4 (at most 8 levels); the coarsest level must hold <= 32768 cells.
 * V-cycle z = M r, omega = 0.9, sigma = 1.5:
 *   u = omega D^-1 f;  e = V-cycle(P^T (f - A u));  u' = u + sigma P e;
 *   result u' + omega D^-1 (f - A u');  coarsest: 24 damped Jacobi sweeps.
 * M is symmetric positive definite, so plain PCG applies.  Grids: nx a
 * multiple of 4; the operator of gbpcg_stencil_apply (block coefficients
 * included).
 * ---------------------------------------------------------------------- */

/* Workspace bytes of gbpcg_mg_vcycle and gbpcg_mg_pcg_solve for a grid. */
int gbpcg_mg_workspace_size(const gbpcg_grid *grid, size_t *bytes);

/* z = M r, one V-cycle (the hierarchy is built in the call): r, z DEVICE
 * FP32 (nz, ny, nx), distinct; *levels (may be NULL) receives the number of
 * levels.  Workspace: DEVICE, gbpcg_mg_workspace_size bytes, 256-byte
 * aligned. */
int gbpcg_mg_vcycle(const gbpcg_grid *grid, const float *r, float *z, void *workspace, size_t workspace_bytes,
                    int32_t *levels, gbpcg_stream stream);

/*
 * PCG (Sec. VII's iteration) with z = M r for A x = b.  b (read) and x
 * (initial guess in, solution out): DEVICE FP64, 16-byte aligned.  opts:
 * precond = GBPCG_PRECOND_MG, io_dtype F64, storage F32, no flags, tol and
 * maxit as for gbpcg_pcg_solve, workspace of gbpcg_mg_workspace_size bytes.
 * Vectors FP32, scalars FP64, the updates of x deferred into a correction
 * vector and residual replacements in FP64 as in gbpcg_pcg_solve; the whole
 * loop is one CUDA graph (the scalars stay on the device).  Fills *result
 * (pass_launches[0] = levels of the hierarchy) and synchronises `stream`.
 */
int gbpcg_mg_pcg_solve(const gbpcg_grid *grid, const double *b, double *x, const gbpcg_opts *opts,
                       gbpcg_result *result, gbpcg_stream stream);

/* ------------------------------------------------------------------------
 * Learned preconditioner (no counterpart in the paper, which preconditions
 * with Jacobi only): z = N(r), a three-level 3D U-net of 3x3x3
 * convolutions without bias, used inside flexible CG.
 *
 *   c1 (2->16), c2 (16->16) = e0                       full resolution
 *   2x2x2 average pool, c3 (16->32), c4 (32->32) = e1  half
 *   2x2x2 average pool, c5 (32->64), c6 (64->64)       quarter
 *   nearest upsample, concat [up, e1] -> c7 (96->32)   half
 *   nearest upsample, concat [up, e0] -> c8 (48->16)   full
 *   c9 (16->1)
 * ReLU after every convolution but c9.  The network works on the
 * Jacobi-scaled system D^{-1/2} A D^{-1/2}, D the operator's diagonal (the
 * sum of the six face weights k_f / h_d^2 at each point): with
 * s = D^{-1/2} r and rms(s) = ||s|| / sqrt(nx ny nz), the input channels are
 * s / rms(s) and log k of the voxel's coefficient block (0 for the Poisson
 * operator), and the last layer's output u becomes
 * z = rms(s) D^{-1/2} u.  N is therefore positively homogeneous:
 * N(a r) = a N(r) for a > 0.  Weights that pass s / rms(s) through
 * unchanged give z = D^{-1} r, the Jacobi preconditioner.
 *
 * Layouts: activations channels-last, (nz, ny, nx, C), BF16; a layer's
 * weights (Co, 27, Ci) with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) reading
 * in[z+dz, y+dy, x+dx]; zero padding.  The FP32 master weights of the whole
 * network are one array of GBPCG_NN_NUM_WEIGHTS floats, layers c1..c9 in
 * order.  Convolutions with 16 or more input and output channels run on the
 * tensor cores (tcgen05, BF16 operands, FP32 accumulation).
 *
 * Grids: each size a multiple of 4 such that every level's voxels split
 * into 128-voxel tiles of whole x-rows or whole planes (any multiple of 512,
 * or powers of two >= 32).  Workspaces: DEVICE, 256-byte aligned, from the
 * matching *_workspace_size; a bounded wait that gives up inside a
 * convolution sets an error word in the workspace (see gbpcg_nn_status),
 * and that call's output is then unspecified (flexible CG checks the word
 * every iteration and falls back to Jacobi).
 * ---------------------------------------------------------------------- */

#define GBPCG_NN_NUM_WEIGHTS 319248

/* Workspace bytes of the gbpcg_conv3_* calls for one shape. */
int gbpcg_conv3_workspace_size(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, size_t *bytes);

/*
 * y[v, o] = sum_{t, i} w[o, t, i] x[v + off(t), i]  (then max(y, 0) when
 * relu != 0).  x: DEVICE BF16 (nz, ny, nx, ci); w: DEVICE BF16 (co, 27, ci);
 * y: DEVICE FP32 (nz, ny, nx, co).  Supported: ci a multiple of 16 with co
 * in {16, 32, 48, 64, 96} (tensor cores), or (ci, co) in {(2, 16), (16, 1),
 * (1, 16)} (CUDA cores).  Arrays 16-byte aligned.
 */
int gbpcg_conv3_forward(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *x, const void *w,
                        float *y, int32_t relu, void *workspace, size_t workspace_bytes, gbpcg_stream stream);

/*
 * gx[v, i] = sum_{t, o} w[o, t, i] gy[v - off(t), o]: the adjoint of
 * gbpcg_conv3_forward in x (computed as a forward convolution with mirrored
 * taps and transposed channels).  gy: DEVICE BF16 (.., co); w: DEVICE BF16
 * (co, 27, ci); gx: DEVICE FP32 (.., ci).  Supported when the forward shape
 * with ci and co exchanged is.
 */
int gbpcg_conv3_backward_data(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *gy,
                              const void *w, float *gx, void *workspace, size_t workspace_bytes,
                              gbpcg_stream stream);

/*
 * gw[o, t, i] = sum_v gy[v, o] x[v + off(t), i]: the gradient in w of a loss
 * that depends on y = conv(x, w) through gy = dL/dy.  x: DEVICE BF16
 * (.., ci); gy: DEVICE BF16 (.., co); gw: DEVICE FP32 (co, 27, ci),
 * overwritten.  ci in {1, 2} or a multiple of 8, co = 1 or a multiple of 8;
 * the sum is taken in a fixed order (bitwise reproducible).
 */
int gbpcg_conv3_backward_weight(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *x,
                                const void *gy, float *gw, void *workspace, size_t workspace_bytes,
                                gbpcg_stream stream);

/* Workspace bytes of the network for a grid: inference (training = 0) or
 * forward + backward (training != 0).  A training workspace serves every
 * gbpcg_nn_* call. */
int gbpcg_nn_workspace_size(int32_t nx, int32_t ny, int32_t nz, int32_t training, size_t *bytes);

/* Tensors that gbpcg_nn_forward and gbpcg_nn_backward leave in a workspace,
 * for inspection (gbpcg_nn_tensor_info).  Level 0 is the grid, level 1 and
 * 2 halve every size once and twice; a tensor of C channels is stored
 * channels-last, (nz, ny, nx, C) of its level. */
enum gbpcg_nn_tensor {
    GBPCG_NN_T_XIN = 0,  /* BF16, 2: network input (s / rms(s), log k) */
    GBPCG_NN_T_A1,       /* BF16, 16: relu(c1) */
    GBPCG_NN_T_K8,       /* BF16, 48: c8 input, up(a7) in 0..31, e0 = relu(c2) in 32..47 */
    GBPCG_NN_T_P1,       /* BF16, 16: pool(e0), level 1 */
    GBPCG_NN_T_A3,       /* BF16, 32: relu(c3), level 1 */
    GBPCG_NN_T_K7,       /* BF16, 96: c7 input, up(a6) in 0..63, e1 = relu(c4) in 64..95, level 1 */
    GBPCG_NN_T_P2,       /* BF16, 32: pool(e1), level 2 */
    GBPCG_NN_T_A5,       /* BF16, 64: relu(c5), level 2 */
    GBPCG_NN_T_A6,       /* BF16, 64: relu(c6), level 2 */
    GBPCG_NN_T_A7,       /* BF16, 32: relu(c7), level 1 */
    GBPCG_NN_T_A8,       /* BF16, 16: relu(c8) */
    GBPCG_NN_T_DSC,      /* F32, 1: D^{-1/2} */
    GBPCG_NN_T_SR,       /* F32, 1: s = D^{-1/2} r */
    GBPCG_NN_T_SCALE,    /* F64 scalar (level -1): rms(s) */
    /* training workspaces only (gbpcg_nn_backward) */
    GBPCG_NN_T_GOUT,     /* BF16, 1: dL/du of the last layer's output u (gz rms(s) D^{-1/2}) */
    GBPCG_NN_T_GA8,      /* BF16, 16: dL/d(c8 output), ReLU mask applied */
    GBPCG_NN_T_GK8,      /* F32, 48: dL/d(c8 input) */
    GBPCG_NN_T_GA7,      /* BF16, 32: dL/d(c7 output), masked, level 1 */
    GBPCG_NN_T_GK7,      /* F32, 96: dL/d(c7 input), level 1 */
    GBPCG_NN_T_GA6,      /* BF16, 64: dL/d(c6 output), masked, level 2 */
    GBPCG_NN_T_GA5,      /* BF16, 64: dL/d(c5 output), masked, level 2 */
    GBPCG_NN_T_T5,       /* F32, 32: dL/d(c5 input), level 2 */
    GBPCG_NN_T_GE1B,     /* BF16, 32: dL/d(c4 output) (skip + pooled path), masked, level 1 */
    GBPCG_NN_T_GA3,      /* BF16, 32: dL/d(c3 output), masked, level 1 */
    GBPCG_NN_T_T3,       /* F32, 16: dL/d(c3 input), level 1 */
    GBPCG_NN_T_GE0B,     /* BF16, 16: dL/d(c2 output) (skip + pooled path), masked */
    GBPCG_NN_T_GA1,      /* BF16, 16: dL/d(c1 output), masked */
    GBPCG_NN_T_COUNT
};

/*
 * Where tensor `index` (gbpcg_nn_tensor) lives in a network workspace of
 * this grid (training != 0: a training workspace): byte offset from the
 * workspace base, element type (gbpcg_dtype), channels per voxel and grid
 * level.  Host-only; launches nothing.  Tensors marked "training" need
 * training != 0 (else GBPCG_ERR_ARG).  A tensor holds what the last
 * gbpcg_nn_forward / gbpcg_nn_backward on that workspace left there.
 */
int gbpcg_nn_tensor_info(int32_t nx, int32_t ny, int32_t nz, int32_t training, int32_t index, size_t *offset,
                         int32_t *dtype, int32_t *channels, int32_t *level);

/*
 * z = N(r).  w: DEVICE FP32 master weights (GBPCG_NN_NUM_WEIGHTS); r, z:
 * DEVICE FP32 (nz, ny, nx); grid->k_block supplies the log k channel.  The
 * activations stay in the workspace for gbpcg_nn_backward.
 */
int gbpcg_nn_forward(const gbpcg_grid *grid, const float *w, const float *r, float *z, void *workspace,
                     size_t workspace_bytes, gbpcg_stream stream);

/*
 * gw = dL/dw for every weight (DEVICE FP32, GBPCG_NN_NUM_WEIGHTS,
 * overwritten), given gz = dL/dz (DEVICE FP32) at the z of the last
 * gbpcg_nn_forward on this (training) workspace.  The normalisation by
 * rms(r) is treated as a constant.
 */
int gbpcg_nn_backward(const gbpcg_grid *grid, const float *gz, float *gw, void *workspace, size_t workspace_bytes,
                      gbpcg_stream stream);

/*
 * Loss of one training pair (r, e = A^{-1} r): for z.Ae >= 0 the relative
 * A-norm error of the best multiple of z (a preconditioned step's line
 * search chooses that multiple, so only the direction of z matters), mirrored
 * for z.Ae < 0 so that only positive multiples of e reach the minimum 0.
 * With a = z.Ae, c = z.Az, E = e.Ae and A the grid's operator:
 *   loss = 1/2 (1 - a |a| / (c E))   (= 1/2 ||(a/c) z - e||_A^2 / E, a >= 0),
 *   gz = dloss/dz = (|a| / (c E)) ((a/c) A z - A e).
 * z, e, gz: DEVICE FP32; loss: DEVICE double (may be NULL).  Training
 * workspace.
 */
int gbpcg_nn_loss(const gbpcg_grid *grid, const float *z, const float *e, float *gz, double *loss,
                  void *workspace, size_t workspace_bytes, gbpcg_stream stream);

/* Adam with bias correction on n FP32 weights (DEVICE w, g, m, v; step >= 1
 * counts from 1). */
int gbpcg_nn_adam(int64_t n, float *w, const float *g, float *m, float *v, int32_t step, double lr, double beta1,
                  double beta2, double eps, gbpcg_stream stream);

/*
 * One training step on one pair: z = N(r); loss and gz as gbpcg_nn_loss;
 * gw = dL/dw; Adam (beta 0.9 / 0.999, eps 1e-8) updates w, m, v in place.
 * z, gz, gw: DEVICE scratch that receives those values; loss: DEVICE double.
 */
int gbpcg_nn_train_step(const gbpcg_grid *grid, float *w, float *m, float *v, int32_t step, double lr,
                        const float *r, const float *e, float *z, float *gz, float *gw, double *loss,
                        void *workspace, size_t workspace_bytes, gbpcg_stream stream);

/* Workspace bytes of gbpcg_fcg_solve (opts as for the solve). */
int gbpcg_fcg_workspace_size(const gbpcg_grid *grid, const gbpcg_opts *opts, size_t *bytes);

/*
 * Flexible CG with truncation m = opts->fcg_m (Notay 2000: p_k = z_k minus
 * its A-projections on the last m directions, alpha_k = p_k.r_k / p_k.Ap_k;
 * m = 1 is the beta = z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k) form) for A x = b
 * with the learned preconditioner z = N(r), N given by the DEVICE FP32
 * weights w.  opts: precond = GBPCG_PRECOND_LEARNED,
 * io_dtype = F64 (b read, x initial guess in / solution out, DEVICE,
 * 16-byte aligned), storage = F32, no flags; tol and maxit as in
 * gbpcg_pcg_solve (maxit counts every A.p product, fallback included).
 * Vectors are FP32, x and the scalars FP64; at recursive convergence the
 * true residual is recomputed in FP64 and, if it misses tol, replaces r
 * (FCG restarts).  Descent check: if p.Ap <= 0, r.z <= 0, a scalar is not
 * finite, the residual grows 10x over 5 iterations, or a convolution timed
 * out, the solve continues from the current x with Jacobi PCG and returns
 * GBPCG_FALLBACK_USED on convergence.  The host reads the scalars once per
 * iteration.  result: iters (all), pass_launches[0] = FCG iterations,
 * pass_launches[1] = Jacobi fallback iterations, pass_ms[0] = time in the
 * network, pass_ms[1] = the rest, replacements.
 */
int gbpcg_fcg_solve(const gbpcg_grid *grid, const float *w, const void *b, void *x, const gbpcg_opts *opts,
                    gbpcg_result *result, gbpcg_stream stream);

/* Synchronises `stream`, then returns GBPCG_TIMEOUT (and clears the word) if
 * a convolution in this workspace gave up a bounded wait since the last
 * check, else GBPCG_OK. */
int gbpcg_nn_status(void *workspace, gbpcg_stream stream);

/*
 * Self-test of the bounded waits (no counterpart in the paper).  Every kernel
 * of the library that waits on an asynchronous copy or MMA polls its mbarrier
 * at most 2^18 times (about one second on GB300) and then reports
 * GBPCG_TIMEOUT instead of hanging.  This call runs that wait in one CTA on a
 * barrier that completes (arrive != 0) or never does (arrive == 0), with at
 * most `polls` polls (1 .. 2^18), and
 * returns GBPCG_OK or GBPCG_TIMEOUT as the device reported it; *ms (may be
 * NULL) receives the kernel's duration.  scratch: 16 bytes of DEVICE memory,
 * 16-byte aligned.  Synchronises `stream`.
 */
int gbpcg_wait_selftest(int32_t arrive, uint32_t polls, void *scratch, double *ms, gbpcg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GBPCG_H */
