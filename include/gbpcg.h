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
    GBPCG_PRECOND_JACOBI = 0
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
                                 bracketed by CUDA events; fills gbpcg_result.pass_ms */
#define GBPCG_FLAG_AUTOTUNE 4u /* batched solves: pick each shape's tile configuration by timing
                                  (cached per shape in the process); the workspace grows by a
                                  scratch x per problem */

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
    double inner_tol;      /* refinement (16-bit storage): relative tolerance of each inner solve */
    int32_t max_outer;     /* refinement: maximum outer FP64 steps */
    int32_t reserved1;
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
 * device looks up that array's device address, so make that first call
 * outside any stream capture.  n is limited to 2^30 elements; larger n
 * returns GBPCG_ERR_ARG.  All calls share the one array: calls that may
 * overlap on the GPU (different streams, or different host threads without
 * ordering) race and must be serialised by the caller.  x, y: DEVICE arrays
 * of n elements of dtype; result: DEVICE double; n = 0 writes 0.
 */
int gbpcg_dot_noalloc(int64_t n, int32_t dtype, const void *x, const void *y, double *result,
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
 * decade of residual reduction and at recursive convergence, flushed into x
 * while the residual is replaced by b - A x computed in FP64 (reliable
 * updates), so the returned x meets the tolerance in its true residual.
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
 * Many independent problems (BASELINE config 3) solved as one CUDA graph:
 * each problem's whole solve (its own device-driven loop, as in
 * gbpcg_pcg_solve) is a branch of one graph, so one launch runs them all
 * concurrently and no problem waits on another's convergence.  grids[i],
 * b[i], x[i] (DEVICE pointers, opts->io_dtype) describe problem i; storage
 * is F32; results[i] receives problem i's outcome (time_ms is the batch's).
 * The workspace (gbpcg_workspace_size_batched) holds every problem's
 * scratch.  Returns GBPCG_OK when all problems converged, else the first
 * other status.  The instantiated graph is cached per argument set.
 */
int gbpcg_workspace_size_batched(int32_t nprob, const gbpcg_grid *grids, const gbpcg_opts *opts,
                                 size_t *bytes);
int gbpcg_pcg_solve_batched(int32_t nprob, const gbpcg_grid *grids, const void *const *b, void *const *x,
                            const gbpcg_opts *opts, gbpcg_result *results, gbpcg_stream stream);

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

#ifdef __cplusplus
}
#endif

#endif /* GBPCG_H */
