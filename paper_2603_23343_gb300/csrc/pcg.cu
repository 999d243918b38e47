// C ABI of the solver (Sec. VII): argument checks, host staging, the graph
// cache, and mixed-precision iterative refinement around 16-bit inner solves.
//
// Refinement (Wilkinson; Moler, J. ACM 14, 1967) with x and b in FP64:
//   r = b - A x (FP64 arithmetic; stored as FP32), s = max |r|
//   stop if ||r||/||b|| <= tol
//   inner: solve (sigma A) d = r / s to inner_tol with BF16/FP16 vectors
//          (sigma = 1 / max_d c_d keeps the operator's entries O(k), r / s
//          keeps the right-hand side O(1): both inside FP16's range)
//   x += sigma s d (FP64)
// The host reads ||r||, ||b|| once per outer step; each inner solve is the
// cached CUDA graph of solver.cuh with 16-bit storage.
#include <cmath>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "solver.cuh"

namespace gb {

// ------------------------------------------------------------ graph cache --

namespace {
struct SolveGraph {
    SolveKey key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_cache_mu;
std::list<SolveGraph> g_cache;  // most recently used first
constexpr size_t kCacheMax = 32;
}  // namespace

cudaGraphExec_t graph_cache_find(const SolveKey &key) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
        if (it->key == key) {
            g_cache.splice(g_cache.begin(), g_cache, it);
            return g_cache.front().exec;
        }
    return nullptr;
}

cudaGraphExec_t graph_cache_put(const SolveKey &key, cudaGraph_t graph, cudaGraphExec_t exec) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto &e : g_cache)
        if (e.key == key) {  // another thread built it first
            cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            return e.exec;
        }
    SolveGraph sg;
    sg.key = key;
    sg.graph = graph;
    sg.exec = exec;
    g_cache.push_front(sg);
    while (g_cache.size() > kCacheMax) {
        cudaGraphExecDestroy(g_cache.back().exec);
        cudaGraphDestroy(g_cache.back().graph);
        g_cache.pop_back();
    }
    return exec;
}

// ------------------------------------------------------------ refinement --

struct __align__(16) OuterState {
    double rr, bb;                 // ||b - A x||^2, ||b||^2 (FP64)
    unsigned long long rmax_bits;  // max |r| as the bit pattern of a non-negative double
    double bscale;                 // 1 / max |r|: scales the inner right-hand side
    double corr;                   // sigma * max |r|: scales the inner solution into x
    double sigma;
    unsigned int ticket;
    unsigned int pad;
    double applied;                // the corr of the last applied update (to undo it)
};

// r = b - A x in FP64 (unscaled operator), r32 = (float) r; sums ||r||^2,
// ||b||^2 and max |r|; the last block derives the inner scalings.
template <bool BLOCK>
__global__ void __launch_bounds__(256)
    outer_residual_kernel(int nx, int ny, int nz, const double *__restrict__ x, const double *__restrict__ b,
                          float *r32, double cx, double cy, double cz, const float *__restrict__ kb,
                          int kbx, int kby, int kbz, const double *__restrict__ tab64, OuterState *os,
                          double *partials) {
    const Coef64 cf{cx, cy, cz, kb, kbx, kby, kbz};
    double w[6];
    face_weights64<false>(w, 0, 0, 0, nx, ny, nz, cf);
    double rr = 0.0, bb = 0.0, mx = 0.0;
    const int rows = ny * nz;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = row % ny, k = row / ny;
        const int64_t base = (int64_t)row * nx;
        for (int i = threadIdx.x; i < nx; i += 256) {
            const int64_t g = base + i;
            if (BLOCK) face_weights64_tab(w, i, j, k, nx, ny, tab64, cf);
            const double ax = apply64<BLOCK>(load_nbr64(x, g, i, j, k, nx, ny, nz), w);
            const double bv = b[g];
            const double r = bv - ax;
            r32[g] = (float)r;
            rr = fma(r, r, rr);
            bb = fma(bv, bv, bb);
            mx = fmax(mx, fabs(r));
        }
    }
    __shared__ double red[8][3];
    rr = warp_sum(rr);
    bb = warp_sum(bb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = rr;
        red[threadIdx.x >> 5][1] = bb;
        red[threadIdx.x >> 5][2] = mx;
    }
    __syncthreads();
    double part[2] = {0.0, 0.0}, tot[2];
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < 8; ++w) {
            part[0] += red[w][0];
            part[1] += red[w][1];
            m = fmax(m, red[w][2]);
        }
        // max of non-negative doubles = max of their bit patterns (published before the ticket)
        atomicMax(&os->rmax_bits, (unsigned long long)__double_as_longlong(m));
    }
    if (grid_sum_last<2, 256>(part, partials, &os->ticket, tot) && threadIdx.x == 0) {
        const double rmax = __longlong_as_double((long long)atomicAdd(&os->rmax_bits, 0ull));
        os->rr = tot[0];
        os->bb = tot[1];
        os->bscale = rmax > 0.0 ? 1.0 / rmax : 1.0;
        os->corr = os->sigma * rmax;
    }
}

// x += sign * c * din (FP64); c = corr (apply) or the last applied corr (undo)
__global__ void refine_update_kernel(double *x, const float *din, OuterState *os, int64_t n, int undo) {
    const double c = undo ? -os->applied : os->corr;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nth) x[i] = fma(c, (double)din[i], x[i]);
}

__global__ void zero_f64_kernel(double *x, int64_t n) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += nth) x[i] = 0.0;
}

struct RefineLayout {
    size_t outer, partials, r32, din, tab64, inner, total;
    WsLayout in;
};

static RefineLayout refine_layout(const gbpcg_grid &g, const gbpcg_opts &o) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    RefineLayout r;
    size_t off = 0;
    r.outer = off; off += 256;
    r.partials = off; off += round256(sizeof(double) * 2 * 8192);
    r.r32 = off; off += round256(n * 4);
    r.din = off; off += round256(n * 4);
    r.tab64 = off; off += round256((size_t)block_count(g) * kTab64 * sizeof(double));
    r.inner = off;
    r.in = ws_layout_n(n, o.storage, GBPCG_F32, false, block_count(g));
    off += r.in.total;
    if (o.flags & GBPCG_FLAG_HOST_IO) off += 2 * round256(n * 8);  // staging of b and x (FP64)
    r.total = off;
    return r;
}

static bool refine_mode(const gbpcg_opts &o) { return o.storage == GBPCG_BF16 || o.storage == GBPCG_F16; }

static size_t workspace_total(const gbpcg_grid &g, const gbpcg_opts &o) {
    if (refine_mode(o)) return refine_layout(g, o).total;
    if (o.flags & GBPCG_FLAG_SPLIT) return split_workspace_size(g);
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    size_t t = ws_layout_n(n, o.storage, o.io_dtype, o.flags & GBPCG_FLAG_HOST_IO, block_count(g)).total;
    if (o.flags & GBPCG_FLAG_AUTOTUNE) t += round256(n * dtype_size(o.io_dtype));  // tuner's scratch x
    return t;
}

static int check_opts(const gbpcg_opts *o) {
    if (!o) return fail_arg("opts is NULL");
    if (o->storage != GBPCG_F32 && o->storage != GBPCG_BF16 && o->storage != GBPCG_F16)
        return fail_arg("storage dtype must be F32, BF16 or F16");
    if (o->io_dtype != GBPCG_F32 && o->io_dtype != GBPCG_F64) return fail_arg("io dtype must be F32 or F64");
    if (refine_mode(*o) && o->io_dtype != GBPCG_F64)
        return fail_arg("16-bit storage (iterative refinement) needs FP64 b and x");
    if (refine_mode(*o) && !(o->inner_tol == 0.0 || (o->inner_tol > 0.0 && o->inner_tol < 1.0)))
        return fail_arg("inner_tol must be 0 (default) or in (0, 1)");
    if (refine_mode(*o) && o->max_outer < 0) return fail_arg("max_outer must be >= 0");
    if (o->precond != GBPCG_PRECOND_JACOBI) return fail_arg("unknown preconditioner");
    if (!(o->tol >= 0.0)) return fail_arg("tol must be >= 0");
    if (o->maxit < 0) return fail_arg("maxit must be >= 0");
    const uint32_t modes = o->flags & (GBPCG_FLAG_PROFILE | GBPCG_FLAG_HOST_LOOP | GBPCG_FLAG_SPLIT);
    if (modes & (modes - 1)) return fail_arg("PROFILE, HOST_LOOP and SPLIT exclude one another");
    if ((o->flags & (GBPCG_FLAG_HOST_LOOP | GBPCG_FLAG_SPLIT)) && refine_mode(*o))
        return fail_arg("HOST_LOOP and SPLIT take FP32 storage");
    if ((o->flags & GBPCG_FLAG_SPLIT) && (o->io_dtype != GBPCG_F32 || (o->flags & GBPCG_FLAG_HOST_IO)))
        return fail_arg("SPLIT takes FP32 device b and x");
    if (o->tile_cfg < 0 || (o->tile_cfg & 0xff) > NUM_CFG || ((o->tile_cfg >> 8) & 0xff) > NUM_CFG ||
        (o->tile_cfg >> 16))
        return fail_arg("tile_cfg selects unknown tile configurations");
    return GBPCG_OK;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Tile configurations of pass A and pass B: explicit (opts->tile_cfg) or
// the default for the grid's width (from a sweep of all pairs at 256^3 on
// GB300: every shape lands within a few percent; whole-row tiles for pass A
// and 128x8 for pass B are at the front).
static void pick_cfgs(const gbpcg_grid &g, const gbpcg_opts &o, int *ca, int *cb) {
    const int narrow = g.nx <= 32 ? CFG_32x16 : g.nx <= 64 ? CFG_64x16 : -1;
    const int def_a = narrow >= 0 ? narrow : (g.nx > 192 && g.nx <= 256) ? CFG_256x4 : CFG_128x8;
    const int def_b = narrow >= 0 ? narrow : CFG_128x8;
    const int ea = o.tile_cfg & 0xff, eb = (o.tile_cfg >> 8) & 0xff;
    *ca = ea ? ea - 1 : def_a;
    *cb = eb ? eb - 1 : def_b;
}

// Reads the device scalars back (and x, for host buffers), fills *result.
static int finish_solve(const SolveState *st_dev, void *x, const void *xd, bool x_host, size_t io_bytes,
                        cudaEvent_t e0, cudaEvent_t e1, gbpcg_result *result, cudaStream_t s) {
    SolveState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, st_dev, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    if (x_host) GB_CUDA(cudaMemcpyAsync(x, xd, io_bytes, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    result->iters = hs.it;
    result->status = hs.status;
    result->rel_res_recursive = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
    result->rel_res_true = hs.bb_true > 0 ? sqrt(hs.rr_true / hs.bb_true) : 0.0;
    result->time_ms = ms;
    result->replacements = hs.n_replace;
    if (hs.status == GBPCG_TIMEOUT) set_error("a bounded device wait timed out during the solve");
    return hs.status;
}

// Outer FP64 refinement loop; b and x are FP64 device arrays.  An outer step
// whose correction does not reduce ||b - A x|| is undone and ends the solve
// (status NOT_CONVERGED): the inner solves have stopped helping.
static int refine_solve(const gbpcg_grid &g, const double *b, double *x, const gbpcg_opts *o, char *ws,
                        const RefineLayout &R, int cfg_a, int cfg_b, bool tma, gbpcg_result *result, cudaStream_t s) {
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    auto cc = [](int m) { double h = 1.0 / (m + 1); return 1.0 / (h * h); };
    const double cmax = std::max(cc(g.nx), std::max(cc(g.ny), cc(g.nz)));
    const float sigma = (float)(1.0 / cmax);
    OuterState *os = reinterpret_cast<OuterState *>(ws + R.outer);
    double *partials = reinterpret_cast<double *>(ws + R.partials);
    float *r32 = reinterpret_cast<float *>(ws + R.r32);
    float *din = reinterpret_cast<float *>(ws + R.din);
    char *inner_ws = ws + R.inner;
    SolveState *ist = reinterpret_cast<SolveState *>(inner_ws + R.in.state);
    // default inner tolerance: BF16's 8-bit mantissa stalls short of 1e-2 on ill-conditioned
    // operators (512^3 lognormal k), so it gets 0.1 and more outer steps; FP16 gets 1e-2
    const double inner_tol = o->inner_tol > 0.0 ? o->inner_tol : (o->storage == GBPCG_BF16 ? 0.1 : 1e-2);
    const SolveCall inner{&g, cfg_a, cfg_b, r32, din, inner_ws, R.in, inner_tol, o->maxit, GBPCG_F32, sigma,
                          &os->bscale};
    const unsigned rb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)g.ny * g.nz, device_sm_count() * 8));
    const unsigned eb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, device_sm_count() * 8));
    // FP64 face weights of the unscaled operator for the outer residual (the
    // inner solves keep their own table, of the scaled operator)
    double *tab64 = reinterpret_cast<double *>(ws + R.tab64);
    if (g.k_block) {
        const int nbx = (g.nx + g.kbx - 1) / g.kbx, nby = (g.ny + g.kby - 1) / g.kby, nbz = (g.nz + g.kbz - 1) / g.kbz;
        const int64_t nb = (int64_t)nbx * nby * nbz;
        const Coef64 cf{cc(g.nx), cc(g.ny), cc(g.nz), g.k_block, g.kbx, g.kby, g.kbz};
        build_face_table64<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 4096)), 256, 0, s>>>(
            g.k_block, nbx, nby, nbz, cf, tab64);
        GB_CUDA(cudaGetLastError());
    }
    OuterState init;
    memset(&init, 0, sizeof(init));
    init.sigma = (double)sigma;
    auto launch_outer = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(os, &init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (e) return e;
        if (g.k_block)
            outer_residual_kernel<true><<<rb, 256, 0, s>>>(g.nx, g.ny, g.nz, x, b, r32, cc(g.nx), cc(g.ny),
                                                          cc(g.nz), g.k_block, g.kbx, g.kby, g.kbz, tab64, os,
                                                          partials);
        else
            outer_residual_kernel<false><<<rb, 256, 0, s>>>(g.nx, g.ny, g.nz, x, b, r32, cc(g.nx), cc(g.ny),
                                                           cc(g.nz), nullptr, 1, 1, 1, nullptr, os, partials);
        return cudaGetLastError();
    };

    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    GB_CUDA(cudaEventRecord(e0, s));
    GB_CUDA(launch_outer());
    int steps = 0, total_iters = 0, status = GBPCG_NOT_CONVERGED, replacements = 0;
    double rel = 0.0, rel_prev = 0.0, corr_applied = 0.0;
    bool have_inner = false;
    for (;;) {
        NvtxRange step_range("refinement outer step");
        OuterState ho;
        SolveState hi;
        GB_CUDA(cudaMemcpyAsync(&ho, os, sizeof(ho), cudaMemcpyDeviceToHost, s));
        if (have_inner) GB_CUDA(cudaMemcpyAsync(&hi, ist, sizeof(hi), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        if (have_inner) {
            total_iters += hi.it;
            replacements += hi.n_replace;
            if (hi.status == GBPCG_BREAKDOWN || hi.status == GBPCG_TIMEOUT) {
                status = hi.status;
                break;
            }
        }
        if (ho.bb == 0.0) {
            zero_f64_kernel<<<eb, 256, 0, s>>>(x, n);
            GB_CUDA(cudaGetLastError());
            rel = 0.0;
            status = GBPCG_OK;
            break;
        }
        rel = sqrt(ho.rr / ho.bb);
        if (have_inner && !(rel < rel_prev)) {
            // the last correction did not reduce the residual: take it back and stop
            init.applied = corr_applied;
            GB_CUDA(cudaMemcpyAsync(os, &init, sizeof(init), cudaMemcpyHostToDevice, s));
            refine_update_kernel<<<eb, 256, 0, s>>>(x, din, os, n, 1);
            GB_CUDA(cudaGetLastError());
            GB_CUDA(launch_outer());
            GB_CUDA(cudaMemcpyAsync(&ho, os, sizeof(ho), cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
            rel = sqrt(ho.rr / ho.bb);
            status = GBPCG_NOT_CONVERGED;
            break;
        }
        if (!std::isfinite(rel)) {
            status = GBPCG_BREAKDOWN;
            break;
        }
        if (rel <= o->tol) {
            status = GBPCG_OK;
            break;
        }
        if (steps >= o->max_outer) {
            status = GBPCG_NOT_CONVERGED;
            break;
        }
        // the inner solve starts from d = 0 (din keeps the last correction until
        // here, so a step can be undone)
        GB_CUDA(cudaMemsetAsync(din, 0, (size_t)n * sizeof(float), s));
        int rc;
        if (o->flags & GBPCG_FLAG_PROFILE) {
            // profile mode: the inner solve's kernels one by one, pass times summed over the steps
            gbpcg_result ir;
            memset(&ir, 0, sizeof(ir));
            rc = o->storage == GBPCG_BF16 ? solve_profiled<__nv_bfloat16>(inner, tma, &ir, s)
                                          : solve_profiled<__half>(inner, tma, &ir, s);
            for (int p = 0; p < 2; ++p) {
                result->pass_ms[p] += ir.pass_ms[p];
                result->pass_launches[p] += ir.pass_launches[p];
                result->pass_ctas[p] = ir.pass_ctas[p];
            }
        } else {
            rc = o->storage == GBPCG_BF16 ? solve_launch<__nv_bfloat16>(inner, tma, s)
                                          : solve_launch<__half>(inner, tma, s);
        }
        if (rc) return rc;
        refine_update_kernel<<<eb, 256, 0, s>>>(x, din, os, n, 0);
        GB_CUDA(cudaGetLastError());
        corr_applied = (double)sigma * __builtin_bit_cast(double, ho.rmax_bits);
        rel_prev = rel;
        GB_CUDA(launch_outer());
        have_inner = true;
        steps += 1;
    }
    GB_CUDA(cudaEventRecord(e1, s));
    GB_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    result->iters = total_iters;
    result->status = status;
    result->refine_steps = steps;
    result->replacements = replacements;
    result->rel_res_recursive = rel;
    result->rel_res_true = rel;
    result->time_ms = ms;
    return status;
}

// ------------------------------------------------------------- batches --

namespace {
struct BatchGraph {
    std::vector<SolveKey> keys;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_batch_mu;
std::list<BatchGraph> g_batch_cache;
constexpr size_t kBatchCacheMax = 4;

// Autotuned tile configurations, per (device, shape, coefficient blocks, io type).
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

TuneKey tune_key(const gbpcg_grid &g, const gbpcg_opts &o) {
    int dev = 0;
    cudaGetDevice(&dev);
    return TuneKey(dev, g.nx, g.ny, g.nz, g.k_block ? g.kbx : 0, g.k_block ? g.kby : 0, g.k_block ? g.kbz : 0,
                   o.storage, o.io_dtype);
}
}  // namespace

// Workspace of one problem inside a batch (256-byte aligned pieces); with
// GBPCG_FLAG_AUTOTUNE each piece ends with a scratch x for the tuner.
static size_t batch_piece(const gbpcg_grid &g, const gbpcg_opts &o, WsLayout *L) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    *L = ws_layout_n(n, o.storage, o.io_dtype, false, block_count(g));
    size_t t = L->total;
    if (o.flags & GBPCG_FLAG_AUTOTUNE) t += round256(n * dtype_size(o.io_dtype));
    return round256(t);
}

// Times each tile configuration that fits the grid (the same one for both
// passes) over a short profiled solve from x = 0 into `xs`, and returns the
// fastest as a tile_cfg code.
static int autotune_one(const gbpcg_grid &g, const gbpcg_opts &o, const void *b, void *xs, char *ws,
                        const WsLayout &L, cudaStream_t s, int *code_out, double *us_out) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const bool tma = tma_ok(sizeof(float), g.nx, {ws + L.z, ws + L.p0, ws + L.p1, ws + L.d});
    double best = 1e300;
    int best_code = 0;
    for (int c = 0; c < NUM_CFG; ++c) {
        if (!cfg_fits(c, g.nx)) continue;
        if (cfg_dims(c).tx > 4 * ((g.nx + 3) / 4) + 64) continue;  // tiles far wider than the grid
        GB_CUDA(cudaMemsetAsync(xs, 0, n * dtype_size(o.io_dtype), s));
        const SolveCall call{&g, c, c, b, xs, ws, L, 0.0, 12, o.io_dtype, 1.0f, nullptr};
        gbpcg_result r;
        memset(&r, 0, sizeof(r));
        if (int rc = solve_profiled<float>(call, tma, &r, s)) return rc;
        GB_CUDA(cudaStreamSynchronize(s));
        const int launches = r.pass_launches[0];
        if (launches <= 1) continue;
        const double us = (r.pass_ms[0] + r.pass_ms[1]) * 1e3 / launches;
        if (us < best) {
            best = us;
            best_code = (c + 1) | ((c + 1) << 8);
        }
    }
    if (!best_code) return fail_arg("no tile configuration could be timed for this grid");
    *code_out = best_code;
    if (us_out) *us_out = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(g, o)] = best_code;
    return GBPCG_OK;
}

namespace {
// Persistent-kernel tile configuration per batch (device, io type, every problem's shape).
std::mutex g_ptune_mu;
std::map<std::vector<int>, int> g_ptune;
}  // namespace

// The batch as one persistent kernel (batch.cu); the workspace starts with
// its tables, problem i's piece sits at off[i].  With GBPCG_FLAG_AUTOTUNE
// each tile configuration is timed over 12 rounds into the pieces' scratch
// x (b only read) and the fastest is kept for this set of shapes.
static int persistent_batch(int nprob, const gbpcg_grid *grids, const void *const *b, void *const *x,
                            const gbpcg_opts *opts, gbpcg_result *results, char *ws, const std::vector<WsLayout> &L,
                            const std::vector<size_t> &off, cudaStream_t s) {
    auto make_calls = [&](bool scratch) {
        std::vector<SolveCall> calls(nprob);
        for (int i = 0; i < nprob; ++i) {
            char *w = ws + off[i];
            void *xi = scratch ? static_cast<void *>(w + L[i].total) : x[i];
            calls[i] = SolveCall{&grids[i], 0, 0, b[i], xi, w, L[i], opts->tol, opts->maxit, opts->io_dtype, 1.0f,
                                 nullptr};
        }
        return calls;
    };
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int> tkey{dev, opts->io_dtype};
    for (int i = 0; i < nprob; ++i) {
        tkey.push_back(grids[i].nx);
        tkey.push_back(grids[i].ny);
        tkey.push_back(grids[i].nz);
    }
    int cfg = 0;
    if (opts->tile_cfg) {
        cfg = (opts->tile_cfg & 0xff) - 1;
        if (cfg < 0 || cfg >= batch_persistent_cfgs() || (opts->tile_cfg >> 8))
            return fail_arg("persistent batch: tile_cfg must be 1, 2 or 3 (64x16, 128x8, 32x32 tiles)");
    } else if (opts->flags & GBPCG_FLAG_AUTOTUNE) {
        int found = -1;
        {
            std::lock_guard<std::mutex> lk(g_ptune_mu);
            auto it = g_ptune.find(tkey);
            if (it != g_ptune.end()) found = it->second;
        }
        if (found < 0) {
            const std::vector<SolveCall> sc = make_calls(true);
            double best = 1e300;
            cudaEvent_t t0, t1;
            GB_CUDA(cudaEventCreate(&t0));
            GB_CUDA(cudaEventCreate(&t1));
            for (int c = 0; c < batch_persistent_cfgs(); ++c) {
                for (int i = 0; i < nprob; ++i)
                    GB_CUDA(cudaMemsetAsync(sc[i].x, 0, (size_t)grids[i].nx * grids[i].ny * grids[i].nz *
                                                            dtype_size(opts->io_dtype), s));
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {  // the first run builds the graph
                    if (int rc = batch_persistent_launch(nprob, grids, sc.data(), ws, c, 0.0, 12, opts->io_dtype, s))
                        return rc;
                    GB_CUDA(cudaEventRecord(t0, s));
                    if (int rc = batch_persistent_launch(nprob, grids, sc.data(), ws, c, 0.0, 12, opts->io_dtype, s))
                        return rc;
                    GB_CUDA(cudaEventRecord(t1, s));
                    GB_CUDA(cudaEventSynchronize(t1));
                    GB_CUDA(cudaEventElapsedTime(&ms, t0, t1));
                }
                if (ms < best) {
                    best = ms;
                    found = c;
                }
            }
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            std::lock_guard<std::mutex> lk(g_ptune_mu);
            g_ptune[tkey] = found;
        }
        cfg = found;
    }
    const std::vector<SolveCall> calls = make_calls(false);
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } guard{e0, e1};
    GB_CUDA(cudaEventRecord(e0, s));
    if (int rc = batch_persistent_launch(nprob, grids, calls.data(), ws, cfg, opts->tol, opts->maxit, opts->io_dtype,
                                         s))
        return rc;
    GB_CUDA(cudaEventRecord(e1, s));
    std::vector<SolveState> hs(nprob);
    for (int i = 0; i < nprob; ++i)
        GB_CUDA(cudaMemcpyAsync(&hs[i], ws + off[i] + L[i].state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    int hdr[2] = {0, 0};  // abort, phases run
    if (int rc = batch_persistent_header(ws, hdr, s)) return rc;
    GB_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int worst = GBPCG_OK;
    for (int i = 0; i < nprob; ++i) {
        gbpcg_result &r = results[i];
        memset(&r, 0, sizeof(r));
        r.iters = hs[i].it;
        r.status = hs[i].status;
        if (hdr[0] && !(hs[i].done && hs[i].status == GBPCG_OK)) r.status = GBPCG_TIMEOUT;
        r.rel_res_recursive = hs[i].bb > 0 ? sqrt(hs[i].rr / hs[i].bb) : 0.0;
        r.rel_res_true = hs[i].bb_true > 0 ? sqrt(hs[i].rr_true / hs[i].bb_true) : 0.0;
        r.time_ms = ms;
        r.replacements = hs[i].n_replace;
        r.pass_launches[0] = 1;        // kernel launches of the whole batch
        r.pass_launches[1] = hdr[1];   // phases the persistent kernel ran, over all problems
        r.pass_ctas[0] = cfg;          // persistent tile configuration used
        if (r.status != GBPCG_OK && worst == GBPCG_OK) worst = r.status;
    }
    if (hdr[0]) set_error("a bounded grid-barrier wait of the persistent batch kernel timed out");
    return worst;
}

static int check_batch(int32_t nprob, const gbpcg_grid *grids, const gbpcg_opts *opts) {
    if (nprob <= 0 || nprob > 4096) return fail_arg("nprob must be in 1..4096");
    if (!grids) return fail_arg("grids is NULL");
    for (int i = 0; i < nprob; ++i)
        if (int rc = check_grid(&grids[i])) return rc;
    if (int rc = check_opts(opts)) return rc;
    if (opts->storage != GBPCG_F32) return fail_arg("batched solves use F32 storage");
    if (opts->flags & (GBPCG_FLAG_HOST_IO | GBPCG_FLAG_PROFILE | GBPCG_FLAG_HOST_LOOP | GBPCG_FLAG_SPLIT))
        return fail_arg("batched solves take device buffers and no profile, host-loop or split flag");
    return GBPCG_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

int gbpcg_tile_config(int32_t index, int32_t *tx, int32_t *ty, int32_t *stages) {
    clear_error();
    if (index < 0 || index >= NUM_CFG) return fail_arg("tile configuration index out of range");
    const CfgDims d = cfg_dims(index);
    if (tx) *tx = d.tx;
    if (ty) *ty = d.ty;
    if (stages) *stages = d.s;
    return GBPCG_OK;
}

int gbpcg_workspace_size(const gbpcg_grid *grid, const gbpcg_opts *opts, size_t *bytes) {
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (int rc = check_opts(opts)) return rc;
    if (!bytes) return fail_arg("bytes is NULL");
    *bytes = workspace_total(*grid, *opts);
    return GBPCG_OK;
}

int gbpcg_pcg_solve(const gbpcg_grid *grid, const void *b, void *x, const gbpcg_opts *opts, gbpcg_result *result,
                    gbpcg_stream stream) {
    NvtxRange range("gbpcg_pcg_solve");
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (int rc = check_opts(opts)) return rc;
    if (!b || !x || !result) return fail_arg("b, x and result must be non-NULL");
    memset(result, 0, sizeof(*result));
    const size_t total = workspace_total(*grid, *opts);
    if (!opts->workspace || opts->workspace_bytes < total) return fail_arg("workspace smaller than gbpcg_workspace_size()");
    if (reinterpret_cast<uintptr_t>(opts->workspace) & 255u) return fail_arg("workspace must be 256-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(opts->workspace);
    const gbpcg_grid g = *grid;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const size_t esz = dtype_size(opts->io_dtype);
    const size_t io_bytes = (size_t)n * esz;
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & (esz - 1))
        return fail_arg("b and x must be aligned to their element size");
    int cfg_a = 0, cfg_b = 0;
    pick_cfgs(g, *opts, &cfg_a, &cfg_b);
    if (!cfg_fits(cfg_a, g.nx) || !cfg_fits(cfg_b, g.nx))
        return fail_arg("tile_cfg selects a whole-row configuration for a grid wider than 256");

    // host buffers are staged through the end of the workspace
    const bool host_io = opts->flags & GBPCG_FLAG_HOST_IO;
    const bool b_host = host_io && !is_device_ptr(b);
    const bool x_host = host_io && !is_device_ptr(x);
    char *stage = ws + total - (host_io ? 2 * round256(io_bytes) : 0);
    const void *bd = b_host ? static_cast<const void *>(stage) : b;
    void *xd = x_host ? static_cast<void *>(stage + round256(io_bytes)) : x;
    if (b_host) GB_CUDA(cudaMemcpyAsync(const_cast<void *>(bd), b, io_bytes, cudaMemcpyHostToDevice, s));
    if (x_host) GB_CUDA(cudaMemcpyAsync(xd, x, io_bytes, cudaMemcpyHostToDevice, s));

    if (refine_mode(*opts)) {
        const RefineLayout R = refine_layout(g, *opts);
        const bool tma = tma_ok(dtype_size(opts->storage), g.nx,
                                {ws + R.inner + R.in.z, ws + R.inner + R.in.p0, ws + R.inner + R.in.p1,
                                 ws + R.inner + R.in.d});
        int rc = refine_solve(g, static_cast<const double *>(bd), static_cast<double *>(xd), opts, ws, R, cfg_a, cfg_b,
                              tma, result, s);
        if (x_host) {
            GB_CUDA(cudaMemcpyAsync(x, xd, io_bytes, cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
        }
        return rc;
    }

    if (opts->flags & GBPCG_FLAG_SPLIT) {
        if (g.k_block) return fail_arg("SPLIT takes the constant-coefficient operator");
        return split_solve(g, static_cast<const float *>(b), static_cast<float *>(x), *opts, result, s);
    }

    const WsLayout L = ws_layout_n((size_t)n, opts->storage, opts->io_dtype, false, block_count(g));
    const bool tma = tma_ok(sizeof(float), g.nx, {ws + L.z, ws + L.p0, ws + L.p1, ws + L.d});
    const SolveCall call{&g, cfg_a, cfg_b, bd, xd, ws, L, opts->tol, opts->maxit, opts->io_dtype, 1.0f, nullptr};
    const SolveState *st = reinterpret_cast<const SolveState *>(ws + L.state);
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    GB_CUDA(cudaEventRecord(e0, s));
    const int rc = (opts->flags & GBPCG_FLAG_PROFILE)     ? solve_profiled<float>(call, tma, result, s)
                   : (opts->flags & GBPCG_FLAG_HOST_LOOP) ? solve_host_loop<float>(call, tma, s)
                                                          : solve_launch<float>(call, tma, s);
    if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
    }
    GB_CUDA(cudaEventRecord(e1, s));
    return finish_solve(st, x, xd, x_host, io_bytes, e0, e1, result, s);
}

int gbpcg_autotune(const gbpcg_grid *grid, const gbpcg_opts *opts, const void *b, int32_t *tile_cfg,
                   double *us_per_iter, gbpcg_stream stream) {
    NvtxRange range("gbpcg_autotune");
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (int rc = check_opts(opts)) return rc;
    if (!b || !tile_cfg) return fail_arg("b and tile_cfg must be non-NULL");
    if (opts->storage != GBPCG_F32) return fail_arg("the autotuner times F32 storage");
    gbpcg_opts o = *opts;
    o.flags |= GBPCG_FLAG_AUTOTUNE;
    WsLayout L;
    const size_t need = batch_piece(*grid, o, &L);
    if (!opts->workspace || opts->workspace_bytes < need)
        return fail_arg("workspace smaller than gbpcg_workspace_size() with GBPCG_FLAG_AUTOTUNE");
    if (reinterpret_cast<uintptr_t>(opts->workspace) & 255u) return fail_arg("workspace must be 256-byte aligned");
    char *ws = static_cast<char *>(opts->workspace);
    int code = 0;
    if (int rc = autotune_one(*grid, o, b, ws + L.total, ws, L, reinterpret_cast<cudaStream_t>(stream), &code,
                              us_per_iter))
        return rc;
    *tile_cfg = code;
    return GBPCG_OK;
}

int gbpcg_autotune_record(const gbpcg_grid *grid, const gbpcg_opts *opts, int32_t tile_cfg) {
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (int rc = check_opts(opts)) return rc;
    gbpcg_opts o = *opts;
    o.tile_cfg = tile_cfg;
    if (int rc = check_opts(&o)) return rc;
    if (!tile_cfg) return fail_arg("tile_cfg 0 is not a configuration");
    int ca = 0, cb = 0;
    pick_cfgs(*grid, o, &ca, &cb);
    if (!cfg_fits(ca, grid->nx) || !cfg_fits(cb, grid->nx)) return fail_arg("configuration does not fit the grid");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(*grid, *opts)] = tile_cfg;
    return GBPCG_OK;
}

int gbpcg_workspace_size_batched(int32_t nprob, const gbpcg_grid *grids, const gbpcg_opts *opts, size_t *bytes) {
    clear_error();
    if (int rc = check_batch(nprob, grids, opts)) return rc;
    if (!bytes) return fail_arg("bytes is NULL");
    size_t total = round256(batch_persistent_bytes(nprob, grids));  // the persistent kernel's tables
    for (int i = 0; i < nprob; ++i) {
        WsLayout L;
        total += batch_piece(grids[i], *opts, &L);
    }
    *bytes = total;
    return GBPCG_OK;
}

int gbpcg_pcg_solve_batched(int32_t nprob, const gbpcg_grid *grids, const void *const *b, void *const *x,
                            const gbpcg_opts *opts, gbpcg_result *results, gbpcg_stream stream) {
    NvtxRange range("gbpcg_pcg_solve_batched");
    clear_error();
    if (int rc = check_batch(nprob, grids, opts)) return rc;
    if (!b || !x || !results) return fail_arg("b, x and results must be non-NULL");
    const size_t esz = dtype_size(opts->io_dtype);
    for (int i = 0; i < nprob; ++i) {
        if (!b[i] || !x[i]) return fail_arg("every b[i] and x[i] must be a device pointer");
        if ((reinterpret_cast<uintptr_t>(b[i]) | reinterpret_cast<uintptr_t>(x[i])) & (esz - 1))
            return fail_arg("b[i] and x[i] must be aligned to their element size");
    }
    const size_t region = round256(batch_persistent_bytes(nprob, grids));
    size_t need = region;
    std::vector<WsLayout> L(nprob);
    std::vector<size_t> off(nprob);
    for (int i = 0; i < nprob; ++i) {
        off[i] = need;
        need += batch_piece(grids[i], *opts, &L[i]);
    }
    if (!opts->workspace || opts->workspace_bytes < need)
        return fail_arg("workspace smaller than gbpcg_workspace_size_batched()");
    if (reinterpret_cast<uintptr_t>(opts->workspace) & 255u) return fail_arg("workspace must be 256-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(opts->workspace);

    if (!(opts->flags & GBPCG_FLAG_BATCH_GRAPH) && batch_persistent_ok(nprob, grids))
        return persistent_batch(nprob, grids, b, x, opts, results, ws, L, off, s);

    // tile configurations: explicit, autotuned (cached per shape), or the defaults
    std::vector<SolveCall> calls(nprob);
    std::vector<int> tma(nprob);
    for (int i = 0; i < nprob; ++i) {
        const gbpcg_grid &g = grids[i];
        gbpcg_opts o = *opts;
        if (!o.tile_cfg && (o.flags & GBPCG_FLAG_AUTOTUNE)) {
            int code = 0;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune.find(tune_key(g, o));
                if (it != g_tune.end()) code = it->second;
            }
            if (!code) {
                if (int rc = autotune_one(g, o, b[i], ws + off[i] + L[i].total, ws + off[i], L[i], s, &code, nullptr))
                    return rc;
            }
            o.tile_cfg = code;
        }
        int ca = 0, cb = 0;
        pick_cfgs(g, o, &ca, &cb);
        if (!cfg_fits(ca, g.nx) || !cfg_fits(cb, g.nx))
            return fail_arg("tile_cfg selects a whole-row configuration for a grid wider than 256");
        char *w = ws + off[i];
        tma[i] = tma_ok(sizeof(float), g.nx, {w + L[i].z, w + L[i].p0, w + L[i].p1, w + L[i].d});
        calls[i] = SolveCall{&grids[i], ca, cb, b[i], x[i], w, L[i], opts->tol, opts->maxit, opts->io_dtype, 1.0f,
                             nullptr};
    }
    std::vector<SolveKey> keys(nprob);
    for (int i = 0; i < nprob; ++i) keys[i] = make_key<float>(calls[i], tma[i] != 0);

    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (auto it = g_batch_cache.begin(); it != g_batch_cache.end(); ++it)
            if (it->keys.size() == keys.size() &&
                std::equal(keys.begin(), keys.end(), it->keys.begin(),
                           [](const SolveKey &a, const SolveKey &c) { return a == c; })) {
                g_batch_cache.splice(g_batch_cache.begin(), g_batch_cache, it);
                exec = g_batch_cache.front().exec;
                break;
            }
        if (!exec) {
            cudaGraph_t graph = nullptr;
            if (int rc = batched_capture<float>(calls.data(), tma.data(), nprob, &graph)) return rc;
            cudaGraphExec_t ex = nullptr;
            cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
            if (e) {
                cudaGraphDestroy(graph);
                return fail_cuda(e, "batched graph instantiate");
            }
            cudaGraphUpload(ex, s);
            BatchGraph bg;
            bg.keys = keys;
            bg.graph = graph;
            bg.exec = ex;
            g_batch_cache.push_front(bg);
            while (g_batch_cache.size() > kBatchCacheMax) {
                cudaGraphExecDestroy(g_batch_cache.back().exec);
                cudaGraphDestroy(g_batch_cache.back().graph);
                g_batch_cache.pop_back();
            }
            exec = ex;
        }
    }
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    GB_CUDA(cudaEventRecord(e0, s));
    GB_CUDA(cudaGraphLaunch(exec, s));
    GB_CUDA(cudaEventRecord(e1, s));
    std::vector<SolveState> hs(nprob);
    for (int i = 0; i < nprob; ++i)
        GB_CUDA(cudaMemcpyAsync(&hs[i], ws + off[i] + L[i].state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = GBPCG_OK;
    for (int i = 0; i < nprob; ++i) {
        gbpcg_result &r = results[i];
        memset(&r, 0, sizeof(r));
        r.iters = hs[i].it;
        r.status = hs[i].status;
        r.rel_res_recursive = hs[i].bb > 0 ? sqrt(hs[i].rr / hs[i].bb) : 0.0;
        r.rel_res_true = hs[i].bb_true > 0 ? sqrt(hs[i].rr_true / hs[i].bb_true) : 0.0;
        r.time_ms = ms;
        r.replacements = hs[i].n_replace;
        if (r.status != GBPCG_OK && worst == GBPCG_OK) worst = r.status;
    }
    return worst;
}

}  // extern "C"
