// Jacobi-PCG on a general sparse matrix in Sliced-ELL form (the format the
// paper's H100 comparator stores the seven-point operator in, Sec. VII-A,
// and the "more general sparse matrix representations" its conclusion names
// as future work).
//
// SELL-C: rows are grouped into slices of C = 32 consecutive rows (one warp,
// one row per lane); slice s stores width_s = max row length of its rows
// entries per row, column-major within the slice (entry j of lane l at
// slice_ptr[s] + 32 j + l), so a warp reads each entry column as one
// 128-byte line.  Short rows are padded with value 0 and their own row as
// the column (an in-bounds gather that adds nothing).
//
// The solver is the textbook iteration split into three kernels per
// iteration, each with its reductions fused in and the scalars kept on the
// device, the whole loop one CUDA graph (as the stencil solver):
//   spmv:    q = A p, p.q               -> alpha (last CTA)
//   update:  x += alpha p (FP64 x), r -= alpha q, z = D^-1 r, r.r, r.z
//                                       -> beta, convergence, replacement
//   p:       p = z + beta p  (z recomputed from r)
// plus an FP64 residual b - A x (gathering the FP64 x) at the start, when
// the recursive residual meets the tolerance or has dropped two decades
// since the last replacement, and at the end.  Per iteration 108 bytes per
// row for a seven-point matrix (values and columns 56, gathers and vectors
// 52), against the matrix-free passes' 32.
#include <algorithm>
#include <cstring>
#include <vector>

#include "solver.cuh"

namespace gb {

namespace {

constexpr int kSell = 32;  // rows per slice
constexpr int kSellThreads = 256;

struct SellDev {
    int64_t n, nslices;
    const int64_t *slice_ptr;
    const int32_t *col;
    const float *val;
    const float *inv_diag;
};

inline SellDev to_dev(const gbpcg_sell &m) {
    return SellDev{m.n, (m.n + kSell - 1) / kSell, m.slice_ptr, m.col, m.val, m.inv_diag};
}

// Row i's range of entries: first entry, count (the slice width), stride 32.
__device__ __forceinline__ void sell_row(const SellDev &A, int64_t i, int64_t &e0, int &w) {
    const int64_t s = i / kSell;
    const int64_t p0 = __ldg(A.slice_ptr + s), p1 = __ldg(A.slice_ptr + s + 1);
    w = (int)((p1 - p0) / kSell);
    e0 = p0 + (i - s * kSell);
}

// y = A x (FP32 products and sums, one row per thread, a slice per warp).
__global__ void __launch_bounds__(kSellThreads)
    sell_spmv_kernel(const SellDev A, const float *__restrict__ x, float *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * kSellThreads) {
        int64_t e;
        int w;
        sell_row(A, i, e, w);
        float s = 0.f;
        for (int j = 0; j < w; ++j, e += kSell) s = fmaf(__ldg(A.val + e), __ldg(x + __ldg(A.col + e)), s);
        y[i] = s;
    }
}

// q = A p and the partial p.q; last CTA: alpha.
__global__ void __launch_bounds__(kSellThreads)
    sell_spmv_dot_kernel(const SellDev A, const float *__restrict__ p, float *__restrict__ q, SolveState *st,
                         double *partials) {
    if (st->done) return;
    float acc[1] = {0.f};
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * kSellThreads) {
        int64_t e;
        int w;
        sell_row(A, i, e, w);
        float s = 0.f;
        for (int j = 0; j < w; ++j, e += kSell) s = fmaf(__ldg(A.val + e), __ldg(p + __ldg(A.col + e)), s);
        q[i] = s;
        acc[0] = fmaf(p[i], s, acc[0]);
    }
    double part[1], tot[1];
    block_sum<1, kSellThreads>(acc, part);
    if (grid_sum_last<1, kSellThreads>(part, partials, &st->ticket[K_PASSA], tot) && threadIdx.x == 0)
        passa_finish(st, tot[0], false);
}

// x += alpha p (FP64), r -= alpha q, z = D^-1 r; partials r.r, r.z; last CTA:
// beta, the convergence test and the replacement trigger.
__global__ void __launch_bounds__(kSellThreads)
    sell_update_kernel(const SellDev A, double *__restrict__ x, const float *__restrict__ p,
                       const float *__restrict__ q, float *__restrict__ r, SolveState *st, double *partials,
                       cudaGraphConditionalHandle cond, cudaGraphConditionalHandle cond_rep, int use_cond) {
    if (st->done) return;
    const int it = st->it;
    const double alpha = st->alpha;
    const float af = (float)alpha;
    float acc[2] = {0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * kSellThreads) {
        const float pi = p[i];
        x[i] = fma(alpha, (double)pi, x[i]);
        const float ri = fmaf(-af, q[i], r[i]);
        r[i] = ri;
        const float zi = __ldg(A.inv_diag + i) * ri;
        acc[0] = fmaf(ri, ri, acc[0]);
        acc[1] = fmaf(ri, zi, acc[1]);
    }
    double part[2], tot[2];
    block_sum<2, kSellThreads>(acc, part);
    if (grid_sum_last<2, kSellThreads>(part, partials, &st->ticket[K_PASSB], tot) && threadIdx.x == 0) {
        passb_finish(st, it, tot[0], tot[1], false);
        if (use_cond) {
            cudaGraphSetConditional(cond, st->done ? 0u : 1u);
            cudaGraphSetConditional(cond_rep, st->replace ? 1u : 0u);
        }
    }
}

// p = D^-1 r + beta p (p = D^-1 r when beta = 0 and p was zeroed).
__global__ void __launch_bounds__(kSellThreads)
    sell_p_kernel(const SellDev A, const float *__restrict__ r, float *__restrict__ p, const SolveState *st) {
    if (st->done) return;
    const float beta = (float)st->beta;
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * kSellThreads)
        p[i] = fmaf(beta, p[i], __ldg(A.inv_diag + i) * r[i]);
}

// r = b - A x with FP64 products and sums (x gathered in FP64); r stored as
// FP32.  INIT: sums r.r, r.z, b.b -> start state; REPLACE: r.r, r.z -> the
// replacement's decisions (only when one was requested); TRUE: r.r -> the
// reported true residual.
template <int MODE>
__global__ void __launch_bounds__(kSellThreads)
    sell_residual_kernel(const SellDev A, const double *__restrict__ b, const double *__restrict__ x,
                         float *__restrict__ r, SolveState *st, double *partials, cudaGraphConditionalHandle cond,
                         int use_cond) {
    if (MODE == RES_REPLACE && (!st->replace || st->done)) return;
    if (MODE == RES_TRUE && st->true_known) return;
    constexpr int NV = res64_nv<MODE>();
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * kSellThreads) {
        int64_t e;
        int w;
        sell_row(A, i, e, w);
        double ax = 0.0;
        for (int j = 0; j < w; ++j, e += kSell) ax = fma((double)__ldg(A.val + e), __ldg(x + __ldg(A.col + e)), ax);
        const double bi = __ldg(b + i);
        const double ri = bi - ax;
        if (MODE == RES_TRUE) {
            s[0] = fma(ri, ri, s[0]);
        } else {
            const float rf = (float)ri;
            r[i] = rf;
            const double zi = (double)(__ldg(A.inv_diag + i) * rf);
            s[0] = fma(ri, ri, s[0]);
            s[1] = fma(ri, zi, s[1]);
            s[2] = fma(bi, bi, s[2]);
        }
    }
    __shared__ double red[kSellThreads / 32][3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const double t = warp_sum(s[v]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = t;
    }
    __syncthreads();
    double part[NV], tot[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        part[v] = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kSellThreads / 32; ++w) part[v] += red[w][v];
    }
    if (!grid_sum_last<NV, kSellThreads>(part, partials, &st->ticket[4 + MODE], tot) || threadIdx.x != 0) return;
    res64_finish<MODE>(st, tot, 1.0);
    if (MODE != RES_TRUE && use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

__global__ void sell_reset_kernel(SolveState *st, double tol, int maxit) {
    memset(st, 0, sizeof(SolveState));
    st->tol2 = tol * tol;
    st->maxit = maxit;
    st->status = GBPCG_NOT_CONVERGED;
}

// x = 0 when b = 0 (the start state marks it)
__global__ void __launch_bounds__(kSellThreads) sell_zero_x_kernel(int64_t n, double *x, const SolveState *st) {
    if (!st->zero_x) return;
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kSellThreads)
        x[i] = 0.0;
}

// ------------------------------------------------------------- assembly --

// Seven-point operator rows in SELL form: entries in column order
// (z-1, y-1, x-1, centre, x+1, y+1, z+1), absent neighbours skipped, the
// slice's remaining entries padded.  Face weights are the stencil's own
// (OpBlock, bitwise the same FP32 values); the diagonal is their sum.
__global__ void __launch_bounds__(kSellThreads)
    sell_stencil_fill_kernel(int nx, int ny, int nz, OpBlock ob, int block, const int64_t *__restrict__ slice_ptr,
                             int32_t *col, float *val, float *inv_diag) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kSellThreads) {
        const int x = (int)(i % nx);
        const int64_t t = i / nx;
        const int y = (int)(t % ny), z = (int)(t / ny);
        float w[6];  // x-, x+, y-, y+, z-, z+
        if (block) {
            ob.weights(x, y, z, w);
        } else {
            w[0] = w[1] = ob.cx;
            w[2] = w[3] = ob.cy;
            w[4] = w[5] = ob.cz;
        }
        const float dg = ((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]);
        const int64_t s = i / kSell;
        const int64_t p0 = slice_ptr[s], p1 = slice_ptr[s + 1];
        const int width = (int)((p1 - p0) / kSell);
        int64_t e = p0 + (i - s * kSell);
        int k = 0;
        auto put = [&](int64_t c, float v) {
            col[e] = (int32_t)c;
            val[e] = v;
            e += kSell;
            ++k;
        };
        if (z > 0) put(i - (int64_t)nx * ny, -w[4]);
        if (y > 0) put(i - nx, -w[2]);
        if (x > 0) put(i - 1, -w[0]);
        put(i, dg);
        if (x < nx - 1) put(i + 1, -w[1]);
        if (y < ny - 1) put(i + nx, -w[3]);
        if (z < nz - 1) put(i + (int64_t)nx * ny, -w[5]);
        while (k < width) put(i, 0.0f);
        inv_diag[i] = 1.0f / dg;
    }
}

// CSR -> SELL: each row's entries in CSR order, then padding; D^-1 from the
// diagonal entry (a row without one, or with a zero diagonal, writes 0).
__global__ void __launch_bounds__(kSellThreads)
    sell_from_csr_kernel(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ ccol,
                         const float *__restrict__ cval, const int64_t *__restrict__ slice_ptr, int32_t *col,
                         float *val, float *inv_diag) {
    for (int64_t i = (int64_t)blockIdx.x * kSellThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kSellThreads) {
        const int64_t s = i / kSell;
        const int width = (int)((slice_ptr[s + 1] - slice_ptr[s]) / kSell);
        int64_t e = slice_ptr[s] + (i - s * kSell);
        float dg = 0.0f;
        int k = 0;
        for (int64_t c = row_ptr[i]; c < row_ptr[i + 1]; ++c, ++k, e += kSell) {
            col[e] = ccol[c];
            val[e] = cval[c];
            if (ccol[c] == i) dg = cval[c];
        }
        for (; k < width; ++k, e += kSell) {
            col[e] = (int32_t)i;
            val[e] = 0.0f;
        }
        inv_diag[i] = dg != 0.0f ? 1.0f / dg : 0.0f;
    }
}

unsigned sell_grid(int64_t n) {
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>({(n + kSellThreads - 1) / kSellThreads, (int64_t)device_sm_count() * 8,
                              (int64_t)kMaxPassBlocks}));
}

// slice_ptr (host) from row lengths: width of a slice = its longest row.
template <typename LenFn>
std::vector<int64_t> slice_layout(int64_t n, LenFn len) {
    const int64_t ns = (n + kSell - 1) / kSell;
    std::vector<int64_t> ptr(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        int w = 0;
        for (int64_t i = s * kSell; i < std::min(n, (s + 1) * kSell); ++i) w = std::max(w, len(i));
        ptr[s + 1] = ptr[s] + (int64_t)w * kSell;
    }
    return ptr;
}

struct SellWs {
    size_t state, partials, r, p, q, total;
};
SellWs sell_ws(int64_t n) {
    SellWs w;
    size_t o = 0;
    w.state = o; o += 256;
    w.partials = o; o += round256(sizeof(double) * 4 * kMaxPassBlocks);
    w.r = o; o += round256((size_t)n * 4);
    w.p = o; o += round256((size_t)n * 4);
    w.q = o; o += round256((size_t)n * 4);
    w.total = o;
    return w;
}

int check_sell(const gbpcg_sell *m) {
    if (!m) return fail_arg("matrix is NULL");
    if (m->n <= 0 || m->n > ((int64_t)1 << 31) - 1) return fail_arg("n must be in 1 .. 2^31 - 1");
    if (m->slice != kSell) return fail_arg("slice must be 32 rows");
    if (!m->slice_ptr || !m->col || !m->val || !m->inv_diag) return fail_arg("NULL matrix array");
    return GBPCG_OK;
}

// One solve's launches, recorded into a graph or launched directly.
struct SellPlan {
    SellDev A;
    const double *b;
    double *x;
    SolveState *st;
    double *partials;
    float *r, *p, *q;
    double tol;
    int maxit;
    unsigned grid;
    cudaGraphConditionalHandle cond = 0, cond_rep = 0;
    int use_cond = 0;

    void setup(cudaStream_t s) {
        sell_reset_kernel<<<1, 1, 0, s>>>(st, tol, maxit);
        cudaMemsetAsync(p, 0, (size_t)A.n * 4, s);
        sell_residual_kernel<RES_INIT><<<grid, kSellThreads, 0, s>>>(A, b, x, r, st, partials, cond, use_cond);
        sell_zero_x_kernel<<<grid, kSellThreads, 0, s>>>(A.n, x, st);
        sell_p_kernel<<<grid, kSellThreads, 0, s>>>(A, r, p, st);
    }
    void body(cudaStream_t s) {
        sell_spmv_dot_kernel<<<grid, kSellThreads, 0, s>>>(A, p, q, st, partials);
        sell_update_kernel<<<grid, kSellThreads, 0, s>>>(A, x, p, q, r, st, partials, cond, cond_rep, use_cond);
    }
    void replace(cudaStream_t s) {
        sell_residual_kernel<RES_REPLACE><<<grid, kSellThreads, 0, s>>>(A, b, x, r, st, partials, cond, use_cond);
    }
    void tail(cudaStream_t s) { sell_p_kernel<<<grid, kSellThreads, 0, s>>>(A, r, p, st); }
    void finish(cudaStream_t s) {
        sell_residual_kernel<RES_TRUE><<<grid, kSellThreads, 0, s>>>(A, b, x, r, st, partials, cond, use_cond);
    }
};

// reset -> r0, p0 -> while(cond){spmv; update; if(replace){residual}; p} -> true residual
int sell_capture(SellPlan &P, cudaGraph_t *out) {
    cudaStream_t cs = nullptr, bs = nullptr, rs = nullptr;
    GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
    auto add_cond = [&](cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                        cudaGraph_t *body_out) -> cudaError_t {
        cudaStreamCaptureStatus cst;
        cudaGraph_t cap = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        cudaError_t e2 = cudaStreamGetCaptureInfo(s, &cst, nullptr, &cap, &deps, nullptr, &ndeps);
        if (e2) return e2;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = type;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        e2 = cudaGraphAddNode(&node, cap, deps, nullptr, ndeps, &cp);
        if (e2) return e2;
        *body_out = cp.conditional.phGraph_out[0];
        return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    };
    cudaGraph_t graph = nullptr;
    bool cap_main = false, cap_b = false, cap_r = false;
    do {
        if (e) break;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e) break;
        cap_main = true;
        cudaStreamCaptureStatus cst;
        cudaGraph_t cap = nullptr;
        e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap, nullptr, nullptr, nullptr);
        if (e) break;
        e = cudaGraphConditionalHandleCreate(&P.cond, cap, 1, cudaGraphCondAssignDefault);
        if (e) break;
        P.use_cond = 1;
        P.setup(cs);
        cudaGraph_t body = nullptr;
        e = add_cond(cs, P.cond, cudaGraphCondTypeWhile, &body);
        if (e) break;
        e = cudaGraphConditionalHandleCreate(&P.cond_rep, body, 0, cudaGraphCondAssignDefault);
        if (e) break;
        e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e) break;
        cap_b = true;
        P.body(bs);
        cudaGraph_t rbody = nullptr;
        e = add_cond(bs, P.cond_rep, cudaGraphCondTypeIf, &rbody);
        if (e) break;
        e = cudaStreamBeginCaptureToGraph(rs, rbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e) break;
        cap_r = true;
        P.replace(rs);
        cudaGraph_t tmp = nullptr;
        e = cudaStreamEndCapture(rs, &tmp);
        cap_r = false;
        if (e) break;
        P.tail(bs);
        e = cudaStreamEndCapture(bs, &tmp);
        cap_b = false;
        if (e) break;
        P.finish(cs);
        e = cudaStreamEndCapture(cs, &graph);
        cap_main = false;
    } while (0);
    cudaGraph_t tmp = nullptr;
    if (cap_r) cudaStreamEndCapture(rs, &tmp);
    if (cap_b) cudaStreamEndCapture(bs, &tmp);
    if (cap_main) {
        cudaStreamEndCapture(cs, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
    }
    if (rs) cudaStreamDestroy(rs);
    if (bs) cudaStreamDestroy(bs);
    cudaStreamDestroy(cs);
    if (e) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail_cuda(e, "SELL solve graph capture");
    }
    *out = graph;
    return GBPCG_OK;
}

}  // namespace

}  // namespace gb

using namespace gb;

extern "C" {

int gbpcg_sell_stencil_layout(const gbpcg_grid *grid, int64_t *slice_ptr, int64_t *nnz_stored,
                              gbpcg_stream stream) {
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (!nnz_stored) return fail_arg("nnz_stored is NULL");
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > ((int64_t)1 << 31) - 1) return fail_arg("SELL column indices are 32-bit: at most 2^31 - 1 rows");
    const std::vector<int64_t> ptr = slice_layout(n, [&](int64_t i) {
        const int x = (int)(i % nx);
        const int64_t t = i / nx;
        const int y = (int)(t % ny), z = (int)(t / ny);
        return 1 + (x > 0) + (x < nx - 1) + (y > 0) + (y < ny - 1) + (z > 0) + (z < nz - 1);
    });
    *nnz_stored = ptr.back();
    if (!slice_ptr) return GBPCG_OK;  // size query
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    GB_CUDA(cudaMemcpyAsync(slice_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBPCG_OK;
}

int gbpcg_sell_from_stencil(const gbpcg_grid *grid, const int64_t *slice_ptr, int32_t *col, float *val,
                            float *inv_diag, gbpcg_stream stream) {
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (!slice_ptr || !col || !val || !inv_diag) return fail_arg("NULL output array");
    const int64_t n = (int64_t)grid->nx * grid->ny * grid->nz;
    if (n > ((int64_t)1 << 31) - 1) return fail_arg("SELL column indices are 32-bit: at most 2^31 - 1 rows");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    OpBlock ob = make_op_block(*grid);
    sell_stencil_fill_kernel<<<sell_grid(n), kSellThreads, 0, s>>>(grid->nx, grid->ny, grid->nz, ob,
                                                                     grid->k_block ? 1 : 0, slice_ptr, col, val,
                                                                     inv_diag);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

int gbpcg_sell_csr_layout(int64_t n, const int64_t *row_ptr, int64_t *slice_ptr, int64_t *nnz_stored,
                          gbpcg_stream stream) {
    clear_error();
    if (n <= 0 || n > ((int64_t)1 << 31) - 1) return fail_arg("n must be in 1 .. 2^31 - 1");
    if (!row_ptr || !nnz_stored) return fail_arg("NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int64_t> rp(n + 1);
    GB_CUDA(cudaMemcpyAsync(rp.data(), row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return fail_arg("row_ptr must be non-decreasing");
    const std::vector<int64_t> ptr = slice_layout(n, [&](int64_t i) { return (int)(rp[i + 1] - rp[i]); });
    *nnz_stored = ptr.back();
    if (!slice_ptr) return GBPCG_OK;
    GB_CUDA(cudaMemcpyAsync(slice_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBPCG_OK;
}

int gbpcg_sell_from_csr(int64_t n, const int64_t *row_ptr, const int32_t *csr_col, const float *csr_val,
                        const int64_t *slice_ptr, int32_t *col, float *val, float *inv_diag, gbpcg_stream stream) {
    clear_error();
    if (n <= 0 || n > ((int64_t)1 << 31) - 1) return fail_arg("n must be in 1 .. 2^31 - 1");
    if (!row_ptr || !csr_col || !csr_val || !slice_ptr || !col || !val || !inv_diag) return fail_arg("NULL array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    sell_from_csr_kernel<<<sell_grid(n), kSellThreads, 0, s>>>(n, row_ptr, csr_col, csr_val, slice_ptr, col, val,
                                                                inv_diag);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

int gbpcg_sell_spmv(const gbpcg_sell *m, const float *x, float *y, gbpcg_stream stream) {
    clear_error();
    if (int rc = check_sell(m)) return rc;
    if (!x || !y || x == y) return fail_arg("x and y must be distinct device arrays");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    sell_spmv_kernel<<<sell_grid(m->n), kSellThreads, 0, s>>>(to_dev(*m), x, y);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

int gbpcg_sell_workspace_size(const gbpcg_sell *m, size_t *bytes) {
    clear_error();
    if (int rc = check_sell(m)) return rc;
    if (!bytes) return fail_arg("bytes is NULL");
    *bytes = sell_ws(m->n).total;
    return GBPCG_OK;
}

int gbpcg_sell_pcg_solve(const gbpcg_sell *m, const double *b, double *x, const gbpcg_opts *opts,
                         gbpcg_result *result, gbpcg_stream stream) {
    NvtxRange range("gbpcg_sell_pcg_solve");
    clear_error();
    if (int rc = check_sell(m)) return rc;
    if (!opts || !b || !x || !result) return fail_arg("NULL argument");
    if (!(opts->tol >= 0.0) || opts->maxit < 0) return fail_arg("tol must be >= 0 and maxit >= 0");
    if (opts->io_dtype != GBPCG_F64 || opts->storage != GBPCG_F32 || opts->precond != GBPCG_PRECOND_JACOBI ||
        opts->flags)
        return fail_arg("SELL solves take FP64 b and x, FP32 vectors, Jacobi, no flags");
    const SellWs W = sell_ws(m->n);
    if (!opts->workspace || opts->workspace_bytes < W.total || (reinterpret_cast<uintptr_t>(opts->workspace) & 255u))
        return fail_arg("workspace: gbpcg_sell_workspace_size() bytes, 256-byte aligned");
    memset(result, 0, sizeof(*result));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(opts->workspace);
    SellPlan P;
    P.A = to_dev(*m);
    P.b = b;
    P.x = x;
    P.st = reinterpret_cast<SolveState *>(ws + W.state);
    P.partials = reinterpret_cast<double *>(ws + W.partials);
    P.r = reinterpret_cast<float *>(ws + W.r);
    P.p = reinterpret_cast<float *>(ws + W.p);
    P.q = reinterpret_cast<float *>(ws + W.q);
    P.tol = opts->tol;
    P.maxit = opts->maxit;
    P.grid = sell_grid(m->n);
    // one graph per call (the device-driven loop); the solve itself dominates its build
    cudaGraph_t graph = nullptr;
    if (int rc = sell_capture(P, &graph)) return rc;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return fail_cuda(e, "SELL graph instantiate");
    struct ExecGuard { cudaGraphExec_t g; ~ExecGuard() { cudaGraphExecDestroy(g); } } eg{exec};
    cudaGraphUpload(exec, s);
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    GB_CUDA(cudaEventRecord(e0, s));
    GB_CUDA(cudaGraphLaunch(exec, s));
    GB_CUDA(cudaEventRecord(e1, s));
    SolveState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, P.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
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
    return hs.status;
}

}  // extern "C"
