// Flexible CG with the learned preconditioner z = N(r) (no counterpart in
// the paper).  N is nonlinear (ReLU), so plain PCG's short recurrence loses
// conjugacy; FCG with truncation m (Notay, SIAM J. Sci. Comput. 22, 2000)
// A-orthogonalises each new direction against the last m explicitly:
//   p_k = z_k - sum_{i=k-m}^{k-1} (z_k.Ap_i / p_i.Ap_i) p_i,
//   alpha_k = p_k.r_k / p_k.Ap_k.
// m = 1 is the familiar beta = z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k) form; a
// larger m keeps a strongly nonlinear N from undoing earlier progress.
//
// One iteration: z = N(r); one fused pass for r.z and every z.Ap_i (the
// projection coefficients are formed on the device); p = z - sum c_i p_i;
// Ap; one fused pass for p.Ap and r.p (alpha on the device); fused update
// x += alpha p (FP64), r -= alpha Ap with r.r.  The directions and their
// A-images live in a ring of m + 1 slots.  Every kernel after a failed
// descent check (r.z <= 0, p.Ap <= 0, a non-finite scalar) leaves x, r and
// p untouched, and the host, which reads the scalars once per iteration,
// switches to Jacobi PCG from the current x (GBPCG_FALLBACK_USED).  At
// recursive convergence the true residual is recomputed in FP64; if it
// misses the tolerance, r is replaced by it and FCG restarts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace gb {

int launch_stencil_f64(const gbpcg_grid &g, const double *p, double *q, cudaStream_t s);

// from nn.cu
size_t nn_layout_total(int X, int Y, int Z, bool training);
size_t nn_layout_err_offset();
bool nn_shape_ok_ext(int X, int Y, int Z);
int nn_prep_ext(const float *w, void *ws, const gbpcg_grid &g, cudaStream_t s);
int nn_forward_ext(const gbpcg_grid &g, const float *r, float *z, void *ws, cudaStream_t s);

constexpr int kMaxDirs = 32;

struct FcgState {
    double bb, rz, rp, rr, rr64;
    double pq[kMaxDirs + 1];  // p.Ap of every ring slot
    double c[kMaxDirs];       // projection coefficients of the current step
    int bad;                  // 1: p.Ap <= 0 or not finite; 2: r.z <= 0 or not finite
    int pad;
    unsigned ticket[4];
};

// The previous directions of one step: ring slots, oldest first.
struct DirSet {
    const float *p[kMaxDirs];
    const float *q[kMaxDirs];
    int slot[kMaxDirs];
    int nd;
};

constexpr int kFcgThreads = 256;
constexpr unsigned kFcgMaxBlocks = 2048;

// d (FP64, in place of A x) = b - A x, and its FP32 copy r = s d (optional)
__global__ void __launch_bounds__(256)
    fcg_residual_kernel(int64_t n, const double *__restrict__ b, double *__restrict__ ax, float *__restrict__ r,
                        double s) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = b[i] - ax[i];
        ax[i] = d;
        if (r) r[i] = (float)(s == 1.0 ? d : d * s);
    }
}

__device__ __forceinline__ float dot4f(const float4 a, const float4 b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// Sums NV per-thread doubles over the block (result in thread 0), then over
// the grid with the fixed-order last-block finish.
template <int NV>
__device__ __forceinline__ bool fcg_reduce(const double (&acc)[NV], double *partials, unsigned *ticket,
                                           double (&tot)[NV]) {
    __shared__ double red[kFcgThreads / 32][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double s = warp_sum(acc[v]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = s;
    }
    __syncthreads();
    double part[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        part[v] = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kFcgThreads / 32; ++w) part[v] += red[w][v];
    }
    return grid_sum_last<NV, kFcgThreads>(part, partials, ticket, tot);
}

// r.z and z.Ap_i of every previous direction; the last block forms the
// projection coefficients c_i = z.Ap_i / p_i.Ap_i and checks r.z > 0.
__global__ void __launch_bounds__(kFcgThreads)
    fcg_mdot_kernel(int64_t n4, FcgState *st, double *partials, const float *__restrict__ r,
                    const float *__restrict__ z, const DirSet d) {
    // FP32 sums per thread (a handful of grid-stride steps), FP64 from the warp sums on:
    // GB300's FP64 pipe would otherwise bound this kernel, not its loads
    float facc[kMaxDirs + 1];
#pragma unroll
    for (int v = 0; v <= kMaxDirs; ++v) facc[v] = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kFcgThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kFcgThreads) {
        const float4 zv = reinterpret_cast<const float4 *>(z)[i];
        facc[0] += dot4f(reinterpret_cast<const float4 *>(r)[i], zv);
#pragma unroll
        for (int j = 0; j < kMaxDirs; ++j)
            if (j < d.nd) facc[1 + j] += dot4f(reinterpret_cast<const float4 *>(d.q[j])[i], zv);
    }
    double acc[kMaxDirs + 1];
#pragma unroll
    for (int v = 0; v <= kMaxDirs; ++v) acc[v] = (double)facc[v];
    double tot[kMaxDirs + 1];
    if (fcg_reduce<kMaxDirs + 1>(acc, partials, &st->ticket[0], tot) && threadIdx.x == 0) {
        const double rz = tot[0];
        bool ok = rz > 0.0 && isfinite(rz);
#pragma unroll
        for (int j = 0; j < kMaxDirs; ++j)  // static indices: no local copy of the parameter arrays
            if (j < d.nd) {
                const double c = tot[1 + j] / st->pq[d.slot[j]];
                ok = ok && isfinite(c);
                st->c[j] = c;
            }
        st->rz = rz;
        if (!ok) st->bad = 2;
    }
}

// p = z - sum_j c_j p_j
__global__ void __launch_bounds__(256)
    fcg_combine_kernel(int64_t n4, const FcgState *st, const float *__restrict__ z, const DirSet d,
                       float *__restrict__ p) {
    if (st->bad) return;
    float c[kMaxDirs];
#pragma unroll
    for (int j = 0; j < kMaxDirs; ++j) c[j] = j < d.nd ? (float)st->c[j] : 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 v = reinterpret_cast<const float4 *>(z)[i];
#pragma unroll
        for (int j = 0; j < kMaxDirs; ++j)
            if (j < d.nd) {
                const float4 pj = reinterpret_cast<const float4 *>(d.p[j])[i];
                v.x = fmaf(-c[j], pj.x, v.x);
                v.y = fmaf(-c[j], pj.y, v.y);
                v.z = fmaf(-c[j], pj.z, v.z);
                v.w = fmaf(-c[j], pj.w, v.w);
            }
        reinterpret_cast<float4 *>(p)[i] = v;
    }
}

// p.Ap and r.p of the new direction; the last block checks p.Ap > 0
__global__ void __launch_bounds__(kFcgThreads)
    fcg_pdots_kernel(int64_t n4, FcgState *st, double *partials, const float *__restrict__ p,
                     const float *__restrict__ q, const float *__restrict__ r, int slot) {
    float facc[2] = {0.0f, 0.0f};
    for (int64_t i = (int64_t)blockIdx.x * kFcgThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kFcgThreads) {
        const float4 pv = reinterpret_cast<const float4 *>(p)[i];
        facc[0] += dot4f(pv, reinterpret_cast<const float4 *>(q)[i]);
        facc[1] += dot4f(pv, reinterpret_cast<const float4 *>(r)[i]);
    }
    double acc[2] = {(double)facc[0], (double)facc[1]};
    double tot[2];
    if (fcg_reduce<2>(acc, partials, &st->ticket[1], tot) && threadIdx.x == 0) {
        st->pq[slot] = tot[0];
        st->rp = tot[1];
        if (!(tot[0] > 0.0) || !isfinite(tot[0]) || !isfinite(tot[1])) st->bad = st->bad ? st->bad : 1;
    }
}

// alpha = r.p / p.Ap; x += alpha p (FP64); r -= alpha Ap; r.r
__global__ void __launch_bounds__(kFcgThreads)
    fcg_update_kernel(int64_t n4, FcgState *st, double *partials, double *__restrict__ x, const float *__restrict__ p,
                      const float *__restrict__ q, float *__restrict__ r, int slot, double inv_s) {
    if (st->bad) return;  // uniform over the grid: no block reaches the reduction
    const double alpha = st->rp / st->pq[slot];
    const float af = (float)alpha;
    const double ax = alpha * inv_s;  // r, p, q are in the scaled units, x in the caller's
    float facc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kFcgThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kFcgThreads) {
        const float4 pv = reinterpret_cast<const float4 *>(p)[i];
        const float4 qv = reinterpret_cast<const float4 *>(q)[i];
        float4 rv = reinterpret_cast<float4 *>(r)[i];
        double2 *x2 = reinterpret_cast<double2 *>(x) + 2 * i;
        double2 xa = x2[0], xb = x2[1];
        xa.x = fma(ax, (double)pv.x, xa.x);
        xa.y = fma(ax, (double)pv.y, xa.y);
        xb.x = fma(ax, (double)pv.z, xb.x);
        xb.y = fma(ax, (double)pv.w, xb.y);
        x2[0] = xa;
        x2[1] = xb;
        rv.x = fmaf(-af, qv.x, rv.x);
        rv.y = fmaf(-af, qv.y, rv.y);
        rv.z = fmaf(-af, qv.z, rv.z);
        rv.w = fmaf(-af, qv.w, rv.w);
        reinterpret_cast<float4 *>(r)[i] = rv;
        facc += dot4f(rv, rv);
    }
    double acc[1] = {(double)facc};
    double tot[1];
    if (fcg_reduce<1>(acc, partials, &st->ticket[2], tot) && threadIdx.x == 0) st->rr = tot[0];
}

struct FcgLayout {
    int m;  // truncation: directions kept
    size_t state, partials, dotws, r, z, ring, d64, nn, pcg, total;  // ring: (m + 1) x (p, Ap)
};

inline int fcg_depth(const gbpcg_opts &o) { return o.fcg_m == 0 ? 24 : o.fcg_m; }

// ring vector length, rounded so that every vector stays 256-byte aligned
inline size_t align_n4(int64_t n) { return ((size_t)n + 63) / 64 * 64; }

static gbpcg_opts fallback_opts(const gbpcg_opts &o) {
    gbpcg_opts f;
    memset(&f, 0, sizeof(f));
    f.tol = o.tol;
    f.maxit = o.maxit;
    f.precond = GBPCG_PRECOND_JACOBI;
    f.storage = GBPCG_F32;
    f.io_dtype = GBPCG_F64;
    return f;
}

static int fcg_layout(const gbpcg_grid &g, const gbpcg_opts &o, FcgLayout *L) {
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    L->m = fcg_depth(o);
    L->state = take(sizeof(FcgState));
    L->partials = take(sizeof(double) * (kMaxDirs + 1) * kFcgMaxBlocks);
    L->dotws = take(gbpcg_dot_workspace_size());
    L->r = take(n * 4);
    L->z = take(n * 4);
    L->ring = take((size_t)2 * (L->m + 1) * align_n4(n) * 4);
    L->d64 = take(n * 8);
    L->nn = take(nn_layout_total(g.nx, g.ny, g.nz, false));
    gbpcg_opts f = fallback_opts(o);
    size_t pcg_bytes = 0;
    int rc = gbpcg_workspace_size(&g, &f, &pcg_bytes);
    if (rc) return rc;
    L->pcg = take(pcg_bytes);
    L->total = off;
    return GBPCG_OK;
}

static int fcg_check(const gbpcg_grid *g, const gbpcg_opts *o) {
    int rc = check_grid(g);
    if (rc) return rc;
    if (!o) return fail_arg("opts is NULL");
    if (o->precond != GBPCG_PRECOND_LEARNED) return fail_arg("gbpcg_fcg_solve needs opts->precond = LEARNED");
    if (o->io_dtype != GBPCG_F64) return fail_arg("gbpcg_fcg_solve needs FP64 b and x (io_dtype F64)");
    if (o->storage != GBPCG_F32) return fail_arg("gbpcg_fcg_solve iterates in FP32 (storage F32)");
    if (o->flags & GBPCG_FLAG_HOST_IO) return fail_arg("gbpcg_fcg_solve takes device b and x");
    if (!(o->tol > 0.0) || o->maxit < 0) return fail_arg("tol must be > 0 and maxit >= 0");
    if (o->fcg_m < 0 || o->fcg_m > kMaxDirs) return fail_arg("fcg_m must be 0 .. 32");
    if (!nn_shape_ok_ext(g->nx, g->ny, g->nz))
        return fail_arg("learned preconditioner: grid sizes must be multiples of 4 whose levels tile into 128 voxels");
    return GBPCG_OK;
}

static unsigned red_blocks(int64_t n4) {
    const int64_t want = (n4 + kFcgThreads * 8 - 1) / (kFcgThreads * 8);
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>({want, (int64_t)device_sm_count() * 4, (int64_t)kFcgMaxBlocks}));
}

}  // namespace gb

using namespace gb;

extern "C" int gbpcg_fcg_workspace_size(const gbpcg_grid *grid, const gbpcg_opts *opts, size_t *bytes) {
    clear_error();
    if (!bytes) return fail_arg("bytes is NULL");
    int rc = fcg_check(grid, opts);
    if (rc) return rc;
    FcgLayout L;
    rc = fcg_layout(*grid, *opts, &L);
    if (rc) return rc;
    *bytes = L.total;
    return GBPCG_OK;
}

extern "C" int gbpcg_fcg_solve(const gbpcg_grid *grid, const float *w, const void *b_, void *x_,
                               const gbpcg_opts *opts, gbpcg_result *result, gbpcg_stream stream) {
    NvtxRange range("gbpcg_fcg_solve");
    clear_error();
    int rc = fcg_check(grid, opts);
    if (rc) return rc;
    if (!w || !b_ || !x_ || !result) return fail_arg("NULL argument");
    if ((reinterpret_cast<uintptr_t>(b_) | reinterpret_cast<uintptr_t>(x_)) & 15u)
        return fail_arg("b and x must be 16-byte aligned");
    FcgLayout L;
    rc = fcg_layout(*grid, *opts, &L);
    if (rc) return rc;
    if (!opts->workspace || opts->workspace_bytes < L.total) return fail_arg("workspace too small");
    if (reinterpret_cast<uintptr_t>(opts->workspace) & 255u) return fail_arg("workspace must be 256-byte aligned");
    const gbpcg_grid &g = *grid;
    const double *b = static_cast<const double *>(b_);
    double *x = static_cast<double *>(x_);
    cudaStream_t s = (cudaStream_t)stream;
    char *base = static_cast<char *>(opts->workspace);
    FcgState *st = reinterpret_cast<FcgState *>(base + L.state);
    double *partials = reinterpret_cast<double *>(base + L.partials);
    void *dotws = base + L.dotws;
    float *r = reinterpret_cast<float *>(base + L.r), *z = reinterpret_cast<float *>(base + L.z);
    const int m = L.m, nslots = m + 1;
    const size_t vlen = align_n4((int64_t)g.nx * g.ny * g.nz);
    auto ring_p = [&](int slot) { return reinterpret_cast<float *>(base + L.ring) + (size_t)(2 * slot) * vlen; };
    auto ring_q = [&](int slot) { return reinterpret_cast<float *>(base + L.ring) + (size_t)(2 * slot + 1) * vlen; };
    double *d64 = reinterpret_cast<double *>(base + L.d64);
    void *nnws = base + L.nn;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz, n4 = n / 4;
    const size_t dws = gbpcg_dot_workspace_size();
    const unsigned rb = red_blocks(n4);
    const unsigned eb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 16));

    memset(result, 0, sizeof(*result));
    cudaEvent_t e0, e1, n0, n1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    GB_CUDA(cudaEventCreate(&n0));
    GB_CUDA(cudaEventCreate(&n1));
    struct EvGuard {
        cudaEvent_t a, b, c, d;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaEventDestroy(c);
            cudaEventDestroy(d);
        }
    } guard{e0, e1, n0, n1};

    FcgState hs;
    memset(&hs, 0, sizeof(hs));
    int herr = 0;
    auto pull = [&]() -> int {
        GB_CUDA(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(&herr, static_cast<char *>(nnws) + nn_layout_err_offset(), sizeof(int),
                                cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        return GBPCG_OK;
    };
    // The FP32 vectors work on s b (s a power of two bringing rms(b) near 1 when it is far
    // from it), so their products neither underflow nor overflow; x stays in the caller's units.
    double s_rhs = 1.0;
    // r = b - A x in FP64 (d64), its scaled FP32 copy in r, ||r||^2 into st->rr64
    auto true_residual = [&](bool to_r) -> int {
        int rc2 = launch_stencil_f64(g, x, d64, s);
        if (rc2) return rc2;
        fcg_residual_kernel<<<eb, 256, 0, s>>>(n, b, d64, to_r ? r : nullptr, s_rhs);
        GB_CUDA(cudaGetLastError());
        return gbpcg_dot(n, GBPCG_F64, d64, d64, &st->rr64, dotws, dws, stream);
    };
    auto precondition = [&]() -> int {
        NvtxRange net_range("learned preconditioner N(r)");
        GB_CUDA(cudaEventRecord(n0, s));
        int rc2 = nn_forward_ext(g, r, z, nnws, s);
        if (rc2) return rc2;
        GB_CUDA(cudaEventRecord(n1, s));
        return GBPCG_OK;
    };
    double nn_ms = 0.0;
    auto add_nn_time = [&]() {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, n0, n1) == cudaSuccess) nn_ms += ms;
    };
    GB_CUDA(cudaEventRecord(e0, s));
    GB_CUDA(cudaMemsetAsync(st, 0, sizeof(FcgState), s));
    GB_CUDA(cudaMemsetAsync(static_cast<char *>(nnws) + nn_layout_err_offset(), 0, sizeof(int), s));
    rc = nn_prep_ext(w, nnws, g, s);
    if (rc) return rc;
    rc = gbpcg_dot(n, GBPCG_F64, b, b, &st->bb, dotws, dws, stream);
    if (rc) return rc;
    rc = pull();
    if (rc) return rc;
    if (hs.bb > 0.0 && std::isfinite(hs.bb)) {
        int e = 0;
        std::frexp(std::sqrt(hs.bb / (double)n), &e);
        if (e < -20 || e > 20) s_rhs = std::ldexp(1.0, -e);
    }
    rc = true_residual(true);
    if (rc) return rc;
    rc = pull();
    if (rc) return rc;
    const double bb = hs.bb;
    int status = GBPCG_NOT_CONVERGED, iters = 0, fcg_iters = 0, replacements = 0;
    double rel = bb > 0.0 ? std::sqrt(hs.rr64 / bb) : 0.0, rel_true = rel;
    bool fallback = false;
    if (bb == 0.0) {
        GB_CUDA(cudaMemsetAsync(x, 0, n * 8, s));
        rel = rel_true = 0.0;
        status = GBPCG_OK;
    } else if (rel <= opts->tol) {
        status = GBPCG_OK;
    } else {
        std::vector<double> hist{rel};
        int nd = 0, cur = 0;  // directions in the window; ring slot of the next one
        while (iters < opts->maxit) {
            NvtxRange it_range("fcg iteration");
            DirSet d;
            memset(&d, 0, sizeof(d));
            d.nd = nd;
            for (int j = 0; j < nd; ++j) {  // oldest first
                const int sl = ((cur - nd + j) % nslots + nslots) % nslots;
                d.p[j] = ring_p(sl);
                d.q[j] = ring_q(sl);
                d.slot[j] = sl;
            }
            float *p = ring_p(cur), *q = ring_q(cur);
            rc = precondition();
            if (rc) return rc;
            fcg_mdot_kernel<<<rb, kFcgThreads, 0, s>>>(n4, st, partials, r, z, d);
            GB_CUDA(cudaGetLastError());
            fcg_combine_kernel<<<eb, 256, 0, s>>>(n4, st, z, d, p);
            GB_CUDA(cudaGetLastError());
            rc = gbpcg_stencil_apply(&g, GBPCG_F32, p, q, stream);
            if (rc) return rc;
            fcg_pdots_kernel<<<rb, kFcgThreads, 0, s>>>(n4, st, partials, p, q, r, cur);
            GB_CUDA(cudaGetLastError());
            fcg_update_kernel<<<rb, kFcgThreads, 0, s>>>(n4, st, partials, x, p, q, r, cur, 1.0 / s_rhs);
            GB_CUDA(cudaGetLastError());
            rc = pull();
            if (rc) return rc;
            add_nn_time();
            if (hs.bad || herr) {  // x and r untouched: this iteration did not happen
                fallback = true;
                break;
            }
            ++iters;
            ++fcg_iters;
            nd = std::min(nd + 1, m);
            cur = (cur + 1) % nslots;
            rel = std::sqrt(hs.rr / bb) / s_rhs;  // hs.rr is ||s r||^2
            hist.push_back(rel);
            if (!std::isfinite(rel)) {
                fallback = true;
                break;
            }
            if (rel <= opts->tol) {
                rc = true_residual(true);
                if (rc) return rc;
                rc = pull();
                if (rc) return rc;
                rel_true = std::sqrt(hs.rr64 / bb);
                if (rel_true <= opts->tol) {
                    status = GBPCG_OK;
                    break;
                }
                ++replacements;
                nd = 0;  // restart from the replaced residual
                continue;
            }
            if (hist.size() > 5 && rel > 10.0 * hist[hist.size() - 6]) {
                fallback = true;
                break;
            }
        }
    }
    int fb_iters = 0;
    if (fallback) {
        gbpcg_opts f = fallback_opts(*opts);
        f.maxit = std::max(0, opts->maxit - iters);
        f.workspace = base + L.pcg;
        f.workspace_bytes = opts->workspace_bytes - L.pcg;
        gbpcg_result fr;
        rc = gbpcg_pcg_solve(&g, b, x, &f, &fr, stream);
        if (rc == GBPCG_ERR_ARG || rc == GBPCG_ERR_CUDA) return rc;
        fb_iters = fr.iters;
        iters += fr.iters;
        rel = fr.rel_res_recursive;
        rel_true = fr.rel_res_true;
        replacements += fr.replacements;
        status = fr.status == GBPCG_OK ? GBPCG_FALLBACK_USED : fr.status;
    } else if (status != GBPCG_OK) {
        rc = true_residual(false);
        if (rc) return rc;
        rc = pull();
        if (rc) return rc;
        rel_true = std::sqrt(hs.rr64 / bb);
    }
    GB_CUDA(cudaEventRecord(e1, s));
    GB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    result->iters = iters;
    result->status = status;
    result->rel_res_recursive = rel;
    result->rel_res_true = rel_true;
    result->time_ms = ms;
    result->pass_ms[0] = nn_ms;
    result->pass_ms[1] = ms - nn_ms;
    result->pass_launches[0] = fcg_iters;
    result->pass_launches[1] = fb_iters;
    result->replacements = replacements;
    result->refine_steps = 0;
    return status;
}
