// Variants that mirror the paper's own experiments on GB300 (none of them is
// on the solver's default path):
//
//   Sec. V    reduction granularity and finish of the dot product: one scalar
//             per CTA (the paper's Method 1) or one per warp (Method 2), added
//             up by the last CTA to arrive, by a second kernel, by FP64
//             atomics, or by a two-level tree of last-arriving CTAs (the
//             analogue of routing partial sums towards the centre, Route 2).
//   Sec. VI-C boundary handling of the stencil: TMA out-of-bounds zero fill,
//             plain loads with explicit bounds checks, or TMA followed by an
//             explicit zero fill of the out-of-grid part of every box.
//   Sec. VII  the paper's FP32 solver: split kernels (stencil, dot, axpy,
//             element-wise scaling) with the scalars read back to the host
//             every iteration (split_solve below, GBPCG_FLAG_SPLIT).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "launch.cuh"

namespace gb {

// ------------------------------------------------ Sec. V: dot variants --

constexpr int kRvThreads = 256;
constexpr int kRvWarps = kRvThreads / 32;
constexpr unsigned kRvMaxBlocks = 8192;
constexpr unsigned kRvGroup = 32;  // CTAs per group of the two-level finish
constexpr unsigned kRvGroups = kRvMaxBlocks / kRvGroup;
// workspace: tickets (one per group, one on top), then partials (one per warp
// of every CTA at most), then group totals, then an atomic accumulator
constexpr size_t kRvTicketBytes = 2048;
constexpr size_t kRvPartialOff = kRvTicketBytes;
constexpr size_t kRvGroupOff = kRvPartialOff + sizeof(double) * kRvWarps * kRvMaxBlocks;
constexpr size_t kRvAccOff = kRvGroupOff + sizeof(double) * kRvGroups;
constexpr size_t kRvWorkspace = kRvAccOff + 256;
static_assert(sizeof(unsigned) * (kRvGroups + 1) <= kRvTicketBytes, "ticket area");

enum DotVariant { DV_CTA_LAST = 0, DV_WARP_LAST = 1, DV_CTA_KERNEL = 2, DV_CTA_ATOMIC = 3, DV_CTA_TREE = 4, DV_COUNT };

// Per-thread part of x.y, streamed as gbpcg_dot streams it (four 16-byte
// vectors of each input in flight per thread, FP32 sums of 8 products added
// into an FP64 accumulator), so the variants differ only in the reduction.
// x, y 16-byte aligned.
__device__ __forceinline__ float dot4v(const float4 a, const float4 b, float s) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
}
__device__ __forceinline__ double thread_dot(int64_t n, const float *__restrict__ x, const float *__restrict__ y) {
    const int64_t tid = (int64_t)blockIdx.x * kRvThreads + threadIdx.x, nth = (int64_t)gridDim.x * kRvThreads;
    const float4 *x4 = reinterpret_cast<const float4 *>(x), *y4 = reinterpret_cast<const float4 *>(y);
    double acc = 0.0;
    const int64_t n4 = n / 4;
    int64_t i = tid;
    for (; i + 3 * nth < n4; i += 4 * nth) {
        const float4 a0 = x4[i], a1 = x4[i + nth], a2 = x4[i + 2 * nth], a3 = x4[i + 3 * nth];
        const float4 b0 = y4[i], b1 = y4[i + nth], b2 = y4[i + 2 * nth], b3 = y4[i + 3 * nth];
        acc += (double)dot4v(a1, b1, dot4v(a0, b0, 0.f));
        acc += (double)dot4v(a3, b3, dot4v(a2, b2, 0.f));
    }
    for (; i < n4; i += nth) acc += (double)dot4v(x4[i], y4[i], 0.f);
    for (int64_t j = 4 * n4 + tid; j < n; j += nth) acc += (double)(x[j] * y[j]);
    return acc;
}

// Fixed-order sum of cnt doubles by one CTA; valid in thread 0.
__device__ __forceinline__ double cta_sum_fixed(const double *v, unsigned cnt) {
    __shared__ double red[kRvWarps];
    double s = 0.0;
    for (unsigned j = threadIdx.x; j < cnt; j += kRvThreads) s += __ldcg(v + j);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRvWarps; ++w) t += red[w];
    __syncthreads();
    return t;
}

template <int VARIANT>
__global__ void __launch_bounds__(kRvThreads)
    dot_variant_kernel(int64_t n, const float *__restrict__ x, const float *__restrict__ y, char *ws, double *out) {
    unsigned *tickets = reinterpret_cast<unsigned *>(ws);
    double *partials = reinterpret_cast<double *>(ws + kRvPartialOff);
    double *groups = reinterpret_cast<double *>(ws + kRvGroupOff);
    double *acc = reinterpret_cast<double *>(ws + kRvAccOff);
    const unsigned bid = blockIdx.x, nblk = gridDim.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double s = warp_sum(thread_dot(n, x, y));
    __shared__ double red[kRvWarps];
    __shared__ bool last;
    if constexpr (VARIANT == DV_WARP_LAST) {
        // every warp publishes its own partial: kRvWarps times the partials of one per CTA
        if (lane == 0) partials[(size_t)bid * kRvWarps + w] = s;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(&tickets[0], 1u) == nblk - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
        const double t = cta_sum_fixed(partials, nblk * kRvWarps);
        if (threadIdx.x == 0) {
            *out = t;
            tickets[0] = 0;
        }
        return;
    } else {
        if (lane == 0) red[w] = s;
        __syncthreads();
        double part = 0.0;
        if (threadIdx.x == 0)
            for (int j = 0; j < kRvWarps; ++j) part += red[j];
        if constexpr (VARIANT == DV_CTA_ATOMIC) {
            if (threadIdx.x == 0) atomicAdd(acc, part);  // summation order varies from run to run
            return;
        } else {
            if (threadIdx.x == 0) {
                partials[bid] = part;
                __threadfence();
            }
            if constexpr (VARIANT == DV_CTA_KERNEL) return;  // a second kernel adds the partials
            if constexpr (VARIANT == DV_CTA_LAST) {
                if (threadIdx.x == 0) last = atomicAdd(&tickets[0], 1u) == nblk - 1;
                __syncthreads();
                if (!last) return;
                __threadfence();
                const double t = cta_sum_fixed(partials, nblk);
                if (threadIdx.x == 0) {
                    *out = t;
                    tickets[0] = 0;
                }
                return;
            }
            if constexpr (VARIANT == DV_CTA_TREE) {
                // the last CTA of each group of kRvGroup adds that group; the last group to
                // finish adds the group totals
                const unsigned g = bid / kRvGroup, g0 = g * kRvGroup;
                const unsigned gsize = min(kRvGroup, nblk - g0), ngroups = (nblk + kRvGroup - 1) / kRvGroup;
                if (threadIdx.x == 0) last = atomicAdd(&tickets[1 + g], 1u) == gsize - 1;
                __syncthreads();
                if (!last) return;
                __threadfence();
                const double t = cta_sum_fixed(partials + g0, gsize);
                __shared__ bool top;
                if (threadIdx.x == 0) {
                    groups[g] = t;
                    tickets[1 + g] = 0;
                    __threadfence();
                    top = atomicAdd(&tickets[0], 1u) == ngroups - 1;
                }
                __syncthreads();
                if (!top) return;
                __threadfence();
                const double tt = cta_sum_fixed(groups, ngroups);
                if (threadIdx.x == 0) {
                    *out = tt;
                    tickets[0] = 0;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kRvThreads) dot_finish_kernel(const char *ws, unsigned nblk, double *out) {
    const double t = cta_sum_fixed(reinterpret_cast<const double *>(ws + kRvPartialOff), nblk);
    if (threadIdx.x == 0) *out = t;
}

__global__ void acc_to_out_kernel(const char *ws, double *out) {
    *out = *reinterpret_cast<const double *>(ws + kRvAccOff);
}

// ------------------------------------ Sec. VI-C: stencil boundary variants --

constexpr int kBvCfg = CFG_64x16;  // the stencil apply's configuration for grids wider than 32

template <bool TMA, bool ZFILL>
static int stencil_variant_launch(const gbpcg_grid &g, const float *p, float *q, cudaStream_t s) {
    using K = PassKernel<float, 64, 16, 4, K_STENCIL, TMA, OpConst>;
    auto *fn = &zmarch_kernel<float, 64, 16, 4, K_STENCIL, TMA, OpConst, ZFILL>;
    GB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem));
    int occ = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, K::threads, K::smem));
    const PassGeom geo = make_geom(kBvCfg, g.nx, g.ny, g.nz, std::max(occ, 1), K::smem);
    PassArgs a{};
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.h0[0] = a.h0[1] = a.h1[0] = a.h1[1] = a.c0 = p;
    a.o0[0] = a.o0[1] = a.o1 = q;
    a.scale = 1.0f;
    a.tiles_x = geo.tiles_x;
    a.zchunk = geo.zchunk;
    PassMaps maps;
    memset(&maps, 0, sizeof(maps));
    if (TMA) {
        if (int rc = make_pass_map<float>(&maps.h0[0], kBvCfg, true, p, g.nx, g.ny, g.nz)) return rc;
        maps.h0[1] = maps.h1[0] = maps.h1[1] = maps.c0 = maps.h0[0];
    }
    fn<<<geo.grid(), K::threads, K::smem, s>>>(maps, a, make_op_const(g.nx, g.ny, g.nz));
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

// ---------------------------------------- Sec. VII: split-kernel FP32 PCG --

// z = c r
__global__ void __launch_bounds__(256) scale_kernel(int64_t n, float c, const float *__restrict__ r, float *__restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) z[i] = c * r[i];
}
// p = z + beta p
__global__ void __launch_bounds__(256) xpay_kernel(int64_t n, const float *__restrict__ z, float beta, float *p) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
        p[i] = fmaf(beta, p[i], z[i]);
}
// r = b - q
__global__ void __launch_bounds__(256) sub_kernel(int64_t n, const float *__restrict__ b, const float *__restrict__ q,
                                                  float *__restrict__ r) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) r[i] = b[i] - q[i];
}

struct SplitLayout {
    size_t dots, dotws, r, z, p, q, total;
};

static SplitLayout split_layout(int64_t n) {
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    SplitLayout L;
    size_t o = 0;
    L.dots = o; o += 256;
    L.dotws = o; o += up(gbpcg_dot_workspace_size());
    L.r = o; o += up((size_t)n * 4);
    L.z = o; o += up((size_t)n * 4);
    L.p = o; o += up((size_t)n * 4);
    L.q = o; o += up((size_t)n * 4);
    L.total = o;
    return L;
}

size_t split_workspace_size(const gbpcg_grid &g) { return split_layout((int64_t)g.nx * g.ny * g.nz).total; }

// Textbook Jacobi-PCG with one kernel per operation and the host holding
// the scalars: per iteration q = A p; p.q (read back: alpha); x += alpha p;
// r -= alpha q; z = D^-1 r; r.z and r.r (read back: beta and the
// convergence test); p = z + beta p.  Eight launches and two host round
// trips per iteration, 76 bytes per point.  FP32 b and x, constant
// coefficient.
int split_solve(const gbpcg_grid &g, const float *b, float *x, const gbpcg_opts &o, gbpcg_result *res,
                cudaStream_t s) {
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const SplitLayout L = split_layout(n);
    char *ws = static_cast<char *>(o.workspace);
    double *dots = reinterpret_cast<double *>(ws + L.dots);
    void *dws = ws + L.dotws;
    const size_t dwb = gbpcg_dot_workspace_size();
    float *r = reinterpret_cast<float *>(ws + L.r), *z = reinterpret_cast<float *>(ws + L.z),
          *p = reinterpret_cast<float *>(ws + L.p), *q = reinterpret_cast<float *>(ws + L.q);
    const OpConst op = make_op_const(g.nx, g.ny, g.nz);
    const float inv_d = op.inv_d;
    const unsigned eb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)device_sm_count() * 8));
    gbpcg_stream st = reinterpret_cast<gbpcg_stream>(s);
    double h[3];
    auto pull = [&](int cnt) -> int {
        GB_CUDA(cudaMemcpyAsync(h, dots, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        return GBPCG_OK;
    };
#define GB_SPLIT_TRY(expr)                 \
    do {                                   \
        int _r = (expr);                   \
        if (_r != GBPCG_OK) return _r;     \
    } while (0)
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } guard{e0, e1};
    GB_CUDA(cudaEventRecord(e0, s));
    // r = b - A x, z = D^-1 r, p = z
    GB_SPLIT_TRY(gbpcg_stencil_apply(&g, GBPCG_F32, x, q, st));
    sub_kernel<<<eb, 256, 0, s>>>(n, b, q, r);
    scale_kernel<<<eb, 256, 0, s>>>(n, inv_d, r, z);
    GB_CUDA(cudaMemcpyAsync(p, z, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    GB_SPLIT_TRY(gbpcg_dot(n, GBPCG_F32, r, z, dots + 0, dws, dwb, st));
    GB_SPLIT_TRY(gbpcg_dot(n, GBPCG_F32, r, r, dots + 1, dws, dwb, st));
    GB_SPLIT_TRY(gbpcg_dot(n, GBPCG_F32, b, b, dots + 2, dws, dwb, st));
    GB_SPLIT_TRY(pull(3));
    double rz = h[0], rr = h[1];
    const double bb = h[2];
    int it = 0, status = GBPCG_NOT_CONVERGED;
    const double tol2 = o.tol * o.tol;
    if (bb == 0.0) {
        GB_CUDA(cudaMemsetAsync(x, 0, (size_t)n * 4, s));
        status = GBPCG_OK;
        rr = 0.0;
    } else if (rr <= tol2 * bb) {
        status = GBPCG_OK;
    }
    while (status == GBPCG_NOT_CONVERGED && it < o.maxit) {
        GB_SPLIT_TRY(gbpcg_stencil_apply(&g, GBPCG_F32, p, q, st));
        GB_SPLIT_TRY(gbpcg_dot(n, GBPCG_F32, p, q, dots + 0, dws, dwb, st));
        GB_SPLIT_TRY(pull(1));
        const double pq = h[0];
        if (!(pq > 0.0) || !std::isfinite(pq)) { status = GBPCG_BREAKDOWN; break; }
        const double alpha = rz / pq;
        GB_SPLIT_TRY(gbpcg_axpy(n, GBPCG_F32, alpha, p, x, st));
        GB_SPLIT_TRY(gbpcg_axpy(n, GBPCG_F32, -alpha, q, r, st));
        scale_kernel<<<eb, 256, 0, s>>>(n, inv_d, r, z);
        GB_SPLIT_TRY(gbpcg_dot(n, GBPCG_F32, r, z, dots + 0, dws, dwb, st));
        GB_SPLIT_TRY(gbpcg_dot(n, GBPCG_F32, r, r, dots + 1, dws, dwb, st));
        GB_SPLIT_TRY(pull(2));
        ++it;
        const double rz_new = h[0];
        rr = h[1];
        if (!std::isfinite(rr) || !(rz_new > 0.0)) { status = GBPCG_BREAKDOWN; break; }
        if (rr <= tol2 * bb) { status = GBPCG_OK; break; }
        const double beta = rz_new / rz;
        rz = rz_new;
        xpay_kernel<<<eb, 256, 0, s>>>(n, z, (float)beta, p);
    }
#undef GB_SPLIT_TRY
    GB_CUDA(cudaGetLastError());
    GB_CUDA(cudaEventRecord(e1, s));
    GB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    res->iters = it;
    res->status = status;
    res->rel_res_recursive = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    res->rel_res_true = 0.0;  // not evaluated: the caller holds FP32 x and b
    res->time_ms = ms;
    return status;
}

}  // namespace gb

using namespace gb;

extern "C" {

size_t gbpcg_dot_variant_workspace_size(void) { return kRvWorkspace; }

int gbpcg_dot_variant(int32_t variant, int64_t n, const float *x, const float *y, double *result, void *workspace,
                      size_t workspace_bytes, gbpcg_stream stream) {
    clear_error();
    if (variant < 0 || variant >= DV_COUNT) return fail_arg("unknown reduction variant");
    if (n <= 0) return fail_arg("n must be positive");
    if (!x || !y || !result) return fail_arg("x, y and result must be non-NULL");
    if (((uintptr_t)x | (uintptr_t)y) & 15u) return fail_arg("x and y must be 16-byte aligned");
    if (!workspace || workspace_bytes < kRvWorkspace || ((uintptr_t)workspace & 255u))
        return fail_arg("workspace: gbpcg_dot_variant_workspace_size() bytes, 256-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const int64_t want = (n + (int64_t)kRvThreads * 16 - 1) / ((int64_t)kRvThreads * 16);
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)device_sm_count() * 8, (int64_t)kRvMaxBlocks}));
    // tickets (and the atomic accumulator) start at zero in every variant
    GB_CUDA(cudaMemsetAsync(ws, 0, kRvTicketBytes, s));
    switch (variant) {
        case DV_CTA_LAST: dot_variant_kernel<DV_CTA_LAST><<<blocks, kRvThreads, 0, s>>>(n, x, y, ws, result); break;
        case DV_WARP_LAST: dot_variant_kernel<DV_WARP_LAST><<<blocks, kRvThreads, 0, s>>>(n, x, y, ws, result); break;
        case DV_CTA_KERNEL:
            dot_variant_kernel<DV_CTA_KERNEL><<<blocks, kRvThreads, 0, s>>>(n, x, y, ws, result);
            dot_finish_kernel<<<1, kRvThreads, 0, s>>>(ws, blocks, result);
            break;
        case DV_CTA_ATOMIC:
            GB_CUDA(cudaMemsetAsync(ws + kRvAccOff, 0, sizeof(double), s));
            dot_variant_kernel<DV_CTA_ATOMIC><<<blocks, kRvThreads, 0, s>>>(n, x, y, ws, result);
            acc_to_out_kernel<<<1, 1, 0, s>>>(ws, result);
            break;
        default: dot_variant_kernel<DV_CTA_TREE><<<blocks, kRvThreads, 0, s>>>(n, x, y, ws, result); break;
    }
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

int gbpcg_stencil_apply_variant(const gbpcg_grid *grid, int32_t variant, const float *p, float *q,
                                gbpcg_stream stream) {
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (grid->k_block) return fail_arg("boundary variants take the constant-coefficient operator");
    if (!p || !q || p == q) return fail_arg("p and q must be distinct non-NULL device pointers");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool tma = tma_ok(sizeof(float), grid->nx, {p, q});
    switch (variant) {
        case 0:
            if (!tma) return fail_arg("TMA variant needs 16-byte aligned arrays with nx a multiple of 4");
            return stencil_variant_launch<true, false>(*grid, p, q, s);
        case 1: return stencil_variant_launch<false, false>(*grid, p, q, s);
        case 2:
            if (!tma) return fail_arg("TMA variant needs 16-byte aligned arrays with nx a multiple of 4");
            return stencil_variant_launch<true, true>(*grid, p, q, s);
        default: return fail_arg("unknown boundary variant");
    }
}

}  // extern "C"
