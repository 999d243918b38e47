// Element-wise axpy (Sec. IV) and the global dot-product reduction (Sec. V).
//
// dot: every thread streams its share with 16-byte loads and forms FP32 sums
// of 8 products, which it adds into an FP64 accumulator; warps reduce with
// shuffles, blocks publish one FP64 partial each, and the last block to
// arrive (atomic ticket) adds the partials in block order -- one pass over
// the data, one launch, a bitwise-reproducible result (the GPU analogue of
// the paper's "reduce locally, then forward one partial" routing).
#include <algorithm>
#include <mutex>

#include "launch.cuh"

namespace gb {

constexpr int kDotThreads = 256;
constexpr unsigned kDotMaxBlocks = 8192;
constexpr size_t kDotWorkspace = 256 + sizeof(double) * kDotMaxBlocks;

__device__ __forceinline__ float dot4(const float a[4], const float b[4], float s) {
    s = fmaf(a[0], b[0], s);
    s = fmaf(a[1], b[1], s);
    s = fmaf(a[2], b[2], s);
    return fmaf(a[3], b[3], s);
}

template <typename T>
__global__ void __launch_bounds__(kDotThreads)
    dot_kernel(int64_t n, const T *__restrict__ x, const T *__restrict__ y, double *partials, unsigned *ticket,
               double *out, int vec) {
    const int64_t tid = (int64_t)blockIdx.x * kDotThreads + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kDotThreads;
    double acc = 0.0;
    int64_t tail0 = 0;
    if (vec) {
        const int64_t n4 = n / 4;
        int64_t i = tid;
        for (; i + 3 * nth < n4; i += 4 * nth) {
            float a0[4], a1[4], a2[4], a3[4], b0[4], b1[4], b2[4], b3[4];
            ld4<T>(x + 4 * i, a0);
            ld4<T>(x + 4 * (i + nth), a1);
            ld4<T>(x + 4 * (i + 2 * nth), a2);
            ld4<T>(x + 4 * (i + 3 * nth), a3);
            ld4<T>(y + 4 * i, b0);
            ld4<T>(y + 4 * (i + nth), b1);
            ld4<T>(y + 4 * (i + 2 * nth), b2);
            ld4<T>(y + 4 * (i + 3 * nth), b3);
            acc += (double)dot4(a1, b1, dot4(a0, b0, 0.f));
            acc += (double)dot4(a3, b3, dot4(a2, b2, 0.f));
        }
        for (; i < n4; i += nth) {
            float a0[4], b0[4];
            ld4<T>(x + 4 * i, a0);
            ld4<T>(y + 4 * i, b0);
            acc += (double)dot4(a0, b0, 0.f);
        }
        tail0 = 4 * n4;
    }
    for (int64_t j = tail0 + tid; j < n; j += nth) acc += (double)(to_f(x[j]) * to_f(y[j]));

    __shared__ double red[kDotThreads / 32];
    double s = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double part[1] = {0.0}, tot[1];
    if (threadIdx.x == 0)
        for (int w = 0; w < kDotThreads / 32; ++w) part[0] += red[w];
    if (grid_sum_last<1, kDotThreads>(part, partials, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

__global__ void __launch_bounds__(kDotThreads)
    dot_f64_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y, double *partials,
                   unsigned *ticket, double *out) {
    const int64_t tid = (int64_t)blockIdx.x * kDotThreads + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kDotThreads;
    double acc = 0.0;
    for (int64_t j = tid; j < n; j += nth) acc = fma(__ldg(x + j), __ldg(y + j), acc);
    __shared__ double red[kDotThreads / 32];
    double s = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double part[1] = {0.0}, tot[1];
    if (threadIdx.x == 0)
        for (int w = 0; w < kDotThreads / 32; ++w) part[0] += red[w];
    if (grid_sum_last<1, kDotThreads>(part, partials, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

template <typename T>
__global__ void __launch_bounds__(256) axpy_kernel(int64_t n, float alpha, const T *__restrict__ x, T *__restrict__ y,
                                                   int vec) {
    const int64_t tid = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * 256;
    int64_t tail0 = 0;
    if (vec) {
        const int64_t n4 = n / 4;
        int64_t i = tid;
        for (; i + 3 * nth < n4; i += 4 * nth) {
            float a[4][4], b[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ld4<T>(x + 4 * (i + u * nth), a[u]);
                ld4<T>(y + 4 * (i + u * nth), b[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int e = 0; e < 4; ++e) b[u][e] = fmaf(alpha, a[u][e], b[u][e]);
                st4<T>(y + 4 * (i + u * nth), b[u]);
            }
        }
        for (; i < n4; i += nth) {
            float a[4], b[4];
            ld4<T>(x + 4 * i, a);
            ld4<T>(y + 4 * i, b);
#pragma unroll
            for (int e = 0; e < 4; ++e) b[e] = fmaf(alpha, a[e], b[e]);
            st4<T>(y + 4 * i, b);
        }
        tail0 = 4 * n4;
    }
    for (int64_t j = tail0 + tid; j < n; j += nth) y[j] = from_f<T>(fmaf(alpha, to_f(x[j]), to_f(y[j])));
}

__global__ void __launch_bounds__(256) axpy_f64_kernel(int64_t n, double alpha, const double *__restrict__ x,
                                                       double *__restrict__ y) {
    const int64_t tid = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * 256;
    for (int64_t j = tid; j < n; j += nth) y[j] = fma(alpha, x[j], y[j]);
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T>
static int dot_typed(int64_t n, const void *x, const void *y, double *out, void *ws, cudaStream_t s) {
    unsigned *ticket = static_cast<unsigned *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + 256);
    // 8 elements per thread per round trip is plenty; cap at 4 blocks per SM slot
    const int64_t want = (n + (int64_t)kDotThreads * 16 - 1) / ((int64_t)kDotThreads * 16);
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)device_sm_count() * 8, (int64_t)kDotMaxBlocks}));
    GB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    const int vec = sizeof(T) == 4 ? (aligned16(x) && aligned16(y)) : (((uintptr_t)x | (uintptr_t)y) & 7u) == 0;
    dot_kernel<T><<<blocks, kDotThreads, 0, s>>>(n, static_cast<const T *>(x), static_cast<const T *>(y), partials,
                                                 ticket, out, vec);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

template <typename T>
static int axpy_typed(int64_t n, double alpha, const void *x, void *y, cudaStream_t s) {
    const int64_t want = (n + 256 * 16 - 1) / (256 * 16);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)device_sm_count() * 8));
    const int vec = sizeof(T) == 4 ? (aligned16(x) && aligned16(y)) : (((uintptr_t)x | (uintptr_t)y) & 7u) == 0;
    axpy_kernel<T><<<blocks, 256, 0, s>>>(n, (float)alpha, static_cast<const T *>(x), static_cast<T *>(y), vec);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

// ------------------------------------------------ dot without allocation --
//
// Scratch for gbpcg_dot_noalloc lives in this file-scope device array: a
// ticket word (first 256 bytes) and one FP64 partial sum per block.  The
// array exists once per GPU that loads the library and stays until the
// process exits.  The grid is sized like gbpcg_dot's (at most 8 blocks per
// SM, each thread striding over the vector), and never beyond the
// kNoAllocMaxBlocks partial slots the array holds.
constexpr unsigned kNoAllocMaxBlocks = 16384;
constexpr int64_t kNoAllocMaxN = (int64_t)1 << 30;
constexpr size_t kNoAllocScratchBytes = 256 + sizeof(double) * kNoAllocMaxBlocks;

static __device__ __align__(256) unsigned char g_dot_scratch[kNoAllocScratchBytes];

// Host code cannot use g_dot_scratch's name as a device address; the real
// address is fetched once per device (with that device current) and cached.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64] = {nullptr};

static int noalloc_scratch(void **out) {
    int dev = -1;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail_arg("device ordinal out of range for the static scratch table");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(g_dot_scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return GBPCG_OK;
}

// Blocks of one allocation-free dot: per_block elements per block, at most
// 8 per SM (the kernels stride over the rest) and never more than the
// array's partial slots.
static unsigned noalloc_blocks(int64_t n, int64_t per_block) {
    const int64_t want = (n + per_block - 1) / per_block;
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>({want, (int64_t)device_sm_count() * 8, (int64_t)kNoAllocMaxBlocks}));
}

template <typename T>
static int dot_noalloc_typed(int64_t n, const void *x, const void *y, double *out, void *scratch, cudaStream_t s) {
    unsigned *ticket = static_cast<unsigned *>(scratch);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(scratch) + 256);
    const unsigned blocks = noalloc_blocks(n, (int64_t)kDotThreads * 16);
    // the array keeps the previous call's contents: the ticket must restart at zero
    GB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    const int vec = sizeof(T) == 4 ? (aligned16(x) && aligned16(y)) : (((uintptr_t)x | (uintptr_t)y) & 7u) == 0;
    dot_kernel<T><<<blocks, kDotThreads, 0, s>>>(n, static_cast<const T *>(x), static_cast<const T *>(y), partials,
                                                 ticket, out, vec);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

size_t gbpcg_dot_workspace_size(void) { return kDotWorkspace; }

int gbpcg_dot(int64_t n, int32_t dtype, const void *x, const void *y, double *result, void *workspace,
              size_t workspace_bytes, gbpcg_stream stream) {
    clear_error();
    if (n < 0) return fail_arg("n must be >= 0");
    if (!result) return fail_arg("result must be a device pointer");
    if (!workspace || workspace_bytes < kDotWorkspace) return fail_arg("workspace smaller than gbpcg_dot_workspace_size()");
    if (reinterpret_cast<uintptr_t>(workspace) & 15u) return fail_arg("workspace must be 16-byte aligned");
    if (n > 0 && (!x || !y)) return fail_arg("x and y must be non-NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) {
        GB_CUDA(cudaMemsetAsync(result, 0, sizeof(double), s));
        return GBPCG_OK;
    }
    switch (dtype) {
        case GBPCG_F32: return dot_typed<float>(n, x, y, result, workspace, s);
        case GBPCG_BF16: return dot_typed<__nv_bfloat16>(n, x, y, result, workspace, s);
        case GBPCG_F16: return dot_typed<__half>(n, x, y, result, workspace, s);
        case GBPCG_F64: {
            unsigned *ticket = static_cast<unsigned *>(workspace);
            double *partials = reinterpret_cast<double *>(static_cast<char *>(workspace) + 256);
            const int64_t want = (n + kDotThreads * 8 - 1) / (kDotThreads * 8);
            const unsigned blocks = (unsigned)std::max<int64_t>(
                1, std::min<int64_t>({want, (int64_t)device_sm_count() * 8, (int64_t)kDotMaxBlocks}));
            GB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
            dot_f64_kernel<<<blocks, kDotThreads, 0, s>>>(n, static_cast<const double *>(x),
                                                         static_cast<const double *>(y), partials, ticket, result);
            GB_CUDA(cudaGetLastError());
            return GBPCG_OK;
        }
        default: return fail_arg("unknown dtype");
    }
}

int gbpcg_axpy(int64_t n, int32_t dtype, double alpha, const void *x, void *y, gbpcg_stream stream) {
    clear_error();
    if (n < 0) return fail_arg("n must be >= 0");
    if (n == 0) return GBPCG_OK;
    if (!x || !y) return fail_arg("x and y must be non-NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (dtype) {
        case GBPCG_F32: return axpy_typed<float>(n, alpha, x, y, s);
        case GBPCG_BF16: return axpy_typed<__nv_bfloat16>(n, alpha, x, y, s);
        case GBPCG_F16: return axpy_typed<__half>(n, alpha, x, y, s);
        case GBPCG_F64: {
            const int64_t want = (n + 256 * 8 - 1) / (256 * 8);
            const unsigned blocks =
                (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)device_sm_count() * 8));
            axpy_f64_kernel<<<blocks, 256, 0, s>>>(n, alpha, static_cast<const double *>(x), static_cast<double *>(y));
            GB_CUDA(cudaGetLastError());
            return GBPCG_OK;
        }
        default: return fail_arg("unknown dtype");
    }
}

int gbpcg_dot_noalloc(int64_t n, int32_t dtype, const void *x, const void *y, double *result, gbpcg_stream stream) {
    clear_error();
    if (n < 0) return fail_arg("n must be >= 0");
    if (n > kNoAllocMaxN)
        return fail_arg("n = " + std::to_string(n) + " exceeds gbpcg_dot_noalloc's static scratch limit of " +
                        std::to_string(kNoAllocMaxN) + " elements; use gbpcg_dot with a workspace");
    if (!result) return fail_arg("result must be a device pointer");
    if (n > 0 && (!x || !y)) return fail_arg("x and y must be non-NULL");
    if (dtype != GBPCG_F32 && dtype != GBPCG_BF16 && dtype != GBPCG_F16 && dtype != GBPCG_F64)
        return fail_arg("unknown dtype");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    if (int rc = noalloc_scratch(&scratch)) return rc;
    if (n == 0) {
        GB_CUDA(cudaMemsetAsync(result, 0, sizeof(double), s));
        return GBPCG_OK;
    }
    switch (dtype) {
        case GBPCG_F32: return dot_noalloc_typed<float>(n, x, y, result, scratch, s);
        case GBPCG_BF16: return dot_noalloc_typed<__nv_bfloat16>(n, x, y, result, scratch, s);
        case GBPCG_F16: return dot_noalloc_typed<__half>(n, x, y, result, scratch, s);
        default: {
            unsigned *ticket = static_cast<unsigned *>(scratch);
            double *partials = reinterpret_cast<double *>(static_cast<char *>(scratch) + 256);
            const unsigned blocks = noalloc_blocks(n, (int64_t)kDotThreads * 8);
            GB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
            dot_f64_kernel<<<blocks, kDotThreads, 0, s>>>(n, static_cast<const double *>(x),
                                                         static_cast<const double *>(y), partials, ticket, result);
            GB_CUDA(cudaGetLastError());
            return GBPCG_OK;
        }
    }
}

}  // extern "C"
