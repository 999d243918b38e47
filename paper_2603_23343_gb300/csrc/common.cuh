// Shared host/device helpers of libgbpcg: error reporting, TMA tensor maps,
// mbarrier waits with an iteration limit, block reductions.
#pragma once

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gbpcg.h"

namespace gb {

// ------------------------------------------------------------------ errors --

void set_error(const std::string &msg);
void clear_error();
int fail_arg(const std::string &msg);
int fail_cuda(cudaError_t e, const char *what);

#define GB_CUDA(call)                                          \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ::gb::fail_cuda(_e, #call); \
    } while (0)

// NVTX range over a host scope (visible in timeline profilers; a no-op when
// no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *msg) { nvtxRangePushA(msg); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------------ dtypes --

inline size_t dtype_size(int dt) {
    switch (dt) {
        case GBPCG_F32: return 4;
        case GBPCG_BF16: return 2;
        case GBPCG_F16: return 2;
        case GBPCG_F64: return 8;
        default: return 0;
    }
}

template <typename T> struct TypeTag;
template <> struct TypeTag<float> { static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };
template <> struct TypeTag<__nv_bfloat16> { static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; };
template <> struct TypeTag<__half> { static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; };

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// Four consecutive elements <-> float[4]; the address is 4-element aligned.
template <typename T> __device__ __forceinline__ void ld4(const T *p, float v[4]);
template <> __device__ __forceinline__ void ld4<float>(const float *p, float v[4]) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <> __device__ __forceinline__ void ld4<__nv_bfloat16>(const __nv_bfloat16 *p, float v[4]) {
    uint2 t = *reinterpret_cast<const uint2 *>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&t.x), b = *reinterpret_cast<__nv_bfloat162 *>(&t.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
template <> __device__ __forceinline__ void ld4<__half>(const __half *p, float v[4]) {
    uint2 t = *reinterpret_cast<const uint2 *>(p);
    __half2 a = *reinterpret_cast<__half2 *>(&t.x), b = *reinterpret_cast<__half2 *>(&t.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
template <typename T> __device__ __forceinline__ void st4(T *p, const float v[4]);
template <> __device__ __forceinline__ void st4<float>(float *p, const float v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void st4<__nv_bfloat16>(__nv_bfloat16 *p, const float v[4]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<uint32_t *>(&a);
    t.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = t;
}
template <> __device__ __forceinline__ void st4<__half>(__half *p, const float v[4]) {
    __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<uint32_t *>(&a);
    t.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = t;
}

// Eight consecutive elements <-> float[8] (16-byte aligned for 16-bit types,
// 32-byte for float).
template <typename T> __device__ __forceinline__ void ld8(const T *p, float v[8]);
template <> __device__ __forceinline__ void ld8<float>(const float *p, float v[8]) {
    ld4<float>(p, v);
    ld4<float>(p + 4, v + 4);
}
template <> __device__ __forceinline__ void ld8<__nv_bfloat16>(const __nv_bfloat16 *p, float v[8]) {
    uint4 t = *reinterpret_cast<const uint4 *>(p);
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[i]);
        float2 f = __bfloat1622float2(h);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
template <> __device__ __forceinline__ void ld8<__half>(const __half *p, float v[8]) {
    uint4 t = *reinterpret_cast<const uint4 *>(p);
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
        float2 f = __half22float2(h);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
template <typename T> __device__ __forceinline__ void st8(T *p, const float v[8]);
template <> __device__ __forceinline__ void st8<float>(float *p, const float v[8]) {
    st4<float>(p, v);
    st4<float>(p + 4, v + 4);
}
template <> __device__ __forceinline__ void st8<__nv_bfloat16>(__nv_bfloat16 *p, const float v[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
template <> __device__ __forceinline__ void st8<__half>(__half *p, const float v[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
// V (4 or 8) consecutive elements
template <typename T, int V> __device__ __forceinline__ void ldv(const T *p, float v[V]) {
    if constexpr (V == 4) ld4<T>(p, v); else ld8<T>(p, v);
}
template <typename T, int V> __device__ __forceinline__ void stv(T *p, const float v[V]) {
    if constexpr (V == 4) st4<T>(p, v); else st8<T>(p, v);
}

// ------------------------------------------------------- TMA tensor maps --

// Encodes a 3D tiled tensor map over a dense (nz, ny, nx) array with box
// (bx, by, bz); out-of-range elements of a box read as zero.
int make_map_3d(CUtensorMap *map, CUtensorMapDataType dt, size_t esize, const void *base, int nx,
                int ny, int nz, int bx, int by, int bz);

// Tiled tensor map of any rank (<= 5): dims[0] is the contiguous dimension,
// strides[d] the byte stride of dimension d + 1 (multiples of 16), box the
// copied box; out-of-range elements read as zero, no swizzle.
int make_map_nd(CUtensorMap *map, CUtensorMapDataType dt, const void *base, int rank, const uint64_t *dims,
                const uint64_t *strides, const uint32_t *box);

// --------------------------------------------------------- device PTX ------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the TMA (async) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Every wait on a TMA or MMA completion is bounded: after this many polls the
// caller records a timeout and stops instead of spinning forever.  A failed
// mbarrier.try_wait suspends about 3.8 us on GB300 (measured with
// gbpcg_wait_selftest), so 2^18 polls give up after about one second -- far
// beyond any legitimate wait (a stage's copy, a CTA's MMAs).
constexpr uint32_t kWaitPolls = 1u << 18;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t polls = kWaitPolls) {
    for (uint32_t i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 3D tiled TMA load of one box into shared memory, completion on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// An L2 policy that marks lines for early eviction: for data the next kernel
// does not read, so that it does not push out what the next kernel does read.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// tma_load_3d with an L2 cache policy
__device__ __forceinline__ void tma_load_3d_hint(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                                 int c2, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// four floats (16-byte aligned) to global memory with an L2 cache policy
__device__ __forceinline__ void st4f_hint(float *p, const float v[4], uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3]), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

// One plain arrival on a shared-memory mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ----------------------------------------------------------- reductions --

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums NV per-thread FP32 values over the block; warp sums in FP32, the
// cross-warp sum in FP64 in warp order.  Result valid in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(const float (&v)[NV], double (&out)[NV]) {
    __shared__ double red[NT / 32][NV > 0 ? NV : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float s = warp_sum(v[i]);
        if (lane == 0) red[w][i] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int j = 0; j < NT / 32; ++j) s += red[j][i];
            out[i] = s;
        }
    }
}

// Last-block finish of a grid-wide sum.  Every block calls this once with its
// partial sums (valid in thread 0).  Returns true in exactly one block (the
// last to arrive); there `total` (valid in thread 0) holds the grid sums,
// added in block order by a fixed tree, so the result does not depend on
// which block came last.  The ticket is reset for the next launch.
template <int NV, int NT>
__device__ __forceinline__ bool group_sum_last(const double (&part)[NV], double *partials, unsigned int *ticket,
                                               unsigned bid, unsigned nblk, double (&total)[NV]);

template <int NV, int NT>
__device__ __forceinline__ bool grid_sum_last(const double (&part)[NV], double *partials,
                                              unsigned int *ticket, double (&total)[NV]) {
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    return group_sum_last<NV, NT>(part, partials, ticket, bid, nblk, total);
}

// The same finish over a group of nblk contributions numbered bid = 0 ..
// nblk - 1 (a persistent CTA may contribute several, one per work item):
// returns true in the CTA whose contribution arrived last, with the sums
// taken in contribution order.
template <int NV, int NT>
__device__ __forceinline__ bool group_sum_last(const double (&part)[NV], double *partials, unsigned int *ticket,
                                               unsigned bid, unsigned nblk, double (&total)[NV]) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) partials[(size_t)bid * NV + i] = part[i];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    __shared__ double red[NT / 32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (unsigned j = threadIdx.x; j < nblk; j += NT) s += __ldcg(partials + (size_t)j * NV + i);
        s = warp_sum(s);
        if (lane == 0) red[w][i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int j = 0; j < NT / 32; ++j) s += red[j][i];
            total[i] = s;
        }
        *ticket = 0u;
    }
    return true;
}

}  // namespace gb
