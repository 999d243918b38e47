// 3x3x3 convolution as an implicit GEMM on the 5th-generation tensor cores
// (tcgen05, sm_103a): the dense contraction of the learned preconditioner.
//
// Layout: activations channels-last (Z, Y, X, C) BF16; weights (Co, 27, Ci)
// BF16 with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1); zero padding, stride 1.
//   out[v, o] = sum_{t, i} W[o, t, i] * in[v + off(t), i]
// GEMM view: M = 128 output voxels consecutive in (z, y, x) order (a row
// segment, or whole rows / planes when X < 128), N = Co, K = 27 * Ci consumed
// 16 at a time.
//
// Data path per K step (one tap, 16 input channels):
//   A tile 128 x 16 and B tile Co x 16 arrive by TMA as two 8-channel
//   boxes each.  An 8-channel box puts every voxel's 8 channels in one
//   16-byte row, so 8 consecutive rows form one 128-byte core matrix: the
//   K-major no-swizzle layout of the UMMA shared-memory descriptor with
//   SBO = 128 B (next 8 rows) and LBO = the distance between the two
//   8-channel halves.  The box origin is shifted by the tap, and TMA fills
//   out-of-grid parts with zeros, which is the convolution's padding.
//   One thread issues the TMA loads, another the tcgen05.mma (D in TMEM,
//   FP32); tcgen05.commit on a per-stage mbarrier frees the stage.
// Epilogue: the four warps read their 32 TMEM lanes (one voxel each) with
// tcgen05.ld, apply the optional ReLU and mask and store BF16 or FP32 into a
// channel slice of the output (so concatenations are free).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace gb {

// ------------------------------------------------------- tcgen05 wrappers --

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulation
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrives on `bar` once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The sum of three 16-column blocks of this thread's TMEM lane (at ta, tb, tc):
// three loads in flight, then one wait, in one asm statement so that no use of
// the registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16_sum3(uint32_t ta, uint32_t tb, uint32_t tc, float v[16]) {
    uint32_t r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%48];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31}, [%49];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
        "%45, %46, %47}, [%50];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
          "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
          "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(ta), "r"(tb), "r"(tc)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]) + __uint_as_float(r[16 + i]) + __uint_as_float(r[32 + i]);
}

// UMMA shared-memory descriptor, K-major, no swizzle: start address, leading
// byte offset (between 8-element K groups), stride byte offset (between
// 8-row M/N groups), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;  // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM columns to allocate for an accumulator of N FP32 columns (a power
// of two, at least 32).
__host__ __device__ constexpr uint32_t tmem_cols(int N) {
    return N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : N <= 256 ? 256u : 512u;
}

struct __align__(128) ConvMaps {
    CUtensorMap act;  // (C, X, Y, Z) BF16, box (8, tx, ty, tz)
    CUtensorMap wgt;  // (27 * Ci, Co) BF16, box (8, Co)
};

// Output voxel tile of the implicit GEMM: 128 voxels consecutive in
// (z, y, x) order, tx * ty * tz = 128.  Valid when X is a multiple of 128,
// or X divides 128 and whole rows (and, below 128 points per plane, whole
// planes) make up the tile.
struct ConvTile {
    int tx, ty, tz;
};

struct ConvArgs {
    int X, Y, Z;
    int ci, co;          // input channels (the input holds exactly ci per voxel) and output channels
    ConvTile tile;
    void *out;           // BF16 or FP32, channels-last, cstride channels per voxel
    int cstride, coff;   // output slice: channels [coff, coff + co) of cstride
    int relu;
    const __nv_bfloat16 *mask;  // optional: out *= (mask > 0), mask channels [moff, moff + co) of mstride
    int mstride, moff;
    int *err;            // set to 1 if a bounded wait gave up
    int nseg, stages;    // z-marching kernel: z segments per column, stages in its ring
};

constexpr int kConvStages = 6;
constexpr uint32_t kConvAStage = 4096;  // 128 voxels x 16 channels x 2 B

template <int CO>
constexpr uint32_t conv_stage_bytes() {
    return (kConvAStage + 2 * CO * 16 + 1023) & ~1023u;
}
// Shared memory past the last stage that no operand should touch: it keeps
// every descriptor-addressed read inside the allocation even under a wrong
// reading of the descriptor's stride fields.
constexpr uint32_t kConvGuard = 32768;
template <int CO>
constexpr uint32_t conv_smem_bytes() {
    return kConvStages * conv_stage_bytes<CO>() + kConvGuard;
}

// One CTA = one 128-voxel tile, four warps.  Warp 0 lane 0 loads stages by
// TMA, warp 1 lane 0 issues the MMAs, all four warps run the epilogue.
template <int CO, typename OUT>
__global__ void __launch_bounds__(128) conv3_tc_kernel(const __grid_constant__ ConvMaps maps, const ConvArgs a) {
    constexpr uint32_t SB = conv_stage_bytes<CO>();
    constexpr uint32_t NCOL = tmem_cols(CO);
    constexpr uint32_t IDESC = idesc_bf16(128, CO);
    constexpr uint32_t STAGE_TX = kConvAStage + 2 * CO * 16;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kConvStages], empty[kConvStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t v0 = (int64_t)blockIdx.x * 128;
    const int x0 = (int)(v0 % a.X);
    const int y0 = (int)((v0 / a.X) % a.Y);
    const int z0 = (int)(v0 / ((int64_t)a.X * a.Y));
    const int kc = a.ci / 16;  // 16-channel steps per tap
    const int KT = 27 * kc;

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < kConvStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, NCOL);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0 && lane == 0) {
        // producer: stage s is refilled once the MMA that read it has completed
        int kk = 0;
        for (; kk < KT; ++kk) {
            const int s = kk % kConvStages;
            if (kk >= kConvStages && !mbar_wait_bounded(&empty[s], ((kk / kConvStages) - 1) & 1)) {
                s_err = 1;
                break;
            }
            const int t = kk / kc, cc = kk - t * kc;
            const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            unsigned char *st = smem + (size_t)s * SB;
            mbar_arrive_expect_tx(&full[s], STAGE_TX);
            for (int h = 0; h < 2; ++h) {
                tma_load_4d(st + h * 2048, &maps.act, &full[s], cc * 16 + h * 8, x0 + dx, y0 + dy, z0 + dz);
                tma_load_2d(st + kConvAStage + h * CO * 16, &maps.wgt, &full[s], t * a.ci + cc * 16 + h * 8, 0);
            }
        }
        // drain: wait (bounded) for the last copy issued into every stage
        for (int s = 0; s < kConvStages; ++s) {
            const int last = kk - 1 - ((kk - 1 - s) % kConvStages + kConvStages) % kConvStages;
            if (last >= 0 && last < kk && !mbar_wait_bounded(&full[s], (last / kConvStages) & 1)) s_err = 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: D[128 x CO] (+)= A[128 x 16] * B[CO x 16]^T per step
        for (int kk = 0; kk < KT; ++kk) {
            const int s = kk % kConvStages;
            if (!mbar_wait_bounded(&full[s], (kk / kConvStages) & 1)) {
                s_err = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)s * SB;
            const uint64_t adesc = umma_desc_kmajor(sa, 2048, 128);
            const uint64_t bdesc = umma_desc_kmajor(sa + kConvAStage, CO * 16, 128);
            mma_bf16(tmem, adesc, bdesc, IDESC, kk > 0 ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&done, 0);
    __syncthreads();
    const bool good = ok && !s_err;
    tc_fence_after();

    // epilogue: warp w reads TMEM lanes 32w .. 32w + 31 = tile rows (voxels)
    const int64_t v = v0 + warp * 32 + lane;
    OUT *out = static_cast<OUT *>(a.out) + v * a.cstride + a.coff;
    const __nv_bfloat16 *mk = a.mask ? a.mask + v * a.mstride + a.moff : nullptr;
#pragma unroll
    for (int c0 = 0; c0 < CO; c0 += 16) {
        float f[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, f);
        float m[16];
        if (mk) {
            ld8(mk + c0, m);
            ld8(mk + c0 + 8, m + 8);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            f[i] = good ? f[i] : 0.0f;
            if (a.relu) f[i] = f[i] < 0.0f ? 0.0f : f[i];  // NaN passes: broken weights stay visible
            if (mk && !(m[i] > 0.0f)) f[i] = 0.0f;
        }
        if constexpr (std::is_same<OUT, float>::value) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) st4(out + c0 + i, f + i);
        } else {
            st8(out + c0, f);
            st8(out + c0 + 8, f + 8);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOL);
    if (!good && threadIdx.x == 0) atomicExch(a.err, 1);
}

// ------------------------------------------------------------------------
// Halo-slab variant for X a multiple of 128: a CTA owns R = 4 rows of 128
// voxels (four M tiles, 4 x CO TMEM columns) of one plane.  A pipeline step
// is one 16-channel chunk of one source plane (dz): the (R + 2) rows x 130
// voxels around the tile arrive in one TMA box per 8-channel half, together
// with that plane's 9 taps of weights.  Every tap (dy, dx) of every M tile
// then reads the slab in place: its A operand starts (rho + dy + 1) rows and
// (dx + 1) voxels into it, a 16-byte multiple, with the same SBO (128 B) and
// LBO (distance between the halves).  Input traffic per output voxel and
// 16-channel chunk: 3 x 6 x 130 x 32 B / 512 = 146 B, against 27 x 32 B =
// 864 B when each tap reloads its tile.

constexpr int kHaloRows = 4;
constexpr int kHaloX = 130;

template <int CO>
struct HaloCfg {
    static constexpr uint32_t A_HALF = ((uint32_t)(16 * kHaloX * (kHaloRows + 2)) + 127) & ~127u;
    static constexpr uint32_t B_HALF = 9u * CO * 16u;  // a multiple of 128 for CO % 16 == 0
    static constexpr uint32_t A_TX = 2u * 16 * kHaloX * (kHaloRows + 2);
    static constexpr uint32_t STAGE_TX = A_TX + 2 * B_HALF;
    static constexpr uint32_t STAGE = (2 * A_HALF + 2 * B_HALF + 1023) & ~1023u;
    // two CTAs per SM (about 110 KB each), so that one CTA's prologue and
    // epilogue overlap the other's loads and MMAs (seven CTAs of one stage
    // each measured the same)
    static constexpr int STAGES = (int)(((110u * 1024u) / STAGE) < 6u ? ((110u * 1024u) / STAGE) : 6u);
    static constexpr uint32_t SMEM = STAGES * STAGE;
    static constexpr uint32_t NCOL = tmem_cols(kHaloRows * CO);
    static_assert(STAGES >= 2, "halo stage too large");
    static_assert(kHaloRows * CO <= 512, "TMEM columns");
};

template <int CO, typename OUT>
__global__ void __launch_bounds__(128) conv3_tc_halo_kernel(const __grid_constant__ ConvMaps maps, const ConvArgs a) {
    using H = HaloCfg<CO>;
    constexpr int S = H::STAGES;
    constexpr uint32_t IDESC = idesc_bf16(128, CO);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * kHaloRows, z0 = blockIdx.z;
    const int kc = a.ci / 16;
    const int KT = 3 * kc;  // (chunk, plane) steps

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, H::NCOL);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0 && lane == 0) {
        int kk = 0;
        for (; kk < KT; ++kk) {
            const int s = kk % S;
            if (kk >= S && !mbar_wait_bounded(&empty[s], ((kk / S) - 1) & 1)) {
                s_err = 1;
                break;
            }
            const int cc = kk / 3, pz = kk - cc * 3;  // chunk, plane (dz = pz - 1)
            unsigned char *st = smem + (size_t)s * H::STAGE;
            mbar_arrive_expect_tx(&full[s], H::STAGE_TX);
            for (int h = 0; h < 2; ++h) {
                tma_load_4d(st + h * H::A_HALF, &maps.act, &full[s], cc * 16 + h * 8, x0 - 1, y0 - 1, z0 + pz - 1);
                // the plane's 9 taps in one box: (8 channels, CO, 9 taps) -> [tap][co][8 channels]
                tma_load_3d(st + 2 * H::A_HALF + h * H::B_HALF, &maps.wgt, &full[s], cc * 16 + h * 8, 0, pz * 9);
            }
        }
        for (int s = 0; s < S; ++s) {
            const int last = kk - 1 - ((kk - 1 - s) % S + S) % S;
            if (last >= 0 && last < kk && !mbar_wait_bounded(&full[s], (last / S) & 1)) s_err = 1;
        }
    } else if (warp == 1 && lane == 0) {
        for (int kk = 0; kk < KT; ++kk) {
            const int s = kk % S;
            if (!mbar_wait_bounded(&full[s], (kk / S) & 1)) {
                s_err = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)s * H::STAGE;
            const uint32_t sb = sa + 2 * H::A_HALF;
#pragma unroll 1
            for (int rho = 0; rho < kHaloRows; ++rho)
#pragma unroll
                for (int tau = 0; tau < 9; ++tau) {
                    const int dy = tau / 3 - 1, dx = tau % 3 - 1;
                    const uint32_t aa = sa + (uint32_t)(((rho + dy + 1) * kHaloX + dx + 1) * 16);
                    const uint64_t adesc = umma_desc_kmajor(aa, H::A_HALF, 128);
                    const uint64_t bdesc = umma_desc_kmajor(sb + (uint32_t)(tau * CO * 16), H::B_HALF, 128);
                    mma_bf16(tmem + (uint32_t)(rho * CO), adesc, bdesc, IDESC, (kk > 0 || tau > 0) ? 1u : 0u);
                }
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&done, 0);
    __syncthreads();
    const bool good = ok && !s_err;
    tc_fence_after();

    // epilogue: warp w reads lanes 32w .. 32w + 31 (voxels x0 + 32w + lane) of each M tile
    const int x = x0 + warp * 32 + lane;
#pragma unroll 1
    for (int rho = 0; rho < kHaloRows; ++rho) {
        const int64_t v = ((int64_t)z0 * a.Y + y0 + rho) * a.X + x;
        OUT *out = static_cast<OUT *>(a.out) + v * a.cstride + a.coff;
        const __nv_bfloat16 *mk = a.mask ? a.mask + v * a.mstride + a.moff : nullptr;
#pragma unroll
        for (int c0 = 0; c0 < CO; c0 += 16) {
            float f[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(rho * CO + c0), f);
            float m[16];
            if (mk) {
                ld8(mk + c0, m);
                ld8(mk + c0 + 8, m + 8);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                f[i] = good ? f[i] : 0.0f;
                if (a.relu) f[i] = f[i] < 0.0f ? 0.0f : f[i];
                if (mk && !(m[i] > 0.0f)) f[i] = 0.0f;
            }
            if constexpr (std::is_same<OUT, float>::value) {
#pragma unroll
                for (int i = 0; i < 16; i += 4) st4(out + c0 + i, f + i);
            } else {
                st8(out + c0, f);
                st8(out + c0 + 8, f + 8);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, H::NCOL);
    if (!good && threadIdx.x == 0) atomicExch(a.err, 1);
}

}  // namespace gb

namespace gb {

// ------------------------------------------------------------------------
// z-marching kernel for 16 output channels (c2, c8), X a multiple of 128.
//
// A CTA owns a column of output voxels, 128 x R = 3 rows (the last column of a
// grid whose Y is not a multiple of 3 is masked), over a z segment
// [zs, ze), and marches its source planes m = zs - 1 .. ze.  One stage holds
// one 16-channel chunk of plane m's slab (R + 2 rows x 130 voxels, zero
// filled outside the grid by TMA) and feeds all three output planes it
// touches: o = m + 1 (taps dz = -1), m (dz = 0) and m - 1 (dz = +1).  Each
// slab is loaded once instead of once per output plane: the halo kernel's
// limit was the L2 delivery of those slabs, about 25 KB per 2,300 SM cycles.
//
// Within a plane, the three taps dy = -1, 0, +1 of one (dz, dx) read the same
// slab row for different output rows, so one MMA serves every tap a slab row
// feeds: for slab row r (r = -1 .. R) and tap (dz, dx),
//   P_r[x, (dy, o)] += sum_i in[m, y0 + r, x + dx, i] W[o, (dz, dy, dx), i]
// over dy in [max(-1, r - R + 1), min(1, r)] (output rows rho = r - dy inside
// the column), N = 16, 32 or 48.  Each P_r has its own TMEM columns (3 R x 16
// for a plane, each column an output partial sum) and the epilogue adds
//   out[rho, x, o] = sum_dy P_{rho + dy}[x, (dy, o)]
// within TMEM lane x.  Per (source plane, chunk) that is 3 x 3 x (R + 2) = 45
// MMAs for three output planes of R rows, against 81 with one MMA per (row,
// tap).  Three output planes are open at a time; their accumulators rotate
// through 3 x 144 of the SM's 512 TMEM columns (one CTA per SM).
//
// Roles: warp 4 lane 0 loads the layer's weights once (all 27 taps stay in
// shared memory, in [chunk][dz][half][dx][dy][co][8] order from a 5D view of
// the (Co, 27, Ci) array) and then streams the slabs by TMA; warp 5 lane 0
// issues the MMAs; warps 0-3 drain each output plane once its last source
// plane is in (warp w reads TMEM lanes 32w .. 32w + 31).  In a stage the MMAs
// into planes m - 1 and m go first; the first MMAs into plane m + 1 reuse the
// accumulator of plane m - 2 and wait, at chunk 0, for its epilogue.

constexpr int kZmMaxStages = 8;

struct ZmCfg {
    static constexpr int CO = 16, R = 3, NR = R + 2;
    static constexpr uint32_t A_HALF = ((uint32_t)(16 * kHaloX * NR) + 127) & ~127u;
    static constexpr uint32_t A_STAGE = (2 * A_HALF + 1023) & ~1023u;
    static constexpr uint32_t A_TX = 2u * 16 * kHaloX * NR;  // bytes the two slab boxes bring
    static constexpr uint32_t B_HALF = 9u * CO * 16u;         // 9 taps (one dz) of 8 channels
    static constexpr int ACC = 3 * R * CO;                    // TMEM columns of one output plane
    static constexpr uint32_t NCOL = 512;
    // resident weights: 6 boxes (3 dz x 2 halves) per 16-channel chunk
    __host__ __device__ static constexpr uint32_t wbytes(int kc) {
        return ((uint32_t)(6 * kc) * B_HALF + 1023) & ~1023u;
    }
    // taps dy_lo(r) .. dy_hi(r) of slab row r, and the first TMEM column of P_r
    __host__ __device__ static constexpr int dy_lo(int r) { return r - R + 1 > -1 ? r - R + 1 : -1; }
    __host__ __device__ static constexpr int dy_hi(int r) { return r < 1 ? r : 1; }
    __host__ __device__ static constexpr int nblk(int r) { return dy_hi(r) - dy_lo(r) + 1; }
    __host__ __device__ static constexpr int col(int r) {
        int c = 0;
        for (int q = -1; q < r; ++q) c += nblk(q) * CO;
        return c;
    }
    static_assert(3 * ACC <= (int)NCOL, "three open output planes in TMEM");
};

// Geometry of work item `item`: column (x0, y0) and z segment [zs, ze).
struct ZmItem {
    int x0, y0, zs, ze;
};
__device__ __forceinline__ ZmItem zm_item(const ConvArgs &a, int item, int tiles_x, int ncols) {
    const int c = item % ncols, g = item / ncols;
    ZmItem t;
    t.x0 = (c % tiles_x) * 128;
    t.y0 = (c / tiles_x) * ZmCfg::R;
    t.zs = (int)((int64_t)g * a.Z / a.nseg);
    t.ze = (int)((int64_t)(g + 1) * a.Z / a.nseg);
    return t;
}

template <typename OUT>
__global__ void __launch_bounds__(192, 1) conv3_tc_zmarch_kernel(const __grid_constant__ ConvMaps maps,
                                                                  const ConvArgs a) {
    using H = ZmCfg;
    constexpr int R = H::R, CO = H::CO;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kZmMaxStages], empty[kZmMaxStages], acc_full[3], acc_empty[3], wbar, done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;
    volatile int *err = &s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kc = a.ci / 16, S = a.stages;
    const int tiles_x = a.X / 128, ncols = tiles_x * ((a.Y + R - 1) / R);
    const int nitems = ncols * a.nseg;
    const uint32_t wb = H::wbytes(kc);

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 3; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&wbar, 1);
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, H::NCOL);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        if (lane == 0) {
            // the layer's weights, once: box (channel half, dz) of chunk cc at
            // ((cc * 3 + dz + 1) * 2 + half) * B_HALF
            mbar_arrive_expect_tx(&wbar, (uint32_t)(6 * kc) * H::B_HALF);
            for (int cc = 0; cc < kc; ++cc)
                for (int dzi = 0; dzi < 3; ++dzi)
                    for (int h = 0; h < 2; ++h)
                        tma_load_5d(smem + (size_t)((cc * 3 + dzi) * 2 + h) * H::B_HALF, &maps.wgt, &wbar,
                                    cc * 16 + h * 8, 0, 0, 0, dzi);
            unsigned char *stages = smem + wb;
            uint32_t step = 0;  // stages issued so far (ring slot step % S, its use step / S)
            for (int item = blockIdx.x; item < nitems && !*err; item += gridDim.x) {
                const ZmItem t = zm_item(a, item, tiles_x, ncols);
                for (int m = t.zs - 1; m <= t.ze && !*err; ++m)
                    for (int cc = 0; cc < kc; ++cc) {
                        const int s = (int)(step % (uint32_t)S);
                        if (step >= (uint32_t)S && !mbar_wait_bounded(&empty[s], ((step / S) - 1) & 1)) {
                            *err = 1;
                            break;
                        }
                        unsigned char *st = stages + (size_t)s * H::A_STAGE;
                        mbar_arrive_expect_tx(&full[s], H::A_TX);
                        for (int h = 0; h < 2; ++h)
                            tma_load_4d(st + h * H::A_HALF, &maps.act, &full[s], cc * 16 + h * 8, t.x0 - 1, t.y0 - 1,
                                        m);
                        ++step;
                    }
            }
            // every issued copy has landed before the CTA can exit
            for (int s = 0; s < S; ++s)
                if (step > (uint32_t)s) {
                    const uint32_t last = (uint32_t)s + ((step - 1 - (uint32_t)s) / S) * S;
                    if (!mbar_wait_bounded(&full[s], (last / S) & 1)) *err = 1;
                }
            if (!mbar_wait_bounded(&wbar, 0)) *err = 1;
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t sbase = smem_u32(smem), stb = sbase + wb;
            bool ok = mbar_wait_bounded(&wbar, 0);
            if (!ok) *err = 1;
            tc_fence_after();
            uint32_t step = 0, J0 = 0;  // stages consumed; output planes of this CTA's earlier items
            for (int item = blockIdx.x; item < nitems && ok && !*err; item += gridDim.x) {
                const ZmItem t = zm_item(a, item, tiles_x, ncols);
                for (int m = t.zs - 1; m <= t.ze && ok; ++m) {
                    // output planes source plane m feeds: m + 1 (dz = -1), m (dz = 0), m - 1 (dz = +1)
                    const bool f_next = m + 1 >= t.zs && m + 1 < t.ze;
                    const bool f_cur = m >= t.zs && m < t.ze;
                    const bool f_prev = m - 1 >= t.zs && m - 1 < t.ze;
                    for (int cc = 0; cc < kc; ++cc, ++step) {
                        const int s = (int)(step % (uint32_t)S);
                        if (!mbar_wait_bounded(&full[s], (step / S) & 1)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t adesc = umma_desc_kmajor(stb + (uint32_t)s * H::A_STAGE, H::A_HALF, 128);
                        // one tap plane dz of this chunk into the accumulator of output plane J
                        auto taps = [&](int dzi, uint32_t J, bool first) {
                            const uint32_t acc = tmem + (J % 3) * (uint32_t)H::ACC;
                            const uint64_t bdesc =
                                umma_desc_kmajor(sbase + (uint32_t)((cc * 3 + dzi) * 2) * H::B_HALF, H::B_HALF, 128);
#pragma unroll
                            for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
                                for (int r = -1; r <= R; ++r) {
                                    // A: slab row r shifted by dx; B: taps (dx, dy_lo(r) .. dy_hi(r)); both
                                    // offsets are 16-byte multiples added to the descriptors' address field
                                    const uint32_t aoff = (uint32_t)((r + 1) * kHaloX + dxi);
                                    const uint32_t boff = (uint32_t)((dxi * 3 + H::dy_lo(r) + 1) * CO);
                                    mma_bf16(acc + (uint32_t)H::col(r), adesc + aoff, bdesc + boff,
                                             idesc_bf16(128, H::nblk(r) * CO), (first && dxi == 0) ? 0u : 1u);
                                }
                        };
                        if (f_prev) taps(2, J0 + (uint32_t)(m - 1 - t.zs), false);
                        if (f_cur) taps(1, J0 + (uint32_t)(m - t.zs), false);
                        if (f_next) {
                            const uint32_t J = J0 + (uint32_t)(m + 1 - t.zs);
                            // plane J's accumulator held plane J - 3 until its epilogue released it
                            if (cc == 0 && J >= 3) {
                                if (!mbar_wait_bounded(&acc_empty[J % 3], ((J / 3) - 1) & 1)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                            }
                            taps(0, J, cc == 0);
                        }
                        mma_commit(&empty[s]);
                        // plane m - 1 has all its source planes once the last chunk of plane m is in
                        if (cc == kc - 1 && f_prev) mma_commit(&acc_full[(J0 + (uint32_t)(m - 1 - t.zs)) % 3]);
                    }
                }
                J0 += (uint32_t)(t.ze - t.zs);
            }
            if (!ok) *err = 1;
            mma_commit(&done);
        }
    } else if (warp < 4) {
        uint32_t J = 0;  // output planes drained so far
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const ZmItem t = zm_item(a, item, tiles_x, ncols);
            const int x = t.x0 + warp * 32 + lane;
            for (int o = t.zs; o < t.ze; ++o, ++J) {
                const int b = (int)(J % 3);
                // warp-uniform: every lane polls the same barrier, the warp agrees on the outcome
                ok = __all_sync(0xffffffffu, !*err && mbar_wait_bounded(&acc_full[b], (J / 3) & 1));
                if (!ok) {
                    if (lane == 0) *err = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * H::ACC);
#pragma unroll
                for (int rho = 0; rho < R; ++rho) {
                    if (t.y0 + rho >= a.Y) continue;  // the masked rows of a grid's last column
                    const int64_t v = ((int64_t)o * a.Y + t.y0 + rho) * a.X + x;
                    OUT *out = static_cast<OUT *>(a.out) + v * a.cstride + a.coff;
                    const __nv_bfloat16 *mk = a.mask ? a.mask + v * a.mstride + a.moff : nullptr;
                    // dy = -1 from P_{rho-1}, 0 from P_rho, +1 from P_{rho+1}
                    float f[16];
                    tmem_ld16_sum3(lane_base + (uint32_t)(H::col(rho - 1) + (-1 - H::dy_lo(rho - 1)) * CO),
                                   lane_base + (uint32_t)(H::col(rho) + (0 - H::dy_lo(rho)) * CO),
                                   lane_base + (uint32_t)(H::col(rho + 1) + (1 - H::dy_lo(rho + 1)) * CO), f);
                    float mv[16];
                    if (mk) {
                        ld8(mk, mv);
                        ld8(mk + 8, mv + 8);
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (a.relu) f[i] = f[i] < 0.0f ? 0.0f : f[i];
                        if (mk && !(mv[i] > 0.0f)) f[i] = 0.0f;
                    }
                    if constexpr (std::is_same<OUT, float>::value) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4) st4(out + i, f + i);
                    } else {
                        st8(out, f);
                        st8(out + 8, f + 8);
                    }
                }
                // the TMEM reads have completed (the loads waited) before the MMAs may reuse the columns
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
            }
        }
    }
    __syncwarp();
    // the MMAs issued (all of them, on every path) have completed before TMEM is freed
    const bool fin = mbar_wait_bounded(&done, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, H::NCOL);
    if (threadIdx.x == 0 && (s_err || !fin)) atomicExch(a.err, 1);
}

// ------------------------------------------------------------------------
// Weight gradient on the tensor cores:
//   gW[o, t, i] = sum_u gy[u - off(t), o] x[u, i]
// as D[(t, o), i] = sum_u A[(t, o), u] B[i, u] with K = voxels.  An M tile
// stacks tp = 128 / Co taps of Co output channels (8 taps of 16 channels,
// 4 of 32, ...); rows past tp Co or past tap 26 are zero.  Both operands
// are MN-major: a TMA box of 8 channels x 128 voxels puts each voxel's 8
// channels in one 16-byte row, i.e. core matrices of 8 voxels (K) x 8
// channels (M or N), K groups 128 B apart (LBO) and 8-channel groups one box
// (2 KB) apart (SBO).  The tap shift is the box origin; TMA's zero fill
// gives gy = 0 outside the grid.  A CTA owns a run of 128-voxel chunks (a
// K slice) and a group of M tiles, accumulates in TMEM (group x Ci columns)
// and writes its sums to its own slot; slots are added in a fixed order.

struct __align__(128) WgMaps {
    CUtensorMap gy;  // (Co, X, Y, Z) BF16, box (8, tx, ty, tz)
    CUtensorMap x;   // (Ci, X, Y, Z) BF16, box (8, tx, ty, tz)
};

struct WgArgs {
    int X, Y, Z, ci, co;
    ConvTile tile;
    int tp, mtiles, group;          // taps per M tile, M tiles, M tiles per CTA
    int chunks, chunks_per_cta;     // 128-voxel chunks in the grid, per CTA
    uint32_t stage_bytes, a_bytes;  // bytes per stage, of which A
    int stages;
    uint32_t ncol;                  // TMEM columns allocated
    float *partials;                // [gridDim.x][co][27][ci]
    int *err;
};

__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
    return idesc_bf16(M, N) | (1u << 15) | (1u << 16);  // A and B MN-major
}

__device__ __forceinline__ uint64_t umma_desc_mnmajor(uint32_t saddr, uint32_t lbo_k, uint32_t sbo_mn) {
    return umma_desc_kmajor(saddr, lbo_k, sbo_mn);  // same fields: LBO between K groups, SBO between MN groups
}

constexpr int kWgMaxStages = 6;

__global__ void __launch_bounds__(128) wgrad_tc_kernel(const __grid_constant__ WgMaps maps, const WgArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kWgMaxStages], empty[kWgMaxStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.stages;
    const int m0 = blockIdx.y * a.group;
    const int gm = min(a.group, a.mtiles - m0);
    const int c_begin = blockIdx.x * a.chunks_per_cta;
    const int c_end = min(a.chunks, c_begin + a.chunks_per_cta);
    const int KT = (c_end - c_begin) * gm;
    const int gpt = a.co / 8;            // 8-channel groups per tap
    const int nb = a.ci / 8;             // B groups
    const uint32_t idesc = idesc_bf16_mn(128, a.ci);

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, a.ncol);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0 && lane == 0) {
        int kk = 0;
        for (; kk < KT; ++kk) {
            const int s = kk % S;
            if (kk >= S && !mbar_wait_bounded(&empty[s], ((kk / S) - 1) & 1)) {
                s_err = 1;
                break;
            }
            const int c = c_begin + kk / gm, mt = m0 + kk % gm;
            const int64_t v0 = (int64_t)c * 128;
            const int x0 = (int)(v0 % a.X), y0 = (int)((v0 / a.X) % a.Y), z0 = (int)(v0 / ((int64_t)a.X * a.Y));
            unsigned char *st = smem + (size_t)s * a.stage_bytes;
            mbar_arrive_expect_tx(&full[s], a.stage_bytes);
            for (int g = 0; g < 16; ++g) {
                const int tau = g / gpt, h = g - tau * gpt, t = mt * a.tp + tau;
                if (tau < a.tp && t < 27) {
                    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                    tma_load_4d(st + g * 2048, &maps.gy, &full[s], h * 8, x0 - dx, y0 - dy, z0 - dz);
                } else {  // a row group past the taps: a box wholly outside the tensor reads as zeros
                    tma_load_4d(st + g * 2048, &maps.gy, &full[s], a.co, x0, y0, z0);
                }
            }
            for (int g = 0; g < nb; ++g) tma_load_4d(st + a.a_bytes + g * 2048, &maps.x, &full[s], g * 8, x0, y0, z0);
        }
        for (int s = 0; s < S; ++s) {
            const int last = kk - 1 - ((kk - 1 - s) % S + S) % S;
            if (last >= 0 && last < kk && !mbar_wait_bounded(&full[s], (last / S) & 1)) s_err = 1;
        }
    } else if (warp == 1 && lane == 0) {
        for (int kk = 0; kk < KT; ++kk) {
            const int s = kk % S;
            if (!mbar_wait_bounded(&full[s], (kk / S) & 1)) {
                s_err = 1;
                break;
            }
            tc_fence_after();
            const int first_chunk = (kk / gm) == 0, mt = kk % gm;
            const uint32_t sa = sbase + (uint32_t)s * a.stage_bytes, sb = sa + a.a_bytes;
#pragma unroll
            for (int k16 = 0; k16 < 8; ++k16) {  // 16 voxels per MMA: two 8-voxel K groups
                const uint64_t ad = umma_desc_mnmajor(sa + k16 * 256, 128, 2048);
                const uint64_t bd = umma_desc_mnmajor(sb + k16 * 256, 128, 2048);
                mma_bf16(tmem + (uint32_t)(mt * a.ci), ad, bd, idesc, (first_chunk && k16 == 0) ? 0u : 1u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&done, 0);
    __syncthreads();
    const bool good = ok && !s_err && KT > 0;
    tc_fence_after();

    // epilogue: TMEM lane = M row = (tau, o); columns = input channels of M tile mt
    const int row = warp * 32 + lane;
    const int tau = row / a.co, o = row - tau * a.co;
    float *slot = a.partials + (int64_t)blockIdx.x * ((int64_t)a.co * 27 * a.ci);
    for (int mt = 0; mt < gm; ++mt) {
        const int t = (m0 + mt) * a.tp + tau;
        const bool valid = tau < a.tp && t < 27;
        for (int c0 = 0; c0 < a.ci; c0 += 16) {
            float f[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * a.ci + c0), f);
            if (valid) {
                float *dst = slot + ((int64_t)o * 27 + t) * a.ci + c0;
#pragma unroll
                for (int i = 0; i < 16; i += 4) {
                    float q[4] = {good ? f[i] : 0.f, good ? f[i + 1] : 0.f, good ? f[i + 2] : 0.f, good ? f[i + 3] : 0.f};
                    st4(dst + i, q);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.ncol);
    if (!good && KT > 0 && threadIdx.x == 0) atomicExch(a.err, 1);
}

}  // namespace gb
