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
