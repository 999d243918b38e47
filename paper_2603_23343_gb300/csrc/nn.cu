// Learned preconditioner z = N(r) (no counterpart in the paper, which keeps
// Jacobi): a three-level 3D U-net of 3x3x3 convolutions without bias,
// channels-last BF16 activations and weights with FP32 accumulation.
//
//   c1 (2->16), c2 (16->16) = e0          level 0 (full resolution)
//   pool, c3 (16->32), c4 (32->32) = e1   level 1
//   pool, c5 (32->64), c6 (64->64)        level 2
//   up, [up(c6), e1] -> c7 (96->32)       level 1
//   up, [up(c7), e0] -> c8 (48->16)       level 0
//   c9 (16->1)                            output, no ReLU
// N acts on the Jacobi-scaled system D^{-1/2} A D^{-1/2} (D the operator's
// diagonal): input channels s / rms(s) with s = D^{-1/2} r, and log k; the
// output is multiplied by rms(s) D^{-1/2}.  (A ReLU network is piecewise
// linear in (r, log k) and cannot form the product r / k that the coefficient
// contrast calls for; the scaling supplies it.)  pool is a 2x2x2 average, up
// nearest-neighbour doubling.
//
// Convolutions with 16+ input and output channels (c2..c8 and their
// data-gradient convolutions) run on the tensor cores (conv_tc.cuh); the
// 2- and 1-channel ends (c1, c9), the weight gradients and the glue run on
// CUDA cores.  Concatenations are free: c2 and c4 write e0 / e1 straight
// into the upper channels of the concatenated buffers, the upsampling
// kernels fill the lower ones.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "conv_tc.cuh"
#include "launch.cuh"

namespace gb {

// ------------------------------------------------------------ the network --

struct LayerDesc {
    int ci, co, level;
};
constexpr int kNumLayers = 9;
constexpr LayerDesc kLayers[kNumLayers] = {{2, 16, 0},  {16, 16, 0}, {16, 32, 1}, {32, 32, 1}, {32, 64, 2},
                                           {64, 64, 2}, {96, 32, 1}, {48, 16, 0}, {16, 1, 0}};
constexpr int64_t layer_size(int l) { return (int64_t)kLayers[l].co * 27 * kLayers[l].ci; }
constexpr int64_t layer_offset(int l) { return l == 0 ? 0 : layer_offset(l - 1) + layer_size(l - 1); }
constexpr int64_t kNumWeights = layer_offset(kNumLayers);
static_assert(kNumWeights == GBPCG_NN_NUM_WEIGHTS, "weight count");

// ------------------------------------------------------ small helpers ------

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline unsigned blocks_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)device_sm_count() * 16));
}
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Tile of the tensor-core convolution for a grid, if it has one.
inline bool conv_tile(int X, int Y, int Z, ConvTile *t) {
    if (X % 128 == 0) {
        *t = {128, 1, 1};
        return true;
    }
    if (128 % X) return false;
    const int ty = 128 / X;
    if (Y % ty == 0) {
        *t = {X, ty, 1};
        return true;
    }
    if (ty % Y) return false;
    const int tz = ty / Y;
    if (Z % tz) return false;
    *t = {X, Y, tz};
    return true;
}

// ----------------------------------------------- tensor-core convolution --

template <int CO, typename OUT>
static int conv_tc_launch(int X, int Y, int Z, int ci, const __nv_bfloat16 *in, const __nv_bfloat16 *w, OUT *out,
                          int cstride, int coff, int relu, const __nv_bfloat16 *mask, int mstride, int moff, int *err,
                          cudaStream_t s) {
    ConvArgs a;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.ci = ci;
    a.co = CO;
    if (!conv_tile(X, Y, Z, &a.tile)) return fail_arg("grid has no 128-voxel convolution tile");
    a.out = out;
    a.cstride = cstride;
    a.coff = coff;
    a.relu = relu;
    a.mask = mask;
    a.mstride = mstride;
    a.moff = moff;
    a.err = err;
    ConvMaps maps;
    const uint64_t dims[4] = {(uint64_t)ci, (uint64_t)X, (uint64_t)Y, (uint64_t)Z};
    const uint64_t strides[3] = {(uint64_t)ci * 2, (uint64_t)ci * 2 * X, (uint64_t)ci * 2 * X * Y};
    const uint32_t box[4] = {8, (uint32_t)a.tile.tx, (uint32_t)a.tile.ty, (uint32_t)a.tile.tz};
    int rc = make_map_nd(&maps.act, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, in, 4, dims, strides, box);
    if (rc) return rc;
    const uint64_t wd[2] = {(uint64_t)27 * ci, (uint64_t)CO};
    const uint64_t wst[1] = {(uint64_t)27 * ci * 2};
    const uint32_t wb[2] = {8, (uint32_t)CO};
    rc = make_map_nd(&maps.wgt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w, 2, wd, wst, wb);
    if (rc) return rc;
    if constexpr (CO == 16) {
        const int kc = ci / 16;
        const uint32_t wbytes = ZmCfg::wbytes(kc);
        // shared memory a CTA may use, less a margin for the static barriers
        constexpr uint32_t kSmemBudget = 227u * 1024u - 2048u;
        const int stages =
            wbytes >= kSmemBudget ? 0 : (int)std::min<uint32_t>(kZmMaxStages, (kSmemBudget - wbytes) / ZmCfg::A_STAGE);
        if (X % 128 == 0 && stages >= 3) {
            // rows of 128: the z-marching kernel; A box (8, 130, 5, 1), one source plane per load
            const uint32_t zbox[4] = {8, (uint32_t)kHaloX, (uint32_t)ZmCfg::NR, 1};
            rc = make_map_nd(&maps.act, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, in, 4, dims, strides, zbox);
            if (rc) return rc;
            // weights (Co, 27, Ci) viewed as (channel, co, dy, dx, dz): one box holds a source plane's
            // 9 taps of 8 channels as [dx][dy][co][8 channels], so the dy taps of one dx are
            // consecutive rows of the B operand
            const uint64_t w5d[5] = {(uint64_t)ci, (uint64_t)CO, 3, 3, 3};
            const uint64_t w5s[4] = {(uint64_t)27 * ci * 2, (uint64_t)3 * ci * 2, (uint64_t)ci * 2,
                                     (uint64_t)9 * ci * 2};
            const uint32_t w5b[5] = {8, (uint32_t)CO, 3, 3, 1};
            rc = make_map_nd(&maps.wgt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w, 5, w5d, w5s, w5b);
            if (rc) return rc;
            static std::once_flag zonce;
            std::call_once(zonce, [] {
                cudaFuncSetAttribute(conv3_tc_zmarch_kernel<OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBudget);
            });
            // one CTA per SM (it holds all 512 TMEM columns); z segments per column chosen so that
            // the CTA with the most work marches the fewest source planes
            const int G = device_sm_count();
            const int64_t ncols = (int64_t)(X / 128) * ((Y + ZmCfg::R - 1) / ZmCfg::R);
            int nseg = 1;
            int64_t best = INT64_MAX;
            for (int ns = 1; ns <= Z; ++ns) {
                const int64_t rounds = (ncols * ns + G - 1) / G;
                const int64_t cost = rounds * ((Z + ns - 1) / ns + 2);
                if (cost < best) {
                    best = cost;
                    nseg = ns;
                }
            }
            if (ncols * nseg > INT32_MAX) return fail_arg("convolution grid too large");
            a.nseg = nseg;
            a.stages = stages;
            const int64_t grid = std::min<int64_t>(ncols * nseg, G);
            const uint32_t smem = wbytes + (uint32_t)stages * ZmCfg::A_STAGE;
            conv3_tc_zmarch_kernel<OUT><<<(unsigned)grid, 192, smem, s>>>(maps, a);
            cudaError_t e = cudaGetLastError();
            return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "conv3_tc_zmarch launch");
        }
    }
    if (X % 128 == 0 && Y % kHaloRows == 0 && Z <= 65535) {
        // rows of 128: the halo-slab kernel, whose A box is (8, 130, rows + 2, 1)
        const uint32_t hbox[4] = {8, (uint32_t)kHaloX, (uint32_t)kHaloRows + 2, 1};
        rc = make_map_nd(&maps.act, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, in, 4, dims, strides, hbox);
        if (rc) return rc;
        // weights as (channel, co, tap): one box carries a plane's 9 taps of 8 channels in the
        // [tap][co][8 channels] order of the B operand (one copy per stage half instead of nine)
        const uint64_t w3d[3] = {(uint64_t)ci, (uint64_t)CO, 27};
        const uint64_t w3s[2] = {(uint64_t)27 * ci * 2, (uint64_t)ci * 2};
        const uint32_t w3b[3] = {8, (uint32_t)CO, 9};
        rc = make_map_nd(&maps.wgt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w, 3, w3d, w3s, w3b);
        if (rc) return rc;
        constexpr uint32_t hsmem = HaloCfg<CO>::SMEM;
        static std::once_flag honce;
        std::call_once(honce, [] {
            cudaFuncSetAttribute(conv3_tc_halo_kernel<CO, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)hsmem);
        });
        conv3_tc_halo_kernel<CO, OUT><<<dim3(X / 128, Y / kHaloRows, Z), 128, hsmem, s>>>(maps, a);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "conv3_tc_halo launch");
    }
    constexpr uint32_t smem = conv_smem_bytes<CO>();
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(conv3_tc_kernel<CO, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    const int64_t tiles = (int64_t)X * Y * Z / 128;
    conv3_tc_kernel<CO, OUT><<<(unsigned)tiles, 128, smem, s>>>(maps, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "conv3_tc launch");
}

template <typename OUT>
static int conv_tc(int X, int Y, int Z, int ci, int co, const __nv_bfloat16 *in, const __nv_bfloat16 *w, OUT *out,
                   int cstride, int coff, int relu, const __nv_bfloat16 *mask, int mstride, int moff, int *err,
                   cudaStream_t s) {
    switch (co) {
        case 16: return conv_tc_launch<16, OUT>(X, Y, Z, ci, in, w, out, cstride, coff, relu, mask, mstride, moff, err, s);
        case 32: return conv_tc_launch<32, OUT>(X, Y, Z, ci, in, w, out, cstride, coff, relu, mask, mstride, moff, err, s);
        case 48: return conv_tc_launch<48, OUT>(X, Y, Z, ci, in, w, out, cstride, coff, relu, mask, mstride, moff, err, s);
        case 64: return conv_tc_launch<64, OUT>(X, Y, Z, ci, in, w, out, cstride, coff, relu, mask, mstride, moff, err, s);
        case 96: return conv_tc_launch<96, OUT>(X, Y, Z, ci, in, w, out, cstride, coff, relu, mask, mstride, moff, err, s);
        default: return fail_arg("tensor-core convolution output channels must be 16, 32, 48, 64 or 96");
    }
}

inline bool conv_tc_ok(int X, int Y, int Z, int ci, int co) {
    ConvTile t;
    return ci % 16 == 0 && ci <= 256 && (co == 16 || co == 32 || co == 48 || co == 64 || co == 96) &&
           conv_tile(X, Y, Z, &t);
}

// ------------------------------------------------ CUDA-core convolution ----
// For the 1- and 2-channel ends of the network.  A thread computes VX
// consecutive x voxels: for each of the 9 (dy, dz) source rows it loads the
// VX + 2 input positions once and applies the 3 x-taps to all VX outputs, so
// loads and shared-memory weight reads are shared by VX outputs.  Weights
// (CO, 27, CI) sit in shared memory as FP32 [t][i][o].

template <int C, typename T>
__device__ __forceinline__ void load_ch(const T *p, float v[C]) {
    if constexpr (C % 8 == 0 && std::is_same<T, __nv_bfloat16>::value) {
#pragma unroll
        for (int i = 0; i < C; i += 8) ld8(p + i, v + i);
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = to_f(p[i]);
    }
}

template <int CI, int CO, int VX, typename TO>
__global__ void __launch_bounds__(256)
    conv3_simt_kernel(int X, int Y, int Z, const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ w,
                      TO *__restrict__ out, int relu, const __nv_bfloat16 *__restrict__ mask, int mstride, int moff,
                      const double *scale, const float *__restrict__ vscale) {
    __shared__ __align__(16) float ws[27 * CI * CO];
    for (int e = threadIdx.x; e < 27 * CI * CO; e += blockDim.x) {
        const int o = e / (27 * CI), r = e - o * 27 * CI;  // r = t * CI + i
        ws[r * CO + o] = __bfloat162float(w[e]);
    }
    __syncthreads();
    const float sc = scale ? (float)*scale : 1.0f;
    const int XQ = X / VX;
    const int64_t n = (int64_t)XQ * Y * Z;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int xq = (int)(u % XQ), y = (int)((u / XQ) % Y), z = (int)(u / ((int64_t)XQ * Y));
        const int x0 = xq * VX;
        float acc[VX][CO];
#pragma unroll
        for (int j = 0; j < VX; ++j)
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[j][o] = 0.0f;
#pragma unroll 1
        for (int r9 = 0; r9 < 9; ++r9) {
            const int yy = y + r9 % 3 - 1, zz = z + r9 / 3 - 1;
            if (yy < 0 || yy >= Y || zz < 0 || zz >= Z) continue;
            const __nv_bfloat16 *row = in + (((int64_t)zz * Y + yy) * X) * CI;
            float iv[VX + 2][CI];
#pragma unroll
            for (int q = 0; q < VX + 2; ++q) {
                const int xx = x0 - 1 + q;
                if (xx >= 0 && xx < X) {
                    load_ch<CI>(row + (int64_t)xx * CI, iv[q]);
                } else {
#pragma unroll
                    for (int i = 0; i < CI; ++i) iv[q][i] = 0.0f;
                }
            }
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const float *wt = ws + (r9 * 3 + dx) * CI * CO;  // tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)
#pragma unroll
                for (int i = 0; i < CI; ++i) {
                    if constexpr (CO % 4 == 0) {
#pragma unroll
                        for (int o = 0; o < CO; o += 4) {
                            const float4 wv = *reinterpret_cast<const float4 *>(wt + i * CO + o);
#pragma unroll
                            for (int j = 0; j < VX; ++j) {
                                const float a = iv[j + dx][i];
                                acc[j][o] = fmaf(a, wv.x, acc[j][o]);
                                acc[j][o + 1] = fmaf(a, wv.y, acc[j][o + 1]);
                                acc[j][o + 2] = fmaf(a, wv.z, acc[j][o + 2]);
                                acc[j][o + 3] = fmaf(a, wv.w, acc[j][o + 3]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int o = 0; o < CO; ++o) {
                            const float wv = wt[i * CO + o];
#pragma unroll
                            for (int j = 0; j < VX; ++j) acc[j][o] = fmaf(iv[j + dx][i], wv, acc[j][o]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < VX; ++j) {
            const int64_t v = ((int64_t)z * Y + y) * X + x0 + j;
            TO *po = out + v * CO;
            const float vs = vscale ? sc * vscale[v] : sc;
#pragma unroll
            for (int o = 0; o < CO; ++o) {
                float f = acc[j][o] * vs;
                if (relu) f = f < 0.0f ? 0.0f : f;  // NaN passes
                if (mask && !(__bfloat162float(mask[v * mstride + moff + o]) > 0.0f)) f = 0.0f;
                acc[j][o] = f;
            }
            if constexpr (CO % 8 == 0 && std::is_same<TO, __nv_bfloat16>::value) {
#pragma unroll
                for (int o = 0; o < CO; o += 8) st8(po + o, acc[j] + o);
            } else {
#pragma unroll
                for (int o = 0; o < CO; ++o) po[o] = from_f<TO>(acc[j][o]);
            }
        }
    }
}

// Strided variant for wide inputs (CI a multiple of 8, X a multiple of 128): a
// warp owns 128 consecutive x voxels of a row and lane l computes x = l + 32 j
// (j < 4), so every warp-wide load reads contiguous memory (one 16-byte vector
// per lane, 512 B per instruction) while each shared-memory weight read still
// feeds four outputs.  The x - 1 / x + 1 neighbours are loaded too (L1 hits).
template <int CI, int CO, typename TO>
__global__ void __launch_bounds__(256)
    conv3_simt_strided_kernel(int X, int Y, int Z, const __nv_bfloat16 *__restrict__ in,
                              const __nv_bfloat16 *__restrict__ w, TO *__restrict__ out, int relu,
                              const __nv_bfloat16 *__restrict__ mask, int mstride, int moff, const double *scale,
                              const float *__restrict__ vscale) {
    constexpr int VX = 4;
    __shared__ __align__(16) float ws[27 * CI * CO];
    for (int e = threadIdx.x; e < 27 * CI * CO; e += blockDim.x) {
        const int o = e / (27 * CI), r = e - o * 27 * CI;  // r = t * CI + i
        ws[r * CO + o] = __bfloat162float(w[e]);
    }
    __syncthreads();
    const float sc = scale ? (float)*scale : 1.0f;
    const int lane = threadIdx.x & 31;
    const int XS = X / 128;
    const int64_t nseg = (int64_t)XS * Y * Z;
    const int64_t wpb = blockDim.x / 32;
    for (int64_t sg = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); sg < nseg; sg += (int64_t)gridDim.x * wpb) {
        const int xs = (int)(sg % XS), y = (int)((sg / XS) % Y), z = (int)(sg / ((int64_t)XS * Y));
        const int xb = xs * 128 + lane;
        float acc[VX][CO];
#pragma unroll
        for (int j = 0; j < VX; ++j)
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[j][o] = 0.0f;
#pragma unroll 1
        for (int r9 = 0; r9 < 9; ++r9) {
            const int yy = y + r9 % 3 - 1, zz = z + r9 / 3 - 1;
            if (yy < 0 || yy >= Y || zz < 0 || zz >= Z) continue;
            const __nv_bfloat16 *row = in + (((int64_t)zz * Y + yy) * X) * CI;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                float iv[VX][CI];
#pragma unroll
                for (int j = 0; j < VX; ++j) {
                    const int xx = xb + 32 * j + dx - 1;
                    if (xx >= 0 && xx < X) {
                        load_ch<CI>(row + (int64_t)xx * CI, iv[j]);
                    } else {
#pragma unroll
                        for (int i = 0; i < CI; ++i) iv[j][i] = 0.0f;
                    }
                }
                const float *wt = ws + (r9 * 3 + dx) * CI * CO;
#pragma unroll
                for (int i = 0; i < CI; ++i)
#pragma unroll
                    for (int o = 0; o < CO; ++o) {
                        const float wv = wt[i * CO + o];
#pragma unroll
                        for (int j = 0; j < VX; ++j) acc[j][o] = fmaf(iv[j][i], wv, acc[j][o]);
                    }
            }
        }
#pragma unroll
        for (int j = 0; j < VX; ++j) {
            const int64_t v = ((int64_t)z * Y + y) * X + xb + 32 * j;
            TO *po = out + v * CO;
            const float vs = vscale ? sc * vscale[v] : sc;
#pragma unroll
            for (int o = 0; o < CO; ++o) {
                float f = acc[j][o] * vs;
                if (relu) f = f < 0.0f ? 0.0f : f;  // NaN passes
                if (mask && !(__bfloat162float(mask[v * mstride + moff + o]) > 0.0f)) f = 0.0f;
                po[o] = from_f<TO>(f);
            }
        }
    }
}

// One output channel (the network's last layer, 16 -> 1), marching in z: warp w of a block owns
// 128 consecutive x outputs of one row (lane l: x = x0 + l + 32 j, j = 0..3) over a z range and
// keeps the partial sums of three output planes in registers.  For input plane m and row y + dy a
// thread loads its own four voxels only (one warp load covers 32 consecutive voxels: 16-byte
// pieces 32 bytes apart, not one piece per 128-byte line) and forms, per voxel, the nine products
// of its CI channels with taps (dz, dy, dx).  Output x adds the dx = 0 product of voxel x, and the
// dx = -1 product of voxel x - 1 and the dx = +1 product of voxel x + 1, which arrive from the
// neighbouring lanes by shuffles; lanes 0 and 31 also form the product of the voxel just outside
// the warp's 128 (x0 - 1, x0 + 128).  Input plane m feeds output planes m + 1, m and m - 1; plane
// m - 1 is then complete and written.  Per output: 27 CI multiply-adds from CI / 8 x 3 sixteen-byte
// loads per input plane.
constexpr int kC1Rows = 8, kC1Chunk = 16;

template <int CI, typename TO>
__global__ void __launch_bounds__(32 * kC1Rows, 2)
    conv3_c1_march_kernel(int X, int Y, int Z, const __nv_bfloat16 *__restrict__ in,
                          const __nv_bfloat16 *__restrict__ w, TO *__restrict__ out, int relu,
                          const __nv_bfloat16 *__restrict__ mask, int mstride, int moff, const double *scale,
                          const float *__restrict__ vscale) {
    static_assert(CI % 8 == 0, "channels come in 16-byte groups");
    __shared__ __align__(16) float ws[27 * CI];  // ws[t * CI + i], t = 9 (dz+1) + 3 (dy+1) + (dx+1)
    for (int e = threadIdx.x; e < 27 * CI; e += blockDim.x) ws[e] = __bfloat162float(w[e]);
    __syncthreads();
    const float sc = scale ? (float)*scale : 1.0f;
    const int lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * 128;
    const int y = blockIdx.y * kC1Rows + (threadIdx.x >> 5);
    const int zb = blockIdx.z * kC1Chunk, ze = min(Z, zb + kC1Chunk);
    // the edge voxel lane 0 (x0 - 1, tap dx = -1) or lane 31 (x0 + 128, tap dx = +1) also forms
    const int ex = lane == 0 ? x0 - 1 : x0 + 128, edx = lane == 0 ? 0 : 2;
    float ap[4], ac[4], an[4];  // partial sums of output planes m - 1, m, m + 1 at x0 + lane + 32 j
#pragma unroll
    for (int j = 0; j < 4; ++j) ap[j] = ac[j] = an[j] = 0.0f;
    for (int m = zb - 1; m <= ze; ++m) {
        // which of the three output planes this input plane still feeds (uniform over the block)
        const bool fn = m + 1 >= zb && m + 1 < ze, fc = m >= zb && m < ze, fp = m - 1 >= zb && m - 1 < ze;
        if (y < Y && m >= 0 && m < Z) {  // uniform over the warp
#pragma unroll 1
            for (int r = 0; r < 3; ++r) {
                const int yy = y + r - 1;
                if (yy < 0 || yy >= Y) continue;
                const __nv_bfloat16 *row = in + ((int64_t)m * Y + yy) * X * CI;
                float P[4][3][3];  // [voxel j][dz + 1][dx + 1]
                float E[3];        // the edge voxel's product with tap dx = edx, per dz + 1
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
                        for (int d3 = 0; d3 < 3; ++d3) P[j][a3][d3] = 0.0f;
#pragma unroll
                for (int a3 = 0; a3 < 3; ++a3) E[a3] = 0.0f;
#pragma unroll
                for (int cb = 0; cb < CI; cb += 8) {
                    float v[4][8], ve[8];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int xx = x0 + lane + 32 * j;
                        if (xx < X) {
                            ld8(row + (int64_t)xx * CI + cb, v[j]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 8; ++c) v[j][c] = 0.0f;
                        }
                    }
                    if (ex >= 0 && ex < X) {
                        ld8(row + (int64_t)ex * CI + cb, ve);
                    } else {
#pragma unroll
                        for (int c = 0; c < 8; ++c) ve[c] = 0.0f;
                    }
#pragma unroll
                    for (int a3 = 0; a3 < 3; ++a3) {
                        if (!(a3 == 0 ? fn : a3 == 1 ? fc : fp)) continue;
#pragma unroll
                        for (int d3 = 0; d3 < 3; ++d3) {
                            const float *wt = ws + (a3 * 9 + r * 3 + d3) * CI + cb;
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                const float wv = wt[c];
#pragma unroll
                                for (int j = 0; j < 4; ++j) P[j][a3][d3] = fmaf(wv, v[j][c], P[j][a3][d3]);
                            }
                        }
                        const float *we = ws + (a3 * 9 + r * 3 + edx) * CI + cb;
#pragma unroll
                        for (int c = 0; c < 8; ++c) E[a3] = fmaf(we[c], ve[c], E[a3]);
                    }
                }
                // output x0 + lane + 32 j adds P[j][.][1] of its own voxel, P[.][.][0] of voxel x - 1
                // (lane - 1, or lane 31 of the previous j, or lane 0's edge product) and
                // P[.][.][2] of voxel x + 1 (lane + 1, or lane 0 of the next j, or lane 31's edge)
#pragma unroll
                for (int a3 = 0; a3 < 3; ++a3) {
                    if (!(a3 == 0 ? fn : a3 == 1 ? fc : fp)) continue;
                    const float e_lo = __shfl_sync(0xffffffffu, E[a3], 0);
                    const float e_hi = __shfl_sync(0xffffffffu, E[a3], 31);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float lo = __shfl_up_sync(0xffffffffu, P[j][a3][0], 1);
                        float hi = __shfl_down_sync(0xffffffffu, P[j][a3][2], 1);
                        const float lo_w = __shfl_sync(0xffffffffu, P[j > 0 ? j - 1 : 0][a3][0], 31);
                        const float hi_w = __shfl_sync(0xffffffffu, P[j < 3 ? j + 1 : 3][a3][2], 0);
                        if (lane == 0) lo = j > 0 ? lo_w : e_lo;
                        if (lane == 31) hi = j < 3 ? hi_w : e_hi;
                        const float sum = P[j][a3][1] + lo + hi;
                        if (a3 == 0) an[j] += sum;       // dz = -1: output plane m + 1 reads input plane m
                        else if (a3 == 1) ac[j] += sum;
                        else ap[j] += sum;               // dz = +1: output plane m - 1
                    }
                }
            }
        }
        if (fp && y < Y) {  // output plane m - 1 has all three input planes
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int xx = x0 + lane + 32 * j;
                if (xx >= X) continue;
                const int64_t v = ((int64_t)(m - 1) * Y + y) * X + xx;
                float f = ap[j] * (vscale ? sc * vscale[v] : sc);
                if (relu) f = f < 0.0f ? 0.0f : f;  // NaN passes
                if (mask && !(__bfloat162float(mask[v * mstride + moff]) > 0.0f)) f = 0.0f;
                out[v] = from_f<TO>(f);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ap[j] = ac[j];
            ac[j] = an[j];
            an[j] = 0.0f;
        }
    }
}

template <int CI, int CO, typename TO>
static int conv_simt_launch(int X, int Y, int Z, const __nv_bfloat16 *in, const __nv_bfloat16 *w, TO *out, int relu,
                            const __nv_bfloat16 *mask, int mstride, int moff, const double *scale,
                            const float *vscale, cudaStream_t s) {
    if constexpr (CO == 1 && CI % 8 == 0) {
        {
            const dim3 grid((unsigned)((X + 127) / 128), (unsigned)((Y + kC1Rows - 1) / kC1Rows),
                            (unsigned)((Z + kC1Chunk - 1) / kC1Chunk));
            conv3_c1_march_kernel<CI, TO><<<grid, 32 * kC1Rows, 0, s>>>(X, Y, Z, in, w, out, relu, mask, mstride,
                                                                        moff, scale, vscale);
            cudaError_t e = cudaGetLastError();
            return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "conv3_c1_march launch");
        }
    }
    if (CI % 8 == 0 && X % 128 == 0) {
        const int64_t nseg = (int64_t)(X / 128) * Y * Z;  // one warp per 128-voxel row segment
        conv3_simt_strided_kernel<CI, CO, TO><<<blocks_for(nseg * 32, 256), 256, 0, s>>>(
            X, Y, Z, in, w, out, relu, mask, mstride, moff, scale, vscale);
    } else if (X % 4 == 0) {
        const int64_t n = (int64_t)(X / 4) * Y * Z;
        conv3_simt_kernel<CI, CO, 4, TO><<<blocks_for(n, 256), 256, 0, s>>>(X, Y, Z, in, w, out, relu, mask, mstride,
                                                                             moff, scale, vscale);
    } else {
        const int64_t n = (int64_t)X * Y * Z;
        conv3_simt_kernel<CI, CO, 1, TO><<<blocks_for(n, 256), 256, 0, s>>>(X, Y, Z, in, w, out, relu, mask, mstride,
                                                                             moff, scale, vscale);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "conv3_simt launch");
}

inline bool conv_simt_ok(int ci, int co) { return (ci == 2 && co == 16) || (ci == 16 && co == 1) || (ci == 1 && co == 16); }

// out = conv(in) * (*scale) * vscale[v] (either factor optional)
template <typename TO>
static int conv_simt(int X, int Y, int Z, int ci, int co, const __nv_bfloat16 *in, const __nv_bfloat16 *w, TO *out,
                     int relu, const __nv_bfloat16 *mask, int mstride, int moff, const double *scale,
                     cudaStream_t s, const float *vscale = nullptr) {
    if (ci == 2 && co == 16)
        return conv_simt_launch<2, 16, TO>(X, Y, Z, in, w, out, relu, mask, mstride, moff, scale, vscale, s);
    if (ci == 16 && co == 1)
        return conv_simt_launch<16, 1, TO>(X, Y, Z, in, w, out, relu, mask, mstride, moff, scale, vscale, s);
    if (ci == 1 && co == 16)
        return conv_simt_launch<1, 16, TO>(X, Y, Z, in, w, out, relu, mask, mstride, moff, scale, vscale, s);
    return fail_arg("no CUDA-core convolution for these channel counts");
}

// ------------------------------------------------------ weight gradients --
// gW[o, t, i] = sum_v gy[v, o] x[v + off(t), i].  A block owns up to 256
// (tap, 4-output, 4-input) register blocks and a range of grid rows; it
// stages one row segment of W voxels at a time (the 9 input rows it touches,
// with a one-voxel halo, and the matching gy) in shared memory as FP32 and
// accumulates outer products.  Each block writes its sums to its own slot of
// a partial buffer; a second kernel adds the slots in a fixed order.

constexpr int kWgThreads = 256;
constexpr int kWgTargetBlocks = 608;

__host__ __device__ constexpr int wg_xs_floats(int W, int ci) { return (9 * (W + 2) * ci + 3) & ~3; }

template <int BO, int BI>
__global__ void __launch_bounds__(kWgThreads)
    wgrad_kernel(int X, int Y, int Z, int ci, int co, int W, int rows_per_block, const __nv_bfloat16 *__restrict__ x,
                 const __nv_bfloat16 *__restrict__ gy, float *__restrict__ partials) {
    extern __shared__ __align__(16) float wsm[];
    float *xs = wsm;                         // [9][W + 2][ci]
    float *gs = wsm + wg_xs_floats(W, ci);   // [W][co], 16-byte aligned
    const int nob = co / BO, nib = ci / BI;
    const int ncombo = 27 * nob * nib;
    const int c = blockIdx.y * kWgThreads + threadIdx.x;
    const bool active = c < ncombo;
    const int t = active ? c / (nob * nib) : 0;
    const int ob = active ? (c / nib) % nob : 0;
    const int ib = active ? c % nib : 0;
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int rk = (dz + 1) * 3 + (dy + 1);
    float acc[BO][BI];
#pragma unroll
    for (int o = 0; o < BO; ++o)
#pragma unroll
        for (int i = 0; i < BI; ++i) acc[o][i] = 0.0f;

    const int nrows = Y * Z;
    const int r0 = blockIdx.x * rows_per_block, r1 = min(nrows, r0 + rows_per_block);
    const int W2 = W + 2;
    for (int row = r0; row < r1; ++row) {
        const int y = row % Y, z = row / Y;
        for (int x0 = 0; x0 < X; x0 += W) {
            __syncthreads();
            // stage x: 9 rows x (W + 2) voxels x ci channels
            if (ci % 8 == 0) {
                const int nch = ci / 8, tot = 9 * W2 * nch;
                for (int e = threadIdx.x; e < tot; e += kWgThreads) {
                    const int ch = e % nch, j = (e / nch) % W2, rr = e / (nch * W2);
                    const int xx = x0 - 1 + j, yy = y + rr % 3 - 1, zz = z + rr / 3 - 1;
                    float v8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (xx >= 0 && xx < X && yy >= 0 && yy < Y && zz >= 0 && zz < Z)
                        ld8(x + (((int64_t)zz * Y + yy) * X + xx) * ci + ch * 8, v8);
                    float *d = xs + (rr * W2 + j) * ci + ch * 8;
#pragma unroll
                    for (int q = 0; q < 8; ++q) d[q] = v8[q];
                }
            } else {
                const int tot = 9 * W2 * ci;
                for (int e = threadIdx.x; e < tot; e += kWgThreads) {
                    const int ch = e % ci, j = (e / ci) % W2, rr = e / (ci * W2);
                    const int xx = x0 - 1 + j, yy = y + rr % 3 - 1, zz = z + rr / 3 - 1;
                    float v = 0.0f;
                    if (xx >= 0 && xx < X && yy >= 0 && yy < Y && zz >= 0 && zz < Z)
                        v = __bfloat162float(x[(((int64_t)zz * Y + yy) * X + xx) * ci + ch]);
                    xs[(rr * W2 + j) * ci + ch] = v;
                }
            }
            // stage gy: W voxels x co channels
            {
                const int64_t base = (((int64_t)z * Y + y) * X + x0) * co;
                for (int e = threadIdx.x; e < W * co; e += kWgThreads) gs[e] = __bfloat162float(gy[base + e]);
            }
            __syncthreads();
            if (active) {
                const float *xp = xs + (rk * W2 + 1 + dx) * ci + ib * BI;
                const float *gp = gs + ob * BO;
#pragma unroll 4
                for (int v = 0; v < W; ++v) {
                    float g[BO], xv[BI];
                    if constexpr (BO == 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(gp + v * co);
                        g[0] = q.x, g[1] = q.y, g[2] = q.z, g[3] = q.w;
                    } else {
#pragma unroll
                        for (int o = 0; o < BO; ++o) g[o] = gp[v * co + o];
                    }
                    if constexpr (BI == 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(xp + v * ci);
                        xv[0] = q.x, xv[1] = q.y, xv[2] = q.z, xv[3] = q.w;
                    } else {
#pragma unroll
                        for (int i = 0; i < BI; ++i) xv[i] = xp[v * ci + i];
                    }
#pragma unroll
                    for (int o = 0; o < BO; ++o)
#pragma unroll
                        for (int i = 0; i < BI; ++i) acc[o][i] = fmaf(g[o], xv[i], acc[o][i]);
                }
            }
        }
    }
    if (active) {
        float *dst = partials + (int64_t)blockIdx.x * (27 * co * ci);
#pragma unroll
        for (int o = 0; o < BO; ++o)
#pragma unroll
            for (int i = 0; i < BI; ++i) dst[((ob * BO + o) * 27 + t) * ci + ib * BI + i] = acc[o][i];
    }
}

__global__ void __launch_bounds__(256)
    sum_slots_kernel(int64_t n, int nslots, const float *__restrict__ partials, float *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) {
        float s = 0.0f;
        for (int k = 0; k < nslots; ++k) s += partials[(int64_t)k * n + e];
        out[e] = s;
    }
}

struct WgradPlan {
    int bo, bi, W, ngroups, S, rows_per_block;
    size_t smem;
};

inline WgradPlan wgrad_plan(int X, int Y, int Z, int ci, int co) {
    WgradPlan p;
    p.bo = co % 4 == 0 ? 4 : 1;
    p.bi = ci % 4 == 0 ? 4 : ci % 2 == 0 ? 2 : 1;
    const int ncombo = 27 * (co / p.bo) * (ci / p.bi);
    p.ngroups = (ncombo + kWgThreads - 1) / kWgThreads;
    p.W = std::min(X, ci <= 48 ? 32 : 16);
    const int rows = Y * Z;
    // about four blocks per SM of a 152-SM part; fixed so that workspace sizes
    // do not depend on the device that asks
    const int want = std::max(1, (kWgTargetBlocks + p.ngroups - 1) / p.ngroups);
    const int S0 = std::min(rows, want);
    p.rows_per_block = (rows + S0 - 1) / S0;
    p.S = (rows + p.rows_per_block - 1) / p.rows_per_block;
    p.smem = (size_t)(wg_xs_floats(p.W, ci) + p.W * co) * sizeof(float);
    return p;
}

inline bool wgrad_ok(int X, int ci, int co) {
    const int W = std::min(X, ci <= 48 ? 32 : 16);
    return X % W == 0 && (wg_xs_floats(W, ci) + W * co) * 4 <= 200 * 1024;
}

// Tensor-core weight gradient (wgrad_tc_kernel): Ci a multiple of 16, Co with
// 128 / Co taps per M tile, grids with 128-voxel tiles.
inline bool wgrad_tc_ok(int X, int Y, int Z, int ci, int co) {
    ConvTile t;
    return ci % 16 == 0 && ci <= 128 && (co == 16 || co == 32 || co == 48 || co == 64 || co == 96) &&
           conv_tile(X, Y, Z, &t) && ((int64_t)X * Y * Z) / 128 <= INT32_MAX;
}

struct WgTcPlan {
    int tp, mtiles, group, ngroups, chunks, cpc, S, stages;
    uint32_t a_bytes, stage_bytes, ncol;
    size_t smem;
};

inline WgTcPlan wgrad_tc_plan(int X, int Y, int Z, int ci, int co) {
    WgTcPlan p;
    p.tp = 128 / co;
    p.mtiles = (27 + p.tp - 1) / p.tp;
    p.group = std::min(p.mtiles, 512 / ci);
    p.ngroups = (p.mtiles + p.group - 1) / p.group;
    p.chunks = (int)(((int64_t)X * Y * Z) / 128);
    // about two CTAs per SM of a 152-SM part, fixed so that workspace sizes do
    // not depend on the device that asks
    const int S0 = std::max(1, std::min(p.chunks, (kWgTargetBlocks / 2 + p.ngroups - 1) / p.ngroups));
    p.cpc = (p.chunks + S0 - 1) / S0;
    p.S = (p.chunks + p.cpc - 1) / p.cpc;
    p.a_bytes = 16u * 2048u;
    p.stage_bytes = p.a_bytes + (uint32_t)(ci / 8) * 2048u;
    p.stages = (int)std::max<uint32_t>(2, std::min<uint32_t>(kWgMaxStages, (200u * 1024u) / p.stage_bytes));
    p.ncol = tmem_cols(p.group * ci);
    p.smem = (size_t)p.stages * p.stage_bytes;
    return p;
}

inline size_t wgrad_partial_bytes(int X, int Y, int Z, int ci, int co) {
    WgradPlan p = wgrad_plan(X, Y, Z, ci, co);
    size_t b = (size_t)p.S * 27 * ci * co * sizeof(float);
    if (wgrad_tc_ok(X, Y, Z, ci, co)) b = std::max(b, (size_t)wgrad_tc_plan(X, Y, Z, ci, co).S * 27 * ci * co * 4);
    return b;
}

static int wgrad_tc(int X, int Y, int Z, int ci, int co, const __nv_bfloat16 *x, const __nv_bfloat16 *gy, float *gw,
                    float *partials, int *err, cudaStream_t s) {
    const WgTcPlan p = wgrad_tc_plan(X, Y, Z, ci, co);
    WgArgs a;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.ci = ci;
    a.co = co;
    conv_tile(X, Y, Z, &a.tile);
    a.tp = p.tp;
    a.mtiles = p.mtiles;
    a.group = p.group;
    a.chunks = p.chunks;
    a.chunks_per_cta = p.cpc;
    a.stage_bytes = p.stage_bytes;
    a.a_bytes = p.a_bytes;
    a.stages = p.stages;
    a.ncol = p.ncol;
    a.partials = partials;
    a.err = err;
    WgMaps maps;
    const uint32_t box[4] = {8, (uint32_t)a.tile.tx, (uint32_t)a.tile.ty, (uint32_t)a.tile.tz};
    const uint64_t gd[4] = {(uint64_t)co, (uint64_t)X, (uint64_t)Y, (uint64_t)Z};
    const uint64_t gs[3] = {(uint64_t)co * 2, (uint64_t)co * 2 * X, (uint64_t)co * 2 * X * Y};
    int rc = make_map_nd(&maps.gy, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, gy, 4, gd, gs, box);
    if (rc) return rc;
    const uint64_t xd[4] = {(uint64_t)ci, (uint64_t)X, (uint64_t)Y, (uint64_t)Z};
    const uint64_t xs[3] = {(uint64_t)ci * 2, (uint64_t)ci * 2 * X, (uint64_t)ci * 2 * X * Y};
    rc = make_map_nd(&maps.x, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, x, 4, xd, xs, box);
    if (rc) return rc;
    cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    wgrad_tc_kernel<<<dim3(p.S, p.ngroups), 128, p.smem, s>>>(maps, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "wgrad_tc launch");
    const int64_t n = (int64_t)27 * ci * co;
    sum_slots_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, p.S, partials, gw);
    e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "sum_slots launch");
}

template <int BO, int BI>
static cudaError_t wgrad_launch(const WgradPlan &p, int X, int Y, int Z, int ci, int co, const __nv_bfloat16 *x,
                                const __nv_bfloat16 *gy, float *partials, cudaStream_t s) {
    cudaFuncSetAttribute(wgrad_kernel<BO, BI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    wgrad_kernel<BO, BI><<<dim3(p.S, p.ngroups), kWgThreads, p.smem, s>>>(X, Y, Z, ci, co, p.W, p.rows_per_block, x,
                                                                        gy, partials);
    return cudaGetLastError();
}

static int wgrad(int X, int Y, int Z, int ci, int co, const __nv_bfloat16 *x, const __nv_bfloat16 *gy, float *gw,
                 float *partials, cudaStream_t s, int *err = nullptr) {
    if (err && wgrad_tc_ok(X, Y, Z, ci, co)) return wgrad_tc(X, Y, Z, ci, co, x, gy, gw, partials, err, s);
    if (!wgrad_ok(X, ci, co)) return fail_arg("weight gradient: unsupported width or channel count");
    WgradPlan p = wgrad_plan(X, Y, Z, ci, co);
    cudaError_t e;
    if (p.bo == 4 && p.bi == 4) e = wgrad_launch<4, 4>(p, X, Y, Z, ci, co, x, gy, partials, s);
    else if (p.bo == 4 && p.bi == 2) e = wgrad_launch<4, 2>(p, X, Y, Z, ci, co, x, gy, partials, s);
    else if (p.bo == 4) e = wgrad_launch<4, 1>(p, X, Y, Z, ci, co, x, gy, partials, s);
    else if (p.bi == 4) e = wgrad_launch<1, 4>(p, X, Y, Z, ci, co, x, gy, partials, s);
    else if (p.bi == 2) e = wgrad_launch<1, 2>(p, X, Y, Z, ci, co, x, gy, partials, s);
    else e = wgrad_launch<1, 1>(p, X, Y, Z, ci, co, x, gy, partials, s);
    if (e != cudaSuccess) return fail_cuda(e, "wgrad launch");
    const int64_t n = (int64_t)27 * ci * co;
    sum_slots_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, p.S, partials, gw);
    e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "sum_slots launch");
}

// --------------------------------------------------------- glue kernels ----

// dsc = D^{-1/2} at every point.  D = sum over the six faces of k_f / h_d^2,
// with k_f the harmonic mean of the two cells' block coefficients on interior
// faces and the cell's own coefficient on boundary faces (kb == NULL: k = 1).
// It depends on the operator only, so a solve computes it once.
// Grid of the per-voxel kernels: 256 threads along x, one block row per y,
// and along z as many blocks as bring the grid to about 16 per SM (the
// kernels stride over the remaining planes, so per-thread set-up, such as
// nn_input_kernel's FP64 rms, is shared by several planes).
static dim3 xyz_grid(int X, int Y, int Z) {
    const int64_t gxy = (int64_t)((X + 255) / 256) * Y;
    const int64_t want = (int64_t)device_sm_count() * 16;
    const int64_t gz = std::max<int64_t>(1, std::min<int64_t>({(int64_t)Z, 65535, (want + gxy - 1) / gxy}));
    return dim3((unsigned)((X + 255) / 256), (unsigned)Y, (unsigned)gz);
}

// Threads take x, blocks y (blockIdx.y) and z (blockIdx.z, striding by
// gridDim.z): no division of a flat index per element; the block indices of
// a thread's column and of its x and y neighbours are fixed per thread.
__global__ void __launch_bounds__(256)
    jacobi_scale_kernel(int X, int Y, int Z, const float *__restrict__ kb, int kbx, int kby, int kbz,
                        float *__restrict__ dsc) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= X) return;
    const float cx = (float)(X + 1) * (float)(X + 1), cy = (float)(Y + 1) * (float)(Y + 1),
                cz = (float)(Z + 1) * (float)(Z + 1);
    const int nbx = (X + kbx - 1) / kbx, nby = (Y + kby - 1) / kby;
    const int bx = x / kbx, bxm = x > 0 ? (x - 1) / kbx : 0, bxp = x + 1 < X ? (x + 1) / kbx : 0;
    const int by = y / kby, bym = y > 0 ? (y - 1) / kby : 0, byp = y + 1 < Y ? (y + 1) / kby : 0;
    for (int z = blockIdx.z; z < Z; z += gridDim.z) {
        const int64_t v = ((int64_t)z * Y + y) * X + x;
        float d;
        if (!kb) {
            d = 2.0f * (cx + cy + cz);
        } else {
            const int bz = z / kbz, bzm = z > 0 ? (z - 1) / kbz : 0, bzp = z + 1 < Z ? (z + 1) / kbz : 0;
            auto K = [&](int px, int py, int pz) { return kb[((int64_t)pz * nby + py) * nbx + px]; };
            const float kc = K(bx, by, bz);
            // face coefficient: harmonic mean with the neighbour's block, the cell's own on the boundary
            auto face = [&](bool inside, int px, int py, int pz) {
                if (!inside) return kc;
                const float kn = K(px, py, pz);
                return 2.0f * kc * kn / (kc + kn);
            };
            d = cx * (face(x > 0, bxm, by, bz) + face(x + 1 < X, bxp, by, bz)) +
                cy * (face(y > 0, bx, bym, bz) + face(y + 1 < Y, bx, byp, bz)) +
                cz * (face(z > 0, bx, by, bzm) + face(z + 1 < Z, bx, by, bzp));
        }
        dsc[v] = 1.0f / sqrtf(d);
    }
}

// s = D^{-1/2} r (n a multiple of 4)
__global__ void __launch_bounds__(256)
    scale_residual_kernel(int64_t n4, const float *__restrict__ r, const float *__restrict__ dsc, float *__restrict__ sr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = reinterpret_cast<const float4 *>(r)[i], d = reinterpret_cast<const float4 *>(dsc)[i];
        reinterpret_cast<float4 *>(sr)[i] = make_float4(a.x * d.x, a.y * d.y, a.z * d.z, a.w * d.w);
    }
}

// Network input: channels (s / rms(s), log k) from the scaled residual s;
// also the output scale rms(s).
__global__ void __launch_bounds__(256)
    nn_input_kernel(int X, int Y, int Z, const float *__restrict__ sr, const double *ss, const float *__restrict__ kb,
                    int kbx, int kby, int kbz, __nv_bfloat16 *__restrict__ xin, double *scale) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;  // z: blockIdx.z, striding
    const int64_t n = (int64_t)X * Y * Z;
    const double rms = sqrt(*ss / (double)n);
    const float inv = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) *scale = rms;
    if (x >= X) return;
    const int nbx = (X + kbx - 1) / kbx, nby = (Y + kby - 1) / kby;
    const int bx = x / kbx, by = y / kby;
    for (int z = blockIdx.z; z < Z; z += gridDim.z) {
        const int64_t v = ((int64_t)z * Y + y) * X + x;
        const float lk = kb ? logf(kb[((int64_t)(z / kbz) * nby + by) * nbx + bx]) : 0.0f;
        __nv_bfloat162 p;
        p.x = __float2bfloat16_rn(sr[v] * inv);
        p.y = __float2bfloat16_rn(lk);
        reinterpret_cast<__nv_bfloat162 *>(xin)[v] = p;
    }
}

// The resampling kernels below map threads to (x, 8-channel group) along a
// row in blockIdx.x and threadIdx.x, and take y and z from blockIdx.y and
// blockIdx.z: no 64-bit division per element (a grid-stride loop with
// v % X, v / X per element made them issue-bound).
struct RowIdx {
    int x, ch, y, z;
};
template <int NC8>
__device__ __forceinline__ bool row_idx(int X, RowIdx &r) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    r.x = e / NC8;
    r.ch = e - r.x * NC8;
    r.y = blockIdx.y;
    r.z = blockIdx.z;
    return r.x < X;
}
inline dim3 row_grid(int X, int nc8, int Y, int Z) {
    return dim3((unsigned)((X * nc8 + 255) / 256), (unsigned)Y, (unsigned)Z);
}

// dst (coarse, C channels) = mean of the 2x2x2 children of src (channels
// [soff, soff + C) of sstride).  One thread per (coarse voxel, 8 channels).
template <int C>
__global__ void __launch_bounds__(256)
    pool2_kernel(int Xc, int Yc, int Zc, const __nv_bfloat16 *__restrict__ src, int sstride, int soff,
                 __nv_bfloat16 *__restrict__ dst) {
    RowIdx r;
    if (!row_idx<C / 8>(Xc, r)) return;
    const int Xf = 2 * Xc, Yf = 2 * Yc;
    const int64_t v = ((int64_t)r.z * Yc + r.y) * Xc + r.x;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int64_t f = (((int64_t)(2 * r.z + (c >> 2)) * Yf + 2 * r.y + ((c >> 1) & 1)) * Xf + 2 * r.x + (c & 1));
        float q[8];
        ld8(src + f * sstride + soff + r.ch * 8, q);
#pragma unroll
        for (int i = 0; i < 8; ++i) s[i] += q[i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] *= 0.125f;
    st8(dst + v * C + r.ch * 8, s);
}

// dst (fine, channels [doff, doff + C) of dstride) = src (coarse, C channels)
// of the parent voxel.
template <int C>
__global__ void __launch_bounds__(256)
    up2_kernel(int Xf, int Yf, int Zf, const __nv_bfloat16 *__restrict__ src, __nv_bfloat16 *__restrict__ dst,
               int dstride, int doff) {
    RowIdx r;
    if (!row_idx<C / 8>(Xf, r)) return;
    const int Xc = Xf / 2, Yc = Yf / 2;
    const int64_t v = ((int64_t)r.z * Yf + r.y) * Xf + r.x;
    const int64_t pv = ((int64_t)(r.z / 2) * Yc + r.y / 2) * Xc + r.x / 2;
    *reinterpret_cast<uint4 *>(dst + v * dstride + doff + r.ch * 8) =
        *reinterpret_cast<const uint4 *>(src + pv * C + r.ch * 8);
}

// dst (coarse, C channels, BF16) = (sum of the 8 fine children of g, FP32
// channels [goff, goff + C) of gstride) * (mask > 0): the adjoint of
// nearest upsampling followed by the ReLU derivative.
template <int C>
__global__ void __launch_bounds__(256)
    up2_adjoint_mask_kernel(int Xc, int Yc, int Zc, const float *__restrict__ g, int gstride, int goff,
                            const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ dst) {
    RowIdx r;
    if (!row_idx<C / 8>(Xc, r)) return;
    const int Xf = 2 * Xc, Yf = 2 * Yc;
    const int64_t v = ((int64_t)r.z * Yc + r.y) * Xc + r.x;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int64_t f = (((int64_t)(2 * r.z + (c >> 2)) * Yf + 2 * r.y + ((c >> 1) & 1)) * Xf + 2 * r.x + (c & 1));
        float q[8];
        ld8(g + f * gstride + goff + r.ch * 8, q);
#pragma unroll
        for (int i = 0; i < 8; ++i) s[i] += q[i];
    }
    float m[8];
    ld8(mask + v * C + r.ch * 8, m);
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = m[i] > 0.0f ? s[i] : 0.0f;
    st8(dst + v * C + r.ch * 8, s);
}

// dst (fine, C channels, BF16) = (skip + t(parent) / 8) * (mask > 0): the
// gradient reaching a skip connection, plus the adjoint of average pooling
// of the coarse gradient t, times the ReLU derivative.
template <int C>
__global__ void __launch_bounds__(256)
    pool_adjoint_skip_mask_kernel(int Xf, int Yf, int Zf, const float *__restrict__ skip, int sstride, int soff,
                                  const float *__restrict__ t, const __nv_bfloat16 *__restrict__ mask, int mstride,
                                  int moff, __nv_bfloat16 *__restrict__ dst) {
    RowIdx r;
    if (!row_idx<C / 8>(Xf, r)) return;
    const int Xc = Xf / 2, Yc = Yf / 2;
    const int64_t v = ((int64_t)r.z * Yf + r.y) * Xf + r.x;
    const int64_t pv = ((int64_t)(r.z / 2) * Yc + r.y / 2) * Xc + r.x / 2;
    float a[8], b[8], m[8];
    ld8(skip + v * sstride + soff + r.ch * 8, a);
    ld8(t + pv * C + r.ch * 8, b);
    ld8(mask + v * mstride + moff + r.ch * 8, m);
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = m[i] > 0.0f ? fmaf(b[i], 0.125f, a[i]) : 0.0f;
    st8(dst + v * C + r.ch * 8, a);
}

// g_out = dL/d(network output) = dL/dz * scale * dsc, rounded to BF16.
__global__ void __launch_bounds__(256)
    scale_to_bf16_kernel(int64_t n, const float *__restrict__ gz, const double *scale, const float *__restrict__ dsc,
                         __nv_bfloat16 *__restrict__ out) {
    const float sc = (float)*scale;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = __float2bfloat16_rn(gz[v] * sc * dsc[v]);
}

struct WeightTable {
    int64_t off[kNumLayers + 1];
    int ci[kNumLayers], co[kNumLayers];
};

inline WeightTable weight_table() {
    WeightTable t;
    for (int l = 0; l <= kNumLayers; ++l) t.off[l] = layer_offset(l);
    for (int l = 0; l < kNumLayers; ++l) t.ci[l] = kLayers[l].ci, t.co[l] = kLayers[l].co;
    return t;
}

// BF16 copies of the FP32 master weights: wf in the forward layout (Co, 27,
// Ci) and wflip[i, t, o] = W[o, 26 - t, i], the weights of the adjoint
// convolution (taps mirrored, channel roles swapped).
__global__ void __launch_bounds__(256)
    weight_prep_kernel(const WeightTable tab, const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf,
                       __nv_bfloat16 *__restrict__ wflip) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tab.off[kNumLayers];
         e += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (e >= tab.off[l + 1]) ++l;
        const int64_t r = e - tab.off[l];
        const int ci = tab.ci[l], co = tab.co[l];
        const int i = (int)(r % ci), t = (int)((r / ci) % 27), o = (int)(r / (27 * ci));
        const __nv_bfloat16 b = __float2bfloat16_rn(w[e]);
        wf[e] = b;
        if (wflip) wflip[tab.off[l] + ((int64_t)i * 27 + (26 - t)) * co + o] = b;
    }
}

// Adam (Kingma & Ba 2015) with bias correction, FP32 state; omb1 = 1 - b1
// and omb2 = 1 - b2 come from the host in double (1 - (float)0.999 is 1.3e-5
// off 1e-3).
__global__ void __launch_bounds__(256)
    adam_kernel(int64_t n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                float *__restrict__ v, float lr, float b1, float omb1, float b2, float omb2, float eps, float bc1,
                float bc2) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + omb1 * ge;
        const float ve = b2 * v[e] + omb2 * ge * ge;
        m[e] = me;
        v[e] = ve;
        w[e] -= lr * (me / bc1) / (sqrtf(ve / bc2) + eps);
    }
}

// Scale-free, sign-aware A-norm loss of one pair: with a = z.Ae, c = z.Az,
// E = e.Ae,
//   loss = 1/2 (1 - a |a| / (c E))  (= 1/2 ||s z - e||_A^2 / E, s = a / c,
//          for a >= 0; rising to 1 for negative multiples of e),
//   gz = dloss/dz = (|a| / (c E)) (s A z - A e).
// gz holds A z on entry.  z = 0 (c = 0) gives loss 1/2 and the gradient
// -A e / E of the unscaled loss there.
__global__ void __launch_bounds__(256)
    loss_finish_kernel(int64_t n, const double *sc, float *__restrict__ gz, const float *__restrict__ ae, double *loss) {
    const double a = sc[0], c = sc[1], E = sc[2];
    double coef = 0.0, sdir = 0.0, l = 0.0;
    if (c > 0.0 && E > 0.0) {
        coef = fabs(a) / (c * E);
        sdir = a / c;
        l = 0.5 * (1.0 - a * fabs(a) / (c * E));
    } else if (E > 0.0) {
        coef = 1.0 / E;
        sdir = 0.0;
        l = 0.5;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) *loss = l;
    const float fc = (float)coef, fs = (float)sdir;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        gz[v] = fc * fmaf(fs, gz[v], -ae[v]);
}

// ------------------------------------------------------ workspace layout --

struct NnLayout {
    int X[3], Y[3], Z[3];
    int64_t V[3];
    size_t wf, wflip, scal, err, dotws;
    size_t dsc, sr;  // D^{-1/2} and the scaled residual (FP32)
    size_t xin, a1, k8, p1, a3, k7, p2, a5, a6, a7, a8;
    size_t gout, ga8, gk8, ga7, gk7, ga6, ga5, t5, ge1b, ga3, t3, ge0b, ga1, part;
    size_t lae;  // loss scratch: A e
    size_t total;
};
// device scalars at layout.scal (doubles); S_LA..S_LE: z.Ae, z.Az, e.Ae
enum { S_RR = 0, S_SCALE, S_LA, S_LC, S_LE, S_LOSS, S_COUNT };

inline bool nn_shape_ok(int X, int Y, int Z) {
    if (X % 4 || Y % 4 || Z % 4) return false;
    for (int l = 0; l < 3; ++l) {
        ConvTile t;
        if (!conv_tile(X >> l, Y >> l, Z >> l, &t)) return false;
    }
    return true;
}

inline NnLayout nn_layout(int X, int Y, int Z, bool training) {
    NnLayout L;
    for (int l = 0; l < 3; ++l) {
        L.X[l] = X >> l, L.Y[l] = Y >> l, L.Z[l] = Z >> l;
        L.V[l] = (int64_t)L.X[l] * L.Y[l] * L.Z[l];
    }
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    const size_t B = 2, F = 4;
    L.wf = take(kNumWeights * B);
    L.wflip = take(kNumWeights * B);
    L.scal = take(S_COUNT * sizeof(double));
    L.err = take(sizeof(int));
    L.dotws = take(gbpcg_dot_workspace_size());
    L.dsc = take(L.V[0] * F);
    L.sr = take(L.V[0] * F);
    L.xin = take(L.V[0] * 2 * B);
    L.a1 = take(L.V[0] * 16 * B);
    L.k8 = take(L.V[0] * 48 * B);
    L.p1 = take(L.V[1] * 16 * B);
    L.a3 = take(L.V[1] * 32 * B);
    L.k7 = take(L.V[1] * 96 * B);
    L.p2 = take(L.V[2] * 32 * B);
    L.a5 = take(L.V[2] * 64 * B);
    L.a6 = take(L.V[2] * 64 * B);
    L.a7 = take(L.V[1] * 32 * B);
    L.a8 = take(L.V[0] * 16 * B);
    if (training) {
        L.gout = take(L.V[0] * B);
        L.ga8 = take(L.V[0] * 16 * B);
        L.gk8 = take(L.V[0] * 48 * F);
        L.ga7 = take(L.V[1] * 32 * B);
        L.gk7 = take(L.V[1] * 96 * F);
        L.ga6 = take(L.V[2] * 64 * B);
        L.ga5 = take(L.V[2] * 64 * B);
        L.t5 = take(L.V[2] * 32 * F);
        L.ge1b = take(L.V[1] * 32 * B);
        L.ga3 = take(L.V[1] * 32 * B);
        L.t3 = take(L.V[1] * 16 * F);
        L.ge0b = take(L.V[0] * 16 * B);
        L.ga1 = take(L.V[0] * 16 * B);
        size_t pb = 0;
        for (int l = 0; l < kNumLayers; ++l) {
            const int lv = kLayers[l].level;
            pb = std::max(pb, wgrad_partial_bytes(L.X[lv], L.Y[lv], L.Z[lv], kLayers[l].ci, kLayers[l].co));
        }
        L.part = take(pb);
        L.lae = take(L.V[0] * F);
    } else {
        L.gout = L.ga8 = L.gk8 = L.ga7 = L.gk7 = L.ga6 = L.ga5 = L.t5 = L.ge1b = L.ga3 = L.t3 = L.ge0b = L.ga1 =
            L.part = L.lae = 0;
    }
    L.total = o;
    return L;
}

struct NnPtrs {
    char *base;
    template <typename T>
    T *at(size_t off) const {
        return reinterpret_cast<T *>(base + off);
    }
};

using bf16 = __nv_bfloat16;

#define GB_TRY(expr)                     \
    do {                                 \
        int _rc = (expr);                \
        if (_rc != GBPCG_OK) return _rc; \
    } while (0)

// ----------------------------------------------------------- forward -------

int nn_weight_prep(const float *w, void *ws, const NnLayout &L, cudaStream_t s) {
    NnPtrs P{static_cast<char *>(ws)};
    weight_prep_kernel<<<blocks_for(kNumWeights, 256), 256, 0, s>>>(weight_table(), w, P.at<bf16>(L.wf),
                                                                     P.at<bf16>(L.wflip));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "weight_prep launch");
}

// D^{-1/2} of the grid's operator into the workspace.
int nn_diag_prep(const gbpcg_grid &g, void *ws, const NnLayout &L, cudaStream_t s) {
    NnPtrs P{static_cast<char *>(ws)};
    jacobi_scale_kernel<<<xyz_grid(L.X[0], L.Y[0], L.Z[0]), 256, 0, s>>>(L.X[0], L.Y[0], L.Z[0], g.k_block, g.kbx,
                                                                        g.kby, g.kbz, P.at<float>(L.dsc));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "jacobi_scale launch");
}

// z = N(r) with the BF16 weights (and, if dsc_ready, D^{-1/2}) already in the workspace.
int nn_forward_prepped(const gbpcg_grid &g, const float *r, float *z, void *ws, const NnLayout &L, cudaStream_t s,
                       bool dsc_ready = false) {
    NnPtrs P{static_cast<char *>(ws)};
    const int X0 = L.X[0], Y0 = L.Y[0], Z0 = L.Z[0], X1 = L.X[1], Y1 = L.Y[1], Z1 = L.Z[1], X2 = L.X[2], Y2 = L.Y[2],
              Z2 = L.Z[2];
    const bf16 *wf = P.at<bf16>(L.wf);
    auto W = [&](int l) { return wf + layer_offset(l); };
    double *sc = P.at<double>(L.scal);
    int *err = P.at<int>(L.err);
    float *dsc = P.at<float>(L.dsc), *sr = P.at<float>(L.sr);
    if (!dsc_ready) GB_TRY(nn_diag_prep(g, ws, L, s));
    scale_residual_kernel<<<blocks_for(L.V[0] / 4, 256), 256, 0, s>>>(L.V[0] / 4, r, dsc, sr);
    GB_CUDA(cudaGetLastError());
    GB_TRY(gbpcg_dot(L.V[0], GBPCG_F32, sr, sr, sc + S_RR, P.base + L.dotws, gbpcg_dot_workspace_size(),
                     (gbpcg_stream)s));
    nn_input_kernel<<<xyz_grid(X0, Y0, Z0), 256, 0, s>>>(X0, Y0, Z0, sr, sc + S_RR, g.k_block, g.kbx, g.kby, g.kbz,
                                                         P.at<bf16>(L.xin), sc + S_SCALE);
    GB_CUDA(cudaGetLastError());
    bf16 *a1 = P.at<bf16>(L.a1), *k8 = P.at<bf16>(L.k8), *p1 = P.at<bf16>(L.p1), *a3 = P.at<bf16>(L.a3),
         *k7 = P.at<bf16>(L.k7), *p2 = P.at<bf16>(L.p2), *a5 = P.at<bf16>(L.a5), *a6 = P.at<bf16>(L.a6),
         *a7 = P.at<bf16>(L.a7), *a8 = P.at<bf16>(L.a8);
    GB_TRY(conv_simt<bf16>(X0, Y0, Z0, 2, 16, P.at<bf16>(L.xin), W(0), a1, 1, nullptr, 0, 0, nullptr, s));
    GB_TRY(conv_tc<bf16>(X0, Y0, Z0, 16, 16, a1, W(1), k8, 48, 32, 1, nullptr, 0, 0, err, s));
    pool2_kernel<16><<<row_grid(X1, 2, Y1, Z1), 256, 0, s>>>(X1, Y1, Z1, k8, 48, 32, p1);
    GB_CUDA(cudaGetLastError());
    GB_TRY(conv_tc<bf16>(X1, Y1, Z1, 16, 32, p1, W(2), a3, 32, 0, 1, nullptr, 0, 0, err, s));
    GB_TRY(conv_tc<bf16>(X1, Y1, Z1, 32, 32, a3, W(3), k7, 96, 64, 1, nullptr, 0, 0, err, s));
    pool2_kernel<32><<<row_grid(X2, 4, Y2, Z2), 256, 0, s>>>(X2, Y2, Z2, k7, 96, 64, p2);
    GB_CUDA(cudaGetLastError());
    GB_TRY(conv_tc<bf16>(X2, Y2, Z2, 32, 64, p2, W(4), a5, 64, 0, 1, nullptr, 0, 0, err, s));
    GB_TRY(conv_tc<bf16>(X2, Y2, Z2, 64, 64, a5, W(5), a6, 64, 0, 1, nullptr, 0, 0, err, s));
    up2_kernel<64><<<row_grid(X1, 8, Y1, Z1), 256, 0, s>>>(X1, Y1, Z1, a6, k7, 96, 0);
    GB_CUDA(cudaGetLastError());
    GB_TRY(conv_tc<bf16>(X1, Y1, Z1, 96, 32, k7, W(6), a7, 32, 0, 1, nullptr, 0, 0, err, s));
    up2_kernel<32><<<row_grid(X0, 4, Y0, Z0), 256, 0, s>>>(X0, Y0, Z0, a7, k8, 48, 0);
    GB_CUDA(cudaGetLastError());
    GB_TRY(conv_tc<bf16>(X0, Y0, Z0, 48, 16, k8, W(7), a8, 16, 0, 1, nullptr, 0, 0, err, s));
    GB_TRY(conv_simt<float>(X0, Y0, Z0, 16, 1, a8, W(8), z, 0, nullptr, 0, 0, sc + S_SCALE, s, dsc));
    return GBPCG_OK;
}

// Gradients of every weight given gz = dL/dz, from the activations the last
// forward left in the workspace.
int nn_backward_ws(const float *gz, float *gw, void *ws, const NnLayout &L, cudaStream_t s) {
    NnPtrs P{static_cast<char *>(ws)};
    const int X0 = L.X[0], Y0 = L.Y[0], Z0 = L.Z[0], X1 = L.X[1], Y1 = L.Y[1], Z1 = L.Z[1], X2 = L.X[2], Y2 = L.Y[2],
              Z2 = L.Z[2];
    const bf16 *wflip = P.at<bf16>(L.wflip);
    auto WT = [&](int l) { return wflip + layer_offset(l); };
    auto G = [&](int l) { return gw + layer_offset(l); };
    double *sc = P.at<double>(L.scal);
    int *err = P.at<int>(L.err);
    float *part = P.at<float>(L.part);
    const bf16 *xin = P.at<bf16>(L.xin), *a1 = P.at<bf16>(L.a1), *k8 = P.at<bf16>(L.k8), *p1 = P.at<bf16>(L.p1),
               *a3 = P.at<bf16>(L.a3), *k7 = P.at<bf16>(L.k7), *p2 = P.at<bf16>(L.p2), *a5 = P.at<bf16>(L.a5),
               *a6 = P.at<bf16>(L.a6), *a7 = P.at<bf16>(L.a7), *a8 = P.at<bf16>(L.a8);
    bf16 *gout = P.at<bf16>(L.gout), *ga8 = P.at<bf16>(L.ga8), *ga7 = P.at<bf16>(L.ga7), *ga6 = P.at<bf16>(L.ga6),
         *ga5 = P.at<bf16>(L.ga5), *ge1b = P.at<bf16>(L.ge1b), *ga3 = P.at<bf16>(L.ga3), *ge0b = P.at<bf16>(L.ge0b),
         *ga1 = P.at<bf16>(L.ga1);
    float *gk8 = P.at<float>(L.gk8), *gk7 = P.at<float>(L.gk7), *t5 = P.at<float>(L.t5), *t3 = P.at<float>(L.t3);

    scale_to_bf16_kernel<<<blocks_for(L.V[0], 256), 256, 0, s>>>(L.V[0], gz, sc + S_SCALE, P.at<float>(L.dsc), gout);
    GB_CUDA(cudaGetLastError());
    // c9 (16 -> 1)
    GB_TRY(wgrad(X0, Y0, Z0, 16, 1, a8, gout, G(8), part, s, err));
    GB_TRY(conv_simt<bf16>(X0, Y0, Z0, 1, 16, gout, WT(8), ga8, 0, a8, 16, 0, nullptr, s));
    // c8 (48 -> 16) on k8 = [up(a7), e0]
    GB_TRY(wgrad(X0, Y0, Z0, 48, 16, k8, ga8, G(7), part, s, err));
    GB_TRY(conv_tc<float>(X0, Y0, Z0, 16, 48, ga8, WT(7), gk8, 48, 0, 0, nullptr, 0, 0, err, s));
    up2_adjoint_mask_kernel<32><<<row_grid(X1, 4, Y1, Z1), 256, 0, s>>>(X1, Y1, Z1, gk8, 48, 0, a7, ga7);
    GB_CUDA(cudaGetLastError());
    // c7 (96 -> 32) on k7 = [up(a6), e1]
    GB_TRY(wgrad(X1, Y1, Z1, 96, 32, k7, ga7, G(6), part, s, err));
    GB_TRY(conv_tc<float>(X1, Y1, Z1, 32, 96, ga7, WT(6), gk7, 96, 0, 0, nullptr, 0, 0, err, s));
    up2_adjoint_mask_kernel<64><<<row_grid(X2, 8, Y2, Z2), 256, 0, s>>>(X2, Y2, Z2, gk7, 96, 0, a6, ga6);
    GB_CUDA(cudaGetLastError());
    // c6 (64 -> 64), c5 (32 -> 64)
    GB_TRY(wgrad(X2, Y2, Z2, 64, 64, a5, ga6, G(5), part, s, err));
    GB_TRY(conv_tc<bf16>(X2, Y2, Z2, 64, 64, ga6, WT(5), ga5, 64, 0, 0, a5, 64, 0, err, s));
    GB_TRY(wgrad(X2, Y2, Z2, 32, 64, p2, ga5, G(4), part, s, err));
    GB_TRY(conv_tc<float>(X2, Y2, Z2, 64, 32, ga5, WT(4), t5, 32, 0, 0, nullptr, 0, 0, err, s));
    // e1: skip gradient (gk7 channels 64..95) + pooled-path gradient, ReLU mask
    pool_adjoint_skip_mask_kernel<32><<<row_grid(X1, 4, Y1, Z1), 256, 0, s>>>(X1, Y1, Z1, gk7, 96, 64, t5, k7, 96,
                                                                              64, ge1b);
    GB_CUDA(cudaGetLastError());
    // c4 (32 -> 32), c3 (16 -> 32)
    GB_TRY(wgrad(X1, Y1, Z1, 32, 32, a3, ge1b, G(3), part, s, err));
    GB_TRY(conv_tc<bf16>(X1, Y1, Z1, 32, 32, ge1b, WT(3), ga3, 32, 0, 0, a3, 32, 0, err, s));
    GB_TRY(wgrad(X1, Y1, Z1, 16, 32, p1, ga3, G(2), part, s, err));
    GB_TRY(conv_tc<float>(X1, Y1, Z1, 32, 16, ga3, WT(2), t3, 16, 0, 0, nullptr, 0, 0, err, s));
    // e0: skip gradient (gk8 channels 32..47) + pooled-path gradient, ReLU mask
    pool_adjoint_skip_mask_kernel<16><<<row_grid(X0, 2, Y0, Z0), 256, 0, s>>>(X0, Y0, Z0, gk8, 48, 32, t3, k8, 48,
                                                                              32, ge0b);
    GB_CUDA(cudaGetLastError());
    // c2 (16 -> 16), c1 (2 -> 16)
    GB_TRY(wgrad(X0, Y0, Z0, 16, 16, a1, ge0b, G(1), part, s, err));
    GB_TRY(conv_tc<bf16>(X0, Y0, Z0, 16, 16, ge0b, WT(1), ga1, 16, 0, 0, a1, 16, 0, err, s));
    GB_TRY(wgrad(X0, Y0, Z0, 2, 16, xin, ga1, G(0), part, s, err));
    return GBPCG_OK;
}

int nn_check(const gbpcg_grid *g, const void *ws, size_t ws_bytes, bool training, NnLayout *L) {
    GB_TRY(check_grid(g));
    if (!nn_shape_ok(g->nx, g->ny, g->nz))
        return fail_arg("learned preconditioner: grid sizes must be multiples of 4 whose levels tile into 128 voxels "
                        "(e.g. powers of two >= 32)");
    if (g->ny > 65535) return fail_arg("learned preconditioner: ny must be at most 65535 (one block row per y)");
    *L = nn_layout(g->nx, g->ny, g->nz, training);
    if (!ws || ws_bytes < L->total) return fail_arg("learned preconditioner: workspace too small");
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return fail_arg("workspace must be 256-byte aligned");
    return GBPCG_OK;
}

// scale-free A-norm loss and its gradient (loss_finish_kernel)
static int nn_loss_ws(const gbpcg_grid &g, const float *z, const float *e, float *gz, double *loss, void *ws,
                      const NnLayout &L, cudaStream_t s) {
    NnPtrs P{static_cast<char *>(ws)};
    double *sc = P.at<double>(L.scal);
    float *ae = P.at<float>(L.lae);
    const int64_t n = L.V[0];
    void *dws = P.base + L.dotws;
    const size_t dwb = gbpcg_dot_workspace_size();
    gbpcg_stream st = (gbpcg_stream)s;
    GB_TRY(gbpcg_stencil_apply(&g, GBPCG_F32, z, gz, st));
    GB_TRY(gbpcg_stencil_apply(&g, GBPCG_F32, e, ae, st));
    GB_TRY(gbpcg_dot(n, GBPCG_F32, z, ae, sc + S_LA, dws, dwb, st));
    GB_TRY(gbpcg_dot(n, GBPCG_F32, z, gz, sc + S_LC, dws, dwb, st));
    GB_TRY(gbpcg_dot(n, GBPCG_F32, e, ae, sc + S_LE, dws, dwb, st));
    loss_finish_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, sc + S_LA, gz, ae, loss ? loss : sc + S_LOSS);
    GB_CUDA(cudaGetLastError());
    return GBPCG_OK;
}

// entry points of the flexible-CG solver (fcg.cu)
size_t nn_layout_total(int X, int Y, int Z, bool training) { return nn_layout(X, Y, Z, training).total; }
size_t nn_layout_err_offset() { return nn_layout(128, 128, 128, false).err; }
bool nn_shape_ok_ext(int X, int Y, int Z) { return nn_shape_ok(X, Y, Z); }
int nn_prep_ext(const float *w, void *ws, const gbpcg_grid &g, cudaStream_t s) {
    const NnLayout L = nn_layout(g.nx, g.ny, g.nz, false);
    GB_TRY(nn_weight_prep(w, ws, L, s));
    return nn_diag_prep(g, ws, L, s);
}
int nn_forward_ext(const gbpcg_grid &g, const float *r, float *z, void *ws, cudaStream_t s) {
    return nn_forward_prepped(g, r, z, ws, nn_layout(g.nx, g.ny, g.nz, false), s, true);
}

}  // namespace gb

using namespace gb;

// ------------------------------------------------------------------ C ABI --

extern "C" int gbpcg_conv3_workspace_size(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, size_t *bytes) {
    clear_error();
    if (!bytes) return fail_arg("bytes is NULL");
    if (nx <= 0 || ny <= 0 || nz <= 0 || ci <= 0 || co <= 0) return fail_arg("sizes must be positive");
    size_t b = 256 + align_up((size_t)27 * ci * co * 2, 256);
    if (wgrad_ok(nx, ci, co) || wgrad_tc_ok(nx, ny, nz, ci, co)) b += wgrad_partial_bytes(nx, ny, nz, ci, co);
    *bytes = b;
    return GBPCG_OK;
}

static int conv_args(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *a, const void *b,
                     const void *c, const void *ws, size_t ws_bytes) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail_arg("grid sizes must be positive");
    if ((int64_t)nx * ny * nz > ((int64_t)1 << 34)) return fail_arg("grid too large");
    if (!a || !b || !c) return fail_arg("NULL array");
    if (!aligned16(a) || !aligned16(b) || !aligned16(c)) return fail_arg("arrays must be 16-byte aligned");
    size_t need = 0;
    int rc = gbpcg_conv3_workspace_size(nx, ny, nz, ci, co, &need);
    if (rc) return rc;
    if (!ws || ws_bytes < need) return fail_arg("workspace too small");
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return fail_arg("workspace must be 256-byte aligned");
    return GBPCG_OK;
}

extern "C" int gbpcg_conv3_forward(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *x,
                                   const void *w, float *y, int32_t relu, void *workspace, size_t workspace_bytes,
                                   gbpcg_stream stream) {
    NvtxRange range("gbpcg_conv3_forward");
    clear_error();
    GB_TRY(conv_args(nx, ny, nz, ci, co, x, w, y, workspace, workspace_bytes));
    cudaStream_t s = (cudaStream_t)stream;
    const bf16 *xi = static_cast<const bf16 *>(x), *wi = static_cast<const bf16 *>(w);
    int *err = static_cast<int *>(workspace);
    if (conv_tc_ok(nx, ny, nz, ci, co))
        return conv_tc<float>(nx, ny, nz, ci, co, xi, wi, y, co, 0, relu, nullptr, 0, 0, err, s);
    if (conv_simt_ok(ci, co)) return conv_simt<float>(nx, ny, nz, ci, co, xi, wi, y, relu, nullptr, 0, 0, nullptr, s);
    return fail_arg("unsupported convolution shape or channel counts");
}

__global__ void flip_one_kernel(int ci, int co, const bf16 *__restrict__ w, bf16 *__restrict__ wflip) {
    const int64_t n = (int64_t)27 * ci * co;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % ci), t = (int)((e / ci) % 27), o = (int)(e / (27 * ci));
        wflip[((int64_t)i * 27 + (26 - t)) * co + o] = w[e];
    }
}

extern "C" int gbpcg_conv3_backward_data(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *gy,
                                         const void *w, float *gx, void *workspace, size_t workspace_bytes,
                                         gbpcg_stream stream) {
    NvtxRange range("gbpcg_conv3_backward_data");
    clear_error();
    GB_TRY(conv_args(nx, ny, nz, ci, co, gy, w, gx, workspace, workspace_bytes));
    cudaStream_t s = (cudaStream_t)stream;
    const bool tc = conv_tc_ok(nx, ny, nz, co, ci), simt = conv_simt_ok(co, ci);
    if (!tc && !simt) return fail_arg("unsupported convolution shape or channel counts");
    int *err = static_cast<int *>(workspace);
    bf16 *wflip = reinterpret_cast<bf16 *>(static_cast<char *>(workspace) + 256);
    flip_one_kernel<<<blocks_for((int64_t)27 * ci * co, 256), 256, 0, s>>>(ci, co, static_cast<const bf16 *>(w), wflip);
    GB_CUDA(cudaGetLastError());
    const bf16 *g = static_cast<const bf16 *>(gy);
    if (tc) return conv_tc<float>(nx, ny, nz, co, ci, g, wflip, gx, ci, 0, 0, nullptr, 0, 0, err, s);
    return conv_simt<float>(nx, ny, nz, co, ci, g, wflip, gx, 0, nullptr, 0, 0, nullptr, s);
}

extern "C" int gbpcg_conv3_backward_weight(int32_t nx, int32_t ny, int32_t nz, int32_t ci, int32_t co, const void *x,
                                           const void *gy, float *gw, void *workspace, size_t workspace_bytes,
                                           gbpcg_stream stream) {
    NvtxRange range("gbpcg_conv3_backward_weight");
    clear_error();
    GB_TRY(conv_args(nx, ny, nz, ci, co, x, gy, gw, workspace, workspace_bytes));
    if (!wgrad_ok(nx, ci, co) && !wgrad_tc_ok(nx, ny, nz, ci, co))
        return fail_arg("weight gradient: unsupported width or channel count");
    if (ci % 8 && ci > 2) return fail_arg("weight gradient: ci must be 1, 2 or a multiple of 8");
    if (co % 8 && co != 1) return fail_arg("weight gradient: co must be 1 or a multiple of 8");
    float *part =
        reinterpret_cast<float *>(static_cast<char *>(workspace) + 256 + align_up((size_t)27 * ci * co * 2, 256));
    return wgrad(nx, ny, nz, ci, co, static_cast<const bf16 *>(x), static_cast<const bf16 *>(gy), gw, part,
                 (cudaStream_t)stream, static_cast<int *>(workspace));
}

extern "C" int gbpcg_nn_workspace_size(int32_t nx, int32_t ny, int32_t nz, int32_t training, size_t *bytes) {
    clear_error();
    if (!bytes) return fail_arg("bytes is NULL");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail_arg("grid sizes must be positive");
    if (!nn_shape_ok(nx, ny, nz))
        return fail_arg("learned preconditioner: grid sizes must be multiples of 4 whose levels tile into 128 voxels");
    *bytes = nn_layout(nx, ny, nz, training != 0).total;
    return GBPCG_OK;
}

extern "C" int gbpcg_nn_tensor_info(int32_t nx, int32_t ny, int32_t nz, int32_t training, int32_t index,
                                    size_t *offset, int32_t *dtype, int32_t *channels, int32_t *level) {
    clear_error();
    if (!offset || !dtype || !channels || !level) return fail_arg("NULL output pointer");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail_arg("grid sizes must be positive");
    if (!nn_shape_ok(nx, ny, nz))
        return fail_arg("learned preconditioner: grid sizes must be multiples of 4 whose levels tile into 128 voxels");
    const NnLayout L = nn_layout(nx, ny, nz, training != 0);
    struct Info { size_t off; int dt, ch, lv; bool train; };
    const Info tab[] = {
        {L.xin, GBPCG_BF16, 2, 0, false},   {L.a1, GBPCG_BF16, 16, 0, false},   {L.k8, GBPCG_BF16, 48, 0, false},
        {L.p1, GBPCG_BF16, 16, 1, false},   {L.a3, GBPCG_BF16, 32, 1, false},   {L.k7, GBPCG_BF16, 96, 1, false},
        {L.p2, GBPCG_BF16, 32, 2, false},   {L.a5, GBPCG_BF16, 64, 2, false},   {L.a6, GBPCG_BF16, 64, 2, false},
        {L.a7, GBPCG_BF16, 32, 1, false},   {L.a8, GBPCG_BF16, 16, 0, false},   {L.dsc, GBPCG_F32, 1, 0, false},
        {L.sr, GBPCG_F32, 1, 0, false},     {L.scal + S_SCALE * sizeof(double), GBPCG_F64, 1, -1, false},
        {L.gout, GBPCG_BF16, 1, 0, true},   {L.ga8, GBPCG_BF16, 16, 0, true},   {L.gk8, GBPCG_F32, 48, 0, true},
        {L.ga7, GBPCG_BF16, 32, 1, true},   {L.gk7, GBPCG_F32, 96, 1, true},    {L.ga6, GBPCG_BF16, 64, 2, true},
        {L.ga5, GBPCG_BF16, 64, 2, true},   {L.t5, GBPCG_F32, 32, 2, true},     {L.ge1b, GBPCG_BF16, 32, 1, true},
        {L.ga3, GBPCG_BF16, 32, 1, true},   {L.t3, GBPCG_F32, 16, 1, true},     {L.ge0b, GBPCG_BF16, 16, 0, true},
        {L.ga1, GBPCG_BF16, 16, 0, true},
    };
    constexpr int kCount = (int)(sizeof(tab) / sizeof(tab[0]));
    static_assert(kCount == GBPCG_NN_T_COUNT, "tensor table and enum disagree");
    if (index < 0 || index >= kCount) return fail_arg("tensor index out of range");
    if (tab[index].train && !training) return fail_arg("that tensor exists only in a training workspace");
    *offset = tab[index].off;
    *dtype = tab[index].dt;
    *channels = tab[index].ch;
    *level = tab[index].lv;
    return GBPCG_OK;
}

extern "C" int gbpcg_nn_forward(const gbpcg_grid *grid, const float *w, const float *r, float *z, void *workspace,
                                size_t workspace_bytes, gbpcg_stream stream) {
    NvtxRange range("gbpcg_nn_forward");
    clear_error();
    NnLayout L;
    GB_TRY(nn_check(grid, workspace, workspace_bytes, false, &L));
    if (!w || !r || !z) return fail_arg("NULL array");
    if (!aligned16(r) || !aligned16(z)) return fail_arg("r and z must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    GB_CUDA(cudaMemsetAsync(static_cast<char *>(workspace) + L.err, 0, sizeof(int), s));
    GB_TRY(nn_weight_prep(w, workspace, L, s));
    return nn_forward_prepped(*grid, r, z, workspace, L, s);
}

extern "C" int gbpcg_nn_backward(const gbpcg_grid *grid, const float *gz, float *gw, void *workspace,
                                 size_t workspace_bytes, gbpcg_stream stream) {
    NvtxRange range("gbpcg_nn_backward");
    clear_error();
    NnLayout L;
    GB_TRY(nn_check(grid, workspace, workspace_bytes, true, &L));
    if (!gz || !gw) return fail_arg("NULL array");
    return nn_backward_ws(gz, gw, workspace, L, (cudaStream_t)stream);
}

extern "C" int gbpcg_nn_adam(int64_t n, float *w, const float *g, float *m, float *v, int32_t step, double lr,
                             double beta1, double beta2, double eps, gbpcg_stream stream) {
    clear_error();
    if (n < 0 || step < 1) return fail_arg("n must be >= 0 and step >= 1");
    if (n == 0) return GBPCG_OK;
    if (!w || !g || !m || !v) return fail_arg("NULL array");
    const float bc1 = (float)(1.0 - pow(beta1, step)), bc2 = (float)(1.0 - pow(beta2, step));
    adam_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        n, w, g, m, v, (float)lr, (float)beta1, (float)(1.0 - beta1), (float)beta2, (float)(1.0 - beta2), (float)eps,
        bc1, bc2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "adam launch");
}

extern "C" int gbpcg_nn_loss(const gbpcg_grid *grid, const float *z, const float *e, float *gz, double *loss,
                             void *workspace, size_t workspace_bytes, gbpcg_stream stream) {
    clear_error();
    NnLayout L;
    GB_TRY(nn_check(grid, workspace, workspace_bytes, true, &L));
    if (!z || !e || !gz) return fail_arg("NULL array");
    return nn_loss_ws(*grid, z, e, gz, loss, workspace, L, (cudaStream_t)stream);
}

extern "C" int gbpcg_nn_train_step(const gbpcg_grid *grid, float *w, float *m, float *v, int32_t step, double lr,
                                   const float *r, const float *e, float *z, float *gz, float *gw, double *loss,
                                   void *workspace, size_t workspace_bytes, gbpcg_stream stream) {
    NvtxRange range("gbpcg_nn_train_step");
    clear_error();
    NnLayout L;
    GB_TRY(nn_check(grid, workspace, workspace_bytes, true, &L));
    if (!w || !m || !v || !r || !e || !z || !gz || !gw) return fail_arg("NULL array");
    if (!aligned16(r) || !aligned16(z) || !aligned16(e) || !aligned16(gz))
        return fail_arg("vectors must be 16-byte aligned");
    if (step < 1) return fail_arg("step must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    GB_CUDA(cudaMemsetAsync(static_cast<char *>(workspace) + L.err, 0, sizeof(int), s));
    GB_TRY(nn_weight_prep(w, workspace, L, s));
    GB_TRY(nn_forward_prepped(*grid, r, z, workspace, L, s));
    GB_TRY(nn_loss_ws(*grid, z, e, gz, loss, workspace, L, s));
    GB_TRY(nn_backward_ws(gz, gw, workspace, L, s));
    return gbpcg_nn_adam(kNumWeights, w, gw, m, v, step, lr, 0.9, 0.999, 1e-8, stream);
}

extern "C" int gbpcg_nn_status(void *workspace, gbpcg_stream stream) {
    clear_error();
    if (!workspace) return fail_arg("workspace is NULL");
    // the error word sits at the same offset in every learned-preconditioner workspace
    const size_t off = nn_layout_err_offset();
    int flag = 0;
    cudaStream_t s = (cudaStream_t)stream;
    GB_CUDA(cudaMemcpyAsync(&flag, static_cast<char *>(workspace) + off, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (!flag) return GBPCG_OK;
    GB_CUDA(cudaMemsetAsync(static_cast<char *>(workspace) + off, 0, sizeof(int), s));
    set_error("a bounded wait in a convolution kernel gave up");
    return GBPCG_TIMEOUT;
}
