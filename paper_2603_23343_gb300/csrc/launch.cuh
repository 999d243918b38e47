// Host side of the z-marching engine: tile configurations, grid geometry,
// tensor-map set-up and the templated launcher.
#pragma once

#include <algorithm>
#include <cmath>

#include "engine.cuh"

namespace gb {

// Tile configurations the library is built with (x width, y height, stages).
enum TileCfg {
    CFG_64x16 = 0,
    CFG_32x16 = 1,
    CFG_128x8 = 2,
    CFG_64x8 = 3,
    CFG_64x8_S6 = 4,
    CFG_128x8_S6 = 5,
    CFG_256x4 = 6,  // whole rows, nx <= 256
    CFG_256x8 = 7,  // whole rows, nx <= 256
    CFG_128x8_S3 = 8,
    CFG_256x4_S3 = 9,  // whole rows, nx <= 256
    NUM_CFG = 10
};
struct CfgDims { int tx, ty, s; };
inline CfgDims cfg_dims(int c) {
    switch (c) {
        case CFG_64x16: return {64, 16, 4};
        case CFG_32x16: return {32, 16, 4};
        case CFG_128x8: return {128, 8, 4};
        case CFG_64x8: return {64, 8, 4};
        case CFG_64x8_S6: return {64, 8, 6};
        case CFG_128x8_S6: return {128, 8, 6};
        case CFG_256x4: return {256, 4, 4};
        case CFG_128x8_S3: return {128, 8, 3};
        case CFG_256x4_S3: return {256, 4, 3};
        default: return {256, 8, 4};
    }
}

// Whether a configuration can serve a grid of width nx.
inline bool cfg_fits(int c, int nx) { return cfg_dims(c).tx != 256 || nx <= 256; }

struct PassGeom {
    int cfg;
    int tiles_x, tiles_y, zchunk, zchunks;
    int zparts;  // CTAs per z chunk (grid y = chunks x zparts)
    size_t smem;
    dim3 grid() const { return dim3((unsigned)(tiles_x * tiles_y), (unsigned)zchunks, 1); }
    unsigned nblocks() const { return (unsigned)(tiles_x * tiles_y * zchunks); }
};

// Upper bound on the CTAs of one pass (sizes the partial-sum scratch).
constexpr unsigned kMaxPassBlocks = 4096;

int device_sm_count();

// Splits z into chunks: among chunk counts that keep chunks at least
// min_zchunk planes deep (and the grid within kMaxPassBlocks), picks the one
// whose CTAs fill the resident slots of the GPU most evenly (the fraction of
// the last wave that is occupied), preferring fewer, deeper chunks on ties.
inline PassGeom make_geom(int cfg, int nx, int ny, int nz, int ctas_per_sm, size_t smem,
                          int min_zchunk = 8) {
    CfgDims d = cfg_dims(cfg);
    PassGeom g;
    g.cfg = cfg;
    g.smem = smem;
    g.tiles_x = (nx + d.tx - 1) / d.tx;
    g.tiles_y = (ny + d.ty - 1) / d.ty;
    const long tiles = (long)g.tiles_x * g.tiles_y;
    const long slots = (long)device_sm_count() * std::max(1, ctas_per_sm);
    const int zmin = std::max(1, std::min(nz, min_zchunk));
    long best_zc = 1;
    double best = -1.0;
    for (long zc = 1; zc <= nz / zmin && tiles * zc <= (long)kMaxPassBlocks; ++zc) {
        const int zchunk = (int)((nz + zc - 1) / zc);
        const long chunks = (nz + zchunk - 1) / zchunk;  // chunks actually formed
        const double waves = (double)(tiles * chunks) / (double)slots;
        const double fill = waves / std::ceil(waves);
        if (fill > best + 0.02) {
            best = fill;
            best_zc = zc;
        }
    }
    int zchunk = (int)((nz + best_zc - 1) / best_zc);
    g.zchunk = std::max(zchunk, 1);
    g.zchunks = (nz + g.zchunk - 1) / g.zchunk;
    g.zparts = 1;
    return g;
}

// Gives a pass the z chunks of another pass (depth `zchunk`), each cut into
// the most parts (at most 4, each at least 8 planes deep) whose CTAs still
// fit the resident slots of the GPU in one wave; every part lies inside one
// chunk of the other pass.
inline void split_chunks(PassGeom &g, int zchunk, int nz, int ctas_per_sm) {
    const long tiles = (long)g.tiles_x * g.tiles_y;
    const long slots = std::min<long>((long)device_sm_count() * std::max(1, ctas_per_sm), kMaxPassBlocks);
    g.zchunk = std::max(zchunk, 1);
    const int chunks = (nz + g.zchunk - 1) / g.zchunk;
    g.zparts = 1;
    for (int parts = 4; parts >= 2; --parts)
        if ((g.zchunk + parts - 1) / parts >= 8 && tiles * chunks * parts <= slots) {
            g.zparts = parts;
            break;
        }
    g.zchunks = chunks * g.zparts;
}

// True when every array meets TMA's rules: 16-byte aligned base and a row
// pitch that is a multiple of 16 bytes.
inline bool tma_ok(size_t esize, int nx, std::initializer_list<const void *> ptrs) {
    if (((size_t)nx * esize) % 16 != 0) return false;
    for (const void *p : ptrs)
        if (p && (reinterpret_cast<uintptr_t>(p) & 15u)) return false;
    return true;
}

template <typename T, int TX, int TY, int S, int KIND, bool TMA, typename Op>
struct PassKernel {
    static constexpr size_t smem = zmarch_smem_bytes<T, TX, TY, S, KIND>();
    static constexpr int threads = TX / (16 / (int)sizeof(T)) * TY;
    static void *fn() { return reinterpret_cast<void *>(&zmarch_kernel<T, TX, TY, S, KIND, TMA, Op>); }
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(zmarch_kernel<T, TX, TY, S, KIND, TMA, Op>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    static int occupancy() {
        int n = 0;
        if (prepare() != cudaSuccess) return 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zmarch_kernel<T, TX, TY, S, KIND, TMA, Op>,
                                                          threads, smem) != cudaSuccess)
            return 1;
        return std::max(n, 1);
    }
    static cudaError_t launch(const PassMaps &maps, const PassArgs &a, const Op &op, dim3 grid,
                              cudaStream_t s) {
        zmarch_kernel<T, TX, TY, S, KIND, TMA, Op><<<grid, threads, smem, s>>>(maps, a, op);
        return cudaGetLastError();
    }
};

// Runtime dispatch over the tile configuration.
#define GB_CFG_DISPATCH(cfg, T, KIND, TMA, Op, CALL)                             \
    [&]() {                                                                    \
        switch (cfg) {                                                         \
            case CFG_64x16: { using K = PassKernel<T, 64, 16, 4, KIND, TMA, Op>; return CALL; } \
            case CFG_32x16: { using K = PassKernel<T, 32, 16, 4, KIND, TMA, Op>; return CALL; } \
            case CFG_128x8: { using K = PassKernel<T, 128, 8, 4, KIND, TMA, Op>; return CALL; } \
            case CFG_64x8: { using K = PassKernel<T, 64, 8, 4, KIND, TMA, Op>; return CALL; }   \
            case CFG_64x8_S6: { using K = PassKernel<T, 64, 8, 6, KIND, TMA, Op>; return CALL; } \
            case CFG_128x8_S6: { using K = PassKernel<T, 128, 8, 6, KIND, TMA, Op>; return CALL; } \
            case CFG_256x4: { using K = PassKernel<T, 256, 4, 4, KIND, TMA, Op>; return CALL; }  \
            case CFG_128x8_S3: { using K = PassKernel<T, 128, 8, 3, KIND, TMA, Op>; return CALL; } \
            case CFG_256x4_S3: { using K = PassKernel<T, 256, 4, 3, KIND, TMA, Op>; return CALL; } \
            default: { using K = PassKernel<T, 256, 8, 4, KIND, TMA, Op>; return CALL; }         \
        }                                                                      \
    }()

// Encodes the tensor map of one array for a configuration: halo boxes
// ((TX + 2 XH) x (TY + 2) x 1) or center boxes (TX x TY x 1).
template <typename T>
int make_pass_map(CUtensorMap *m, int cfg, bool halo, const void *base, int nx, int ny, int nz) {
    CfgDims d = cfg_dims(cfg);
    const int xh = d.tx == 256 ? 0 : 16 / (int)sizeof(T);
    if (halo) return make_map_3d(m, TypeTag<T>::tma, sizeof(T), base, nx, ny, nz, d.tx + 2 * xh, d.ty + 2, 1);
    return make_map_3d(m, TypeTag<T>::tma, sizeof(T), base, nx, ny, nz, d.tx, d.ty, 1);
}

inline OpConst make_op_const(int nx, int ny, int nz, float scale = 1.0f) {
    auto c = [](int n) { double h = 1.0 / (n + 1); return 1.0 / (h * h); };
    OpConst o;
    o.cx = (float)(c(nx) * scale);
    o.cy = (float)(c(ny) * scale);
    o.cz = (float)(c(nz) * scale);
    o.d = (float)(2.0 * ((double)o.cx + (double)o.cy + (double)o.cz));
    o.inv_d = (float)(1.0 / (2.0 * ((double)o.cx + (double)o.cy + (double)o.cz)));
    return o;
}

inline OpBlock make_op_block(const gbpcg_grid &g, float scale = 1.0f) {
    auto c = [](int n) { double h = 1.0 / (n + 1); return 1.0 / (h * h); };
    OpBlock o;
    o.inv_d = 0.0f;
    o.kb = g.k_block;
    o.nx = g.nx; o.ny = g.ny; o.nz = g.nz;
    o.kbx = g.kbx; o.kby = g.kby; o.kbz = g.kbz;
    o.nbx = (g.nx + g.kbx - 1) / g.kbx;
    o.nby = (g.ny + g.kby - 1) / g.kby;
    o.cx = (float)(c(g.nx) * scale); o.cy = (float)(c(g.ny) * scale); o.cz = (float)(c(g.nz) * scale);
    return o;
}

inline OpTable make_op_table(const gbpcg_grid &g, float scale, const float4 *tab) {
    auto c = [](int n) { double h = 1.0 / (n + 1); return 1.0 / (h * h); };
    OpTable o;
    o.inv_d = 0.0f;
    o.tab = tab;
    o.nx = g.nx; o.ny = g.ny; o.nz = g.nz;
    o.kbx = g.kbx; o.kby = g.kby; o.kbz = g.kbz;
    o.nbx = (g.nx + g.kbx - 1) / g.kbx;
    o.nby = (g.ny + g.kby - 1) / g.kby;
    o.grouped4 = g.kbx % 4 == 0;
    o.grouped8 = g.kbx % 8 == 0;
    o.cx = (float)(c(g.nx) * scale); o.cy = (float)(c(g.ny) * scale); o.cz = (float)(c(g.nz) * scale);
    return o;
}

inline int64_t block_count(const gbpcg_grid &g) {
    if (!g.k_block) return 0;
    return (int64_t)((g.nx + g.kbx - 1) / g.kbx) * ((g.ny + g.kby - 1) / g.kby) * ((g.nz + g.kbz - 1) / g.kbz);
}

// Validates a grid description; returns GBPCG_OK or GBPCG_ERR_ARG.
int check_grid(const gbpcg_grid *g);

}  // namespace gb
