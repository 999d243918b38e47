// C ABI: version, errors, tensor maps and the stencil apply (Sec. VI).
#include <mutex>
#include <string>

#include "launch.cuh"
#include "stencil64.cuh"

namespace gb {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
int fail_arg(const std::string &msg) {
    set_error("invalid argument: " + msg);
    return GBPCG_ERR_ARG;
}
int fail_cuda(cudaError_t e, const char *what) {
    set_error(std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") in " + what);
    return GBPCG_ERR_CUDA;
}

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

int make_map_3d(CUtensorMap *map, CUtensorMapDataType dt, size_t esize, const void *base, int nx, int ny,
                int nz, int bx, int by, int bz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is unavailable");
        return GBPCG_ERR_CUDA;
    }
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return GBPCG_ERR_CUDA;
    }
    return GBPCG_OK;
}

int make_map_nd(CUtensorMap *map, CUtensorMapDataType dt, const void *base, int rank, const uint64_t *dims,
                const uint64_t *strides, const uint32_t *box) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is unavailable");
        return GBPCG_ERR_CUDA;
    }
    if (rank < 1 || rank > 5) return fail_arg("tensor map rank");
    cuuint64_t d[5], st[4];
    cuuint32_t bx[5], estr[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        estr[i] = 1;
        if (i + 1 < rank) st[i] = strides[i];
    }
    CUresult r = fn(map, dt, rank, const_cast<void *>(base), d, st, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return GBPCG_ERR_CUDA;
    }
    return GBPCG_OK;
}

int check_grid(const gbpcg_grid *g) {
    if (!g) return fail_arg("grid is NULL");
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return fail_arg("grid sizes must be positive");
    if ((int64_t)g->nx * g->ny > (int64_t)1 << 31 || (int64_t)g->nx * g->ny * g->nz > (int64_t)1 << 40)
        return fail_arg("grid too large");
    if (g->k_block && (g->kbx <= 0 || g->kby <= 0 || g->kbz <= 0))
        return fail_arg("block edges must be positive with a coefficient array");
    return GBPCG_OK;
}

// FP64 operator: one thread per point (loads through the read-only cache).
template <bool BLOCK>
__global__ void stencil_f64_kernel(int nx, int ny, int nz, const double *__restrict__ p, double *__restrict__ q,
                                   double cx, double cy, double cz, const float *__restrict__ kb, int kbx, int kby,
                                   int kbz) {
    const int64_t n = (int64_t)nx * ny * nz;
    const Coef64 cf{cx, cy, cz, kb, kbx, kby, kbz};
    double w[6];
    face_weights64<false>(w, 0, 0, 0, nx, ny, nz, cf);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g % nx);
        const int64_t t = g / nx;
        const int j = (int)(t % ny), k = (int)(t / ny);
        if (BLOCK) face_weights64<true>(w, i, j, k, nx, ny, nz, cf);
        q[g] = apply64<BLOCK>(load_nbr64(p, g, i, j, k, nx, ny, nz), w);
    }
}

template <typename T, typename Op>
static int stencil_engine(const gbpcg_grid &gr, const void *p, void *q, const Op &op, cudaStream_t s) {
    const int nx = gr.nx, ny = gr.ny, nz = gr.nz;
    const int cfg = nx <= 32 ? CFG_32x16 : CFG_64x16;
    const bool tma = tma_ok(sizeof(T), nx, {p, q});
    PassArgs a{};
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.h0[0] = a.h0[1] = p;
    a.h1[0] = a.h1[1] = p;
    a.c0 = p;
    a.o0[0] = a.o0[1] = q;
    a.o1 = q;
    a.scale = 1.0f;
    PassMaps maps;
    memset(&maps, 0, sizeof(maps));
    int occ = tma ? GB_CFG_DISPATCH(cfg, T, K_STENCIL, true, Op, K::occupancy())
                  : GB_CFG_DISPATCH(cfg, T, K_STENCIL, false, Op, K::occupancy());
    size_t smem = tma ? GB_CFG_DISPATCH(cfg, T, K_STENCIL, true, Op, K::smem)
                      : GB_CFG_DISPATCH(cfg, T, K_STENCIL, false, Op, K::smem);
    PassGeom geo = make_geom(cfg, nx, ny, nz, occ, smem);
    a.tiles_x = geo.tiles_x;
    a.zchunk = geo.zchunk;
    if (tma) {
        int rc = make_pass_map<T>(&maps.h0[0], cfg, true, p, nx, ny, nz);
        if (rc) return rc;
        maps.h0[1] = maps.h0[0];
        maps.h1[0] = maps.h1[1] = maps.h0[0];
        maps.c0 = maps.h0[0];
    }
    cudaError_t e = tma ? GB_CFG_DISPATCH(cfg, T, K_STENCIL, true, Op, K::launch(maps, a, op, geo.grid(), s))
                        : GB_CFG_DISPATCH(cfg, T, K_STENCIL, false, Op, K::launch(maps, a, op, geo.grid(), s));
    if (e != cudaSuccess) return fail_cuda(e, "stencil launch");
    return GBPCG_OK;
}

template <typename T>
static int stencil_typed(const gbpcg_grid &g, const void *p, void *q, cudaStream_t s) {
    if (g.k_block) return stencil_engine<T>(g, p, q, make_op_block(g), s);
    return stencil_engine<T>(g, p, q, make_op_const(g.nx, g.ny, g.nz), s);
}

int launch_stencil_f64(const gbpcg_grid &g, const double *p, double *q, cudaStream_t s) {
    auto c = [](int n) { double h = 1.0 / (n + 1); return 1.0 / (h * h); };
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, (int64_t)device_sm_count() * 8);
    if (g.k_block)
        stencil_f64_kernel<true><<<(unsigned)blocks, threads, 0, s>>>(g.nx, g.ny, g.nz, p, q, c(g.nx), c(g.ny),
                                                                      c(g.nz), g.k_block, g.kbx, g.kby, g.kbz);
    else
        stencil_f64_kernel<false><<<(unsigned)blocks, threads, 0, s>>>(g.nx, g.ny, g.nz, p, q, c(g.nx), c(g.ny),
                                                                       c(g.nz), nullptr, 1, 1, 1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBPCG_OK : fail_cuda(e, "stencil_f64 launch");
}

}  // namespace gb

using namespace gb;

extern "C" {

const char *gbpcg_version(void) { return "gbpcg 0.1 sm_103a"; }

const char *gbpcg_last_error(void) { return g_last_error.c_str(); }

int gbpcg_stencil_apply(const gbpcg_grid *grid, int32_t dtype, const void *p, void *q, gbpcg_stream stream) {
    clear_error();
    if (int rc = check_grid(grid)) return rc;
    if (!p || !q) return fail_arg("p and q must be non-NULL device pointers");
    if (p == q) return fail_arg("p and q must not alias");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (dtype) {
        case GBPCG_F32: return stencil_typed<float>(*grid, p, q, s);
        case GBPCG_BF16: return stencil_typed<__nv_bfloat16>(*grid, p, q, s);
        case GBPCG_F16: return stencil_typed<__half>(*grid, p, q, s);
        case GBPCG_F64:
            return launch_stencil_f64(*grid, static_cast<const double *>(p), static_cast<double *>(q), s);
        default: return fail_arg("unknown dtype");
    }
}

}  // extern "C"

// ----------------------------------------------------------- self-test -----
// One CTA initialises an mbarrier for one arrival and waits on it with the
// library's bounded wait (at most `polls` polls); thread 0 arrives first only
// when `arrive` is set.  Without the arrival the wait gives up and the CTA
// writes GBPCG_TIMEOUT to *status instead of spinning on: the path every
// kernel of the library takes when a copy or an MMA never completes.

namespace gb {
__global__ void wait_selftest_kernel(int arrive, uint32_t polls, int *status, long long *cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        const long long t0 = clock64();
        const bool ok = mbar_wait_bounded(&bar, 0, polls);
        *cycles = clock64() - t0;
        *status = ok ? GBPCG_OK : GBPCG_TIMEOUT;
    }
}
}  // namespace gb

extern "C" int gbpcg_wait_selftest(int32_t arrive, uint32_t polls, void *scratch, double *ms, gbpcg_stream stream) {
    using namespace gb;
    clear_error();
    if (polls == 0 || polls > kWaitPolls) return fail_arg("polls must be 1 .. 2^18");
    if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 15u)) return fail_arg("scratch must be 16-byte aligned");
    int *d = static_cast<int *>(scratch);
    long long *cyc = reinterpret_cast<long long *>(static_cast<char *>(scratch) + 8);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    wait_selftest_kernel<<<1, 32, 0, s>>>(arrive, polls, d, cyc);
    cudaEventRecord(e1, s);
    int st = -1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (ms) *ms = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail_cuda(e, "wait self-test");
    if (st == GBPCG_TIMEOUT) set_error("bounded wait gave up (self-test)");
    return st;
}
