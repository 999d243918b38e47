// Jacobi-preconditioned CG (Sec. VII) as one CUDA graph per problem:
//
//   reset -> init (r0 = b - A x0 in FP64) ->
//   while (cond) { K_PASSA ; K_PASSB ; if (replace) { flush ; replace } } ->
//   finalize -> FP64 true residual
//
// The loop is a conditional WHILE node; the last CTA of each pass decides
// (from the grid-wide sums it has just finished) whether to continue and sets
// the condition from the device, so no scalar goes back to the host during
// the solve.  Per iteration the two data passes move 20 + 12 bytes per grid
// point in FP32 (see engine.cuh), against 44 for a three-kernel
// stencil / update-x-r / update-p split.
//
// Accuracy with FP32 vectors (reliable updates, van der Vorst & Ye, SIAM J.
// Sci. Comput. 22, 2000): the updates alpha p go into a correction vector d
// instead of x, so their rounding is relative to |d|, not |x|.  Whenever
// ||r|| has dropped by two decades since the last time, and when the recursive
// residual meets the tolerance, d is flushed into x and the recursive
// residual is replaced by b - A x evaluated in FP64; the iteration continues
// from the replaced residual (p is kept).  Convergence is therefore decided
// on a true residual.  x and b may be FP32 or FP64: they are only touched by
// the init, the replacements and the finalize, never by the per-iteration
// passes.  With FP32 x the rounding of x itself bounds the attainable true
// residual (about 1e-6 relative at 256^3); the solve stops with
// GBPCG_NOT_CONVERGED if confirmations stop making progress.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "launch.cuh"
#include "stencil64.cuh"

namespace gb {

// ------------------------------------------------------------- kernels --

static __global__ void reset_state_kernel(SolveState *st, double tol, int maxit) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        memset(st, 0, sizeof(SolveState));
        st->tol2 = tol * tol;
        st->maxit = maxit;
        st->status = GBPCG_NOT_CONVERGED;
    }
}

// Per-block face coefficients for OpTable: {k, k_x-, k_x+, k_y-},
// {k_y+, k_z-, k_z+, 0}; a face towards a neighbouring block carries the
// harmonic mean (the same FP32 expression as OpBlock), a face on the domain
// boundary the block's own k.
static __global__ void build_face_table(const float *__restrict__ kb, int nbx, int nby, int nbz, float4 *tab) {
    const int64_t nb = (int64_t)nbx * nby * nbz;
    auto hm = [](float a, float b) { return 2.0f * a * b / (a + b); };
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(t % nbx), by = (int)((t / nbx) % nby), bz = (int)(t / ((int64_t)nbx * nby));
        auto K = [&](int x, int y, int z) { return __ldg(kb + ((int64_t)z * nby + y) * nbx + x); };
        const float k = K(bx, by, bz);
        tab[2 * t] = make_float4(k, bx > 0 ? hm(k, K(bx - 1, by, bz)) : k, bx < nbx - 1 ? hm(k, K(bx + 1, by, bz)) : k,
                                 by > 0 ? hm(k, K(bx, by - 1, bz)) : k);
        tab[2 * t + 1] = make_float4(by < nby - 1 ? hm(k, K(bx, by + 1, bz)) : k, bz > 0 ? hm(k, K(bx, by, bz - 1)) : k,
                                     bz < nbz - 1 ? hm(k, K(bx, by, bz + 1)) : k, 0.0f);
    }
}

// FP64 face-weight table of the residual kernels (stencil64.cuh), one
// thread per block.
static __global__ void build_face_table64(const float *kb, int nbx, int nby, int nbz, Coef64 cf, double *tab) {
    const int64_t nb = (int64_t)nbx * nby * nbz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(t % nbx), by = (int)((t / nbx) % nby), bz = (int)(t / ((int64_t)nbx * nby));
        face_table64_block(tab + kTab64 * t, kb, bx, by, bz, nbx, nby, nbz, cf);
    }
}

// max |b| into st->rhs_bits (integer maxima of the bit patterns: no FP64 work).
template <typename X>
__global__ void __launch_bounds__(256) rhs_max_kernel(const X *__restrict__ b, int64_t n, SolveState *st) {
    using U = typename std::conditional<sizeof(X) == 8, unsigned long long, unsigned int>::type;
    constexpr U kAbs = (U)~((U)1 << (8 * sizeof(X) - 1));
    U m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        X v = __ldg(b + i);
        U u;
        memcpy(&u, &v, sizeof(U));
        u &= kAbs;
        m = u > m ? u : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const U t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) {
        X v;
        memcpy(&v, &m, sizeof(U));
        atomicMax(&st->rhs_bits, (unsigned long long)__double_as_longlong((double)v));
    }
}

enum ResMode { RES_INIT = 0, RES_REPLACE = 1, RES_TRUE = 2 };

struct Res64Args {
    int nx, ny, nz;
    const void *x, *b;
    void *z;   // storage type T of the kernel
    float *d;  // the correction vector is FP32 for every storage type
    double cx, cy, cz;
    const float *kb;
    int kbx, kby, kbz;
    const double *tab64;   // FP64 face weights per coefficient block (build_face_table64)
    const double *bscale;  // NULL, or a device scalar multiplying b (inner refinement solves)
    int rhs_auto;          // 1: b and x are scaled by rhs_scale(st->rhs_bits) (plain solves)
    int store_r;           // 1: store r itself into z (preconditioners other than Jacobi)
    SolveState *st;
    double *partials;
    cudaGraphConditionalHandle cond;
    int use_cond;
};

constexpr double kHuge = 1e300;

// Compensated FP32 sum (Kahan): the running error of each addition is fed
// back into the next, so the sum of a thread's terms is good to a few FP32
// roundings however many there are.
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// r = b - A x with FP64 differences and sums of differences (stencil64.cuh),
// one block per grid row (x fastest).
//   RES_INIT     z = D^-1 r, d = 0; FP64 sums r.r, r.z, b.b -> start state
//   RES_REPLACE  z = D^-1 r; sums r.r, r.z -> replacement decisions
//   RES_TRUE     sum r.r -> reported true residual (b.b is the start
//                state's).  Skipped when the solve ended on a replacement
//                that already evaluated this x (it left x unchanged).
// REPLACE and TRUE sum in compensated FP32 the values r 2^-e and z 2^-e,
// with 2^e the power of two just above rms(b), so the squares stay
// far from FP32 overflow and underflow; the products come back scaled by
// 2^(2e) exactly.  GB300's FP64 rate is the reason: these kernels keep its
// FP64 pipe busy (about 40 us per FP64 operation per point at 256^3,
// measured), and the FP64 operations of a replacement drop from 16 (stencil,
// b - A x, two FP64 dot products) to 11.
template <int MODE>
constexpr int res64_nv() { return MODE == RES_INIT ? 3 : MODE == RES_REPLACE ? 2 : 1; }

// One CTA's part of the residual sums over rows row0, row0 + rstep, ...
// below row1 (a row = nx consecutive points, row index j + ny k); the
// block sums land in part[] (valid in thread 0) and *unscale receives the
// factor that undoes the sums' power-of-two scaling.  CG: x was written
// earlier in the same launch (persistent kernels), read it through L2.
template <int MODE, typename X, typename Bt, bool BLOCK, typename T, bool CG = false>
__device__ __forceinline__ void res64_rows(const Res64Args &a, int row0, int row1, int rstep,
                                           double (&part)[res64_nv<MODE>()], double *unscale_out) {
    // a persistent launch (CG) reads scalars other SMs wrote during the launch
    typename std::conditional<CG, const volatile SolveState *, const SolveState *>::type st = a.st;
    const X *__restrict__ x = static_cast<const X *>(a.x);
    const Bt *__restrict__ b = static_cast<const Bt *>(a.b);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const Coef64 cf{a.cx, a.cy, a.cz, a.kb, a.kbx, a.kby, a.kbz};
    const bool bscaled = a.bscale != nullptr;
    const double bsc = bscaled ? *a.bscale : 1.0;
    // FP32 sums: scale 2^-e, unscale 2^(2e).  b arrives with max |b| within [2^-21, 2^20)
    // (rhs_scale, or the refinement's own scaling), so r itself is far from FP32's limits.
    float fs = 1.0f;
    double unscale = 1.0;
    if (MODE != RES_INIT) {
        const double bb = st->bb;
        if (bb > 0.0 && isfinite(bb)) {
            int e = 0;
            frexp(sqrt(bb / ((double)nx * ny * nz)), &e);
            e = max(-100, min(100, e));
            fs = __int_as_float((127 - e) << 23);
            unscale = ldexp(1.0, 2 * e);
        }
    }
    *unscale_out = unscale;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    KahanF k0, k1;
    double w[6];
    face_weights64<false>(w, 0, 0, 0, nx, ny, nz, cf);
    const float dg_const = diag64(w);
    // plain solves work on s b and s x: r = s (b - A x) (one more FP64 multiply, only when s != 1)
    const double s_rhs = a.rhs_auto ? rhs_scale(st->rhs_bits) : 1.0;
    auto sweep = [&](auto scaled_tag) {
        constexpr bool SC = decltype(scaled_tag)::value;
        for (int row = row0; row < row1; row += rstep) {
            const int j = row % ny, k = row / ny;
            const int64_t base = (int64_t)row * nx;
            for (int i = threadIdx.x; i < nx; i += 256) {
                const int64_t g = base + i;
                const Nbr64 u = load_nbr64<X, CG>(x, g, i, j, k, nx, ny, nz);
                if (BLOCK) face_weights64_tab(w, i, j, k, nx, ny, a.tab64, cf);
                const double ax = apply64<BLOCK>(u, w);
                const double bl = (double)__ldg(b + g);
                const double bv0 = bscaled ? bsc * bl : bl;
                const double r = SC ? s_rhs * (bv0 - ax) : bv0 - ax;
                const double bv = SC ? s_rhs * bv0 : bv0;
                const float rf = (float)r;
                const float rs = rf * fs;
                if (MODE == RES_TRUE) {
                    k0.add(rs * rs);
                } else {
                    const float dg = BLOCK ? diag64(w) : dg_const;
                    const T zt = from_f<T>(a.store_r ? rf : rf / dg);
                    static_cast<T *>(a.z)[g] = zt;
                    if (MODE == RES_INIT) {
                        s0 = fma(r, r, s0);
                        s1 = fma(r, (double)to_f(zt), s1);
                        s2 = fma(bv, bv, s2);
                        static_cast<float *>(a.d)[g] = 0.0f;
                    } else {
                        k0.add(rs * rs);
                        k1.add(rs * (to_f(zt) * fs));
                    }
                }
            }
        }
    };
    if (s_rhs != 1.0) sweep(std::true_type{});
    else sweep(std::false_type{});
    if (MODE != RES_INIT) {
        s0 = k0.value();
        s1 = k1.value();
    }
    constexpr int NV = res64_nv<MODE>();
    __shared__ double red[8][3];
    s0 = warp_sum(s0);
    if (NV > 1) s1 = warp_sum(s1);
    if (NV > 2) s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = s0;
        red[threadIdx.x >> 5][1] = s1;
        red[threadIdx.x >> 5][2] = s2;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v] = 0.0;
    if (threadIdx.x == 0)
        for (int wi = 0; wi < 8; ++wi)
#pragma unroll
            for (int v = 0; v < NV; ++v) part[v] += red[wi][v];
    __syncthreads();  // red is reused by the next call
}

// The last contribution's step after the residual sums (thread 0):
// RES_TRUE records the reported true residual, RES_INIT the start state,
// RES_REPLACE the replacement's decisions.
// SP: `SolveState *`, or `volatile SolveState *` in a persistent kernel.
template <int MODE, typename SP>
__device__ __forceinline__ void res64_finish(SP st, const double (&tot)[res64_nv<MODE>()], double unscale) {
    if (MODE == RES_TRUE) {
        st->rr_true = tot[0] * unscale;
        st->bb_true = st->bb;
        return;
    }
    if (MODE == RES_INIT) {
        const double rr = tot[0], rz = tot[1], bb = tot[2 < res64_nv<MODE>() ? 2 : 0];
        st->bb = bb; st->rr = rr; st->rz = rz; st->rr_rep = rr; st->rr_conf = kHuge;
        st->it = 0; st->pending = 0; st->zero_x = 0; st->replace = 0; st->true_known = 0;
        if (bb == 0.0) { st->zero_x = 1; st->done = 1; st->status = GBPCG_OK; }
        else if (rr <= st->tol2 * bb) { st->done = 1; st->status = GBPCG_OK; }
        else if (!isfinite(rz) || !(rz > 0.0)) { st->done = 1; st->status = GBPCG_BREAKDOWN; }
        else if (st->maxit <= 0) { st->done = 1; st->status = GBPCG_NOT_CONVERGED; }
        else { st->done = 0; st->status = GBPCG_NOT_CONVERGED; }
    } else {
        const double rrt = tot[0] * unscale, rzt = tot[1 < res64_nv<MODE>() ? 1 : 0] * unscale;
        const int kind = st->replace;  // 1: two decades of progress, 2: recursive residual met tol
        st->rr = rrt;
        st->rr_rep = rrt;
        st->replace = 0;
        st->pending = 0;
        st->n_replace += 1;
        if (rrt <= st->tol2 * st->bb) { st->done = 1; st->status = GBPCG_OK; }
        else if (!isfinite(rrt) || !isfinite(rzt) || !(rzt > 0.0)) { st->done = 1; st->status = GBPCG_BREAKDOWN; }
        else if (st->it >= st->maxit) { st->done = 1; st->status = GBPCG_NOT_CONVERGED; }
        else if (kind == 2 && rrt > 0.25 * st->rr_conf) { st->done = 1; st->status = GBPCG_NOT_CONVERGED; }
        else {
            if (kind == 2) st->rr_conf = rrt;
            st->beta = rzt / st->rz;
            st->rz = rzt;
        }
        // converged here: the flush emptied d and cleared the pending update,
        // so the finalize leaves x as this pass evaluated it
        if (st->done && st->status == GBPCG_OK) {
            st->true_known = 1;
            st->rr_true = rrt;
            st->bb_true = st->bb;
        }
    }
}

template <int MODE, typename X, typename Bt, bool BLOCK, typename T>
__global__ void __launch_bounds__(256) residual64_kernel(const Res64Args a) {
    SolveState *st = a.st;
    if (MODE == RES_REPLACE && (!st->replace || st->done)) return;
    if (MODE == RES_TRUE && st->true_known) return;
    constexpr int NV = res64_nv<MODE>();
    double part[NV], tot[NV], unscale = 1.0;
    res64_rows<MODE, X, Bt, BLOCK, T>(a, blockIdx.x, a.ny * a.nz, gridDim.x, part, &unscale);
    if (!grid_sum_last<NV, 256>(part, a.partials, &st->ticket[4 + MODE], tot) || threadIdx.x != 0) return;
    res64_finish<MODE>(st, tot, unscale);
    if (MODE == RES_TRUE) return;
    if (a.use_cond) cudaGraphSetConditional(a.cond, st->done ? 0u : 1u);
}

// x += (d + alpha_{it-1} p_{it-1}) / s: the increment is in the solver's scaled
// units (s = rhs_scale, or 1), x in the caller's.
template <typename X, typename T>
__device__ __forceinline__ void add_increment(X *x, float *d, const T *p, float a, int64_t n, double inv_s,
                                              bool clear_d) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    if (inv_s == 1.0) {
        for (int64_t i = tid; i < n; i += nth) {
            x[i] = x[i] + (X)fmaf(a, to_f(p[i]), d[i]);
            if (clear_d) d[i] = 0.0f;
        }
    } else {
        const X is = (X)inv_s;  // a power of two: exact in X unless X's exponent range ends first
        for (int64_t i = tid; i < n; i += nth) {
            x[i] = x[i] + (X)fmaf(a, to_f(p[i]), d[i]) * is;
            if (clear_d) d[i] = 0.0f;
        }
    }
}

// Residual replacement, step 1: x += d + alpha_{it-1} p_{it-1} (pending), d = 0.
template <typename X, typename T>
__global__ void flush_kernel(SolveState *st, X *x, float *d, const T *p0, const T *p1, int64_t n, int rhs_auto) {
    if (!st->replace || st->done) return;
    const T *p = ((st->it - 1) & 1) ? p1 : p0;
    const float a = st->pending ? (float)st->alpha : 0.0f;
    add_increment<X, T>(x, d, p, a, n, rhs_auto ? 1.0 / rhs_scale(st->rhs_bits) : 1.0, true);
}

// x += d + alpha_{it-1} p_{it-1} (the pending update, if any); x = 0 when b = 0.
template <typename X, typename T>
__global__ void finalize_kernel(const SolveState *st, X *x, const float *d, const T *p0, const T *p1, int64_t n,
                                int rhs_auto) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    if (st->zero_x) {
        for (int64_t i = tid; i < n; i += nth) x[i] = X(0);
        return;
    }
    const T *p = ((st->it - 1) & 1) ? p1 : p0;
    const float a = st->pending ? (float)st->alpha : 0.0f;
    add_increment<X, T>(x, const_cast<float *>(d), p, a, n, rhs_auto ? 1.0 / rhs_scale(st->rhs_bits) : 1.0, false);
}

// ----------------------------------------------------------- workspace --

struct WsLayout {
    size_t state, partials, z, p0, p1, d, tab, tab64, bstage, xstage, total;
};

static inline size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// Solver workspace: scalars, partial sums, z, p0, p1, d (storage type) and,
// for host I/O, staging copies of b and x.
static inline WsLayout ws_layout_n(size_t n, int storage, int io_dtype, bool host_io, int64_t nblocks) {
    const size_t vs = round256(n * dtype_size(storage));
    const size_t io = round256(n * dtype_size(io_dtype));
    WsLayout w;
    size_t off = 0;
    w.state = off; off += 256;
    w.partials = off; off += round256(sizeof(double) * 4 * kMaxPassBlocks);
    w.z = off; off += vs;
    w.p0 = off; off += vs;
    w.p1 = off; off += vs;
    w.d = off; off += round256(n * sizeof(float));  // d is FP32 for every storage type
    w.tab = off; off += round256((size_t)nblocks * 2 * sizeof(float4));  // face table (block coefficient)
    w.tab64 = off; off += round256((size_t)nblocks * kTab64 * sizeof(double));  // FP64 face weights
    w.bstage = w.xstage = 0;
    if (host_io) {
        w.bstage = off; off += io;
        w.xstage = off; off += io;
    }
    w.total = off;
    return w;
}

// ------------------------------------------------------------ the graph --

struct SolveKey {
    int dev, nx, ny, nz, kbx, kby, kbz, maxit, cfg_a, cfg_b, tma, io, storage;
    float op_scale;
    const void *kb, *b, *x, *ws, *bscale;
    double tol;
    bool operator==(const SolveKey &o) const { return memcmp(this, &o, sizeof(SolveKey)) == 0; }
};

// Instantiated solve graphs, cached by everything they bake in (pcg.cu).
cudaGraphExec_t graph_cache_find(const SolveKey &key);
cudaGraphExec_t graph_cache_put(const SolveKey &key, cudaGraph_t graph, cudaGraphExec_t exec);

// Everything one solve launches, set up once: geometry, tensor maps, kernel
// arguments.  The same launch functions serve graph capture and the
// event-timed profile mode.  X is the type of x and b (float or double), T
// the storage type of the iteration vectors z, p0, p1, d.
template <typename Op, bool TMA, typename X, typename T>
struct SolvePlan {
    gbpcg_grid g;
    Op op;
    int cfg_a, cfg_b;
    const X *b;
    X *x;
    SolveState *st;
    double *partials;
    T *z, *p0, *p1;
    float *d;
    char *tab;
    double *tab64;
    PassGeom ga, gb;
    PassMaps ma, mb;
    static constexpr int64_t kL2HintPoints = (int64_t)1 << 25;  // 33.5 M points (322^3)
    PassArgs aa, ab;
    Res64Args ra;
    double tol;
    int maxit;
    cudaGraphConditionalHandle cond_loop = 0, cond_rep = 0;
    int use_cond = 0;

    int init(const gbpcg_grid &grid, const Op &o, int ca, int cb, const X *bb, X *xx, char *ws, const WsLayout &L,
             double tl, int mi_, double op_scale, const double *bscale) {
        g = grid; op = o; cfg_a = ca; cfg_b = cb; b = bb; x = xx; tol = tl; maxit = mi_;
        st = reinterpret_cast<SolveState *>(ws + L.state);
        partials = reinterpret_cast<double *>(ws + L.partials);
        z = reinterpret_cast<T *>(ws + L.z);
        p0 = reinterpret_cast<T *>(ws + L.p0);
        p1 = reinterpret_cast<T *>(ws + L.p1);
        d = reinterpret_cast<float *>(ws + L.d);
        tab = ws + L.tab;
        tab64 = reinterpret_cast<double *>(ws + L.tab64);
        const int nx = g.nx, ny = g.ny, nz = g.nz;
        // kernel attributes and occupancy (never during a capture)
        int occ_a = GB_CFG_DISPATCH(cfg_a, T, K_PASSA, TMA, Op, K::occupancy());
        int occ_b = GB_CFG_DISPATCH(cfg_b, T, K_PASSB, TMA, Op, K::occupancy());
        ga = make_geom(cfg_a, nx, ny, nz, occ_a, GB_CFG_DISPATCH(cfg_a, T, K_PASSA, TMA, Op, K::smem));
        // pass B uses pass A's z chunks (it marches them downwards), so each
        // of its CTAs starts on the planes pass A's CTAs finished with
        gb = make_geom(cfg_b, nx, ny, nz, occ_b, GB_CFG_DISPATCH(cfg_b, T, K_PASSB, TMA, Op, K::smem));
        split_chunks(gb, ga.zchunk, nz, occ_b);
        memset(&ma, 0, sizeof(ma));
        memset(&mb, 0, sizeof(mb));
        if (TMA) {
            int rc = 0;
            rc |= make_pass_map<T>(&ma.h0[0], cfg_a, true, z, nx, ny, nz);
            ma.h0[1] = ma.h0[0];
            rc |= make_pass_map<T>(&ma.h1[0], cfg_a, true, p0, nx, ny, nz);
            rc |= make_pass_map<T>(&ma.h1[1], cfg_a, true, p1, nx, ny, nz);
            rc |= make_pass_map<float>(&ma.c0, cfg_a, false, d, nx, ny, nz);
            rc |= make_pass_map<T>(&mb.h0[0], cfg_b, true, p0, nx, ny, nz);
            rc |= make_pass_map<T>(&mb.h0[1], cfg_b, true, p1, nx, ny, nz);
            mb.h1[0] = mb.h1[1] = mb.h0[0];
            rc |= make_pass_map<T>(&mb.c0, cfg_b, false, z, nx, ny, nz);
            if (rc) return GBPCG_ERR_CUDA;
        }
        memset(&aa, 0, sizeof(aa));
        memset(&ab, 0, sizeof(ab));
        for (PassArgs *a : {&aa, &ab}) {
            a->nx = nx; a->ny = ny; a->nz = nz;
            a->st = st;
            a->partials = partials;
            a->scale = 1.0f;
        }
        aa.tiles_x = ga.tiles_x; aa.zchunk = ga.zchunk; aa.zparts = ga.zparts;
        // L2 hints in pass A where pass B's data (8 B per point) is within about twice the L2
        aa.l2hint = (int64_t)nx * ny * nz <= kL2HintPoints ? 1 : 0;
        aa.h0[0] = aa.h0[1] = z; aa.h1[0] = p0; aa.h1[1] = p1; aa.c0 = d; aa.o0[0] = p0; aa.o0[1] = p1; aa.o1 = d;
        ab.tiles_x = gb.tiles_x; ab.zchunk = gb.zchunk; ab.zparts = gb.zparts;
        ab.h0[0] = p0; ab.h0[1] = p1; ab.h1[0] = ab.h1[1] = p0; ab.c0 = z; ab.o0[0] = ab.o0[1] = z; ab.o1 = z;
        auto cc = [](int m) { double h = 1.0 / (m + 1); return 1.0 / (h * h); };
        memset(&ra, 0, sizeof(ra));
        ra.nx = nx; ra.ny = ny; ra.nz = nz;
        ra.x = x; ra.b = b; ra.z = z; ra.d = d;
        ra.cx = cc(nx) * op_scale; ra.cy = cc(ny) * op_scale; ra.cz = cc(nz) * op_scale;
        ra.bscale = bscale;
        ra.rhs_auto = bscale ? 0 : 1;  // inner refinement solves come scaled by the outer loop
        ra.kb = g.k_block;
        ra.kbx = g.k_block ? g.kbx : 1; ra.kby = g.k_block ? g.kby : 1; ra.kbz = g.k_block ? g.kbz : 1;
        ra.tab64 = tab64;
        ra.st = st;
        ra.partials = partials;
        return GBPCG_OK;
    }

    void set_cond(cudaGraphConditionalHandle c, cudaGraphConditionalHandle cr, int use) {
        cond_loop = c;
        cond_rep = cr;
        use_cond = use;
        aa.cond = ab.cond = c;
        aa.cond_replace = ab.cond_replace = cr;
        aa.use_cond = ab.use_cond = use;
        ra.cond = c;
        ra.use_cond = use;
    }

    unsigned stream_blocks(int64_t n, int per) const {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, (int64_t)device_sm_count() * 8));
    }
    unsigned row_blocks() const {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)g.ny * g.nz, (int64_t)device_sm_count() * 8));
    }

    template <int MODE>
    void launch_res64(cudaStream_t s) {
        if (g.k_block)
            residual64_kernel<MODE, X, X, true, T><<<row_blocks(), 256, 0, s>>>(ra);
        else
            residual64_kernel<MODE, X, X, false, T><<<row_blocks(), 256, 0, s>>>(ra);
    }

    cudaError_t launch_setup(cudaStream_t s) {
        reset_state_kernel<<<1, 32, 0, s>>>(st, tol, maxit);
        if (ra.rhs_auto) {
            const int64_t n = (int64_t)g.nx * g.ny * g.nz;
            rhs_max_kernel<X><<<stream_blocks(n, 2048), 256, 0, s>>>(b, n, st);
        }
        if (g.k_block) {
            const int nbx = (g.nx + g.kbx - 1) / g.kbx, nby = (g.ny + g.kby - 1) / g.kby, nbz = (g.nz + g.kbz - 1) / g.kbz;
            const int64_t nb = (int64_t)nbx * nby * nbz;
            const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 4096));
            build_face_table<<<blocks, 256, 0, s>>>(g.k_block, nbx, nby, nbz, reinterpret_cast<float4 *>(tab));
            const Coef64 cf{ra.cx, ra.cy, ra.cz, g.k_block, g.kbx, g.kby, g.kbz};
            build_face_table64<<<blocks, 256, 0, s>>>(g.k_block, nbx, nby, nbz, cf, tab64);
        }
        launch_res64<RES_INIT>(s);
        return cudaGetLastError();
    }
    cudaError_t launch_a(cudaStream_t s) {
        return GB_CFG_DISPATCH(cfg_a, T, K_PASSA, TMA, Op, K::launch(ma, aa, op, ga.grid(), s));
    }
    cudaError_t launch_b(cudaStream_t s) {
        return GB_CFG_DISPATCH(cfg_b, T, K_PASSB, TMA, Op, K::launch(mb, ab, op, gb.grid(), s));
    }

    // flush d into x, then r = b - A x in FP64 (both no-ops unless st->replace)
    cudaError_t launch_replace(cudaStream_t s) {
        const int64_t n = (int64_t)g.nx * g.ny * g.nz;
        flush_kernel<X, T><<<stream_blocks(n, 1024), 256, 0, s>>>(st, x, d, p0, p1, n, ra.rhs_auto);
        launch_res64<RES_REPLACE>(s);
        return cudaGetLastError();
    }

    cudaError_t launch_final(cudaStream_t s) {
        const int64_t n = (int64_t)g.nx * g.ny * g.nz;
        finalize_kernel<X, T><<<stream_blocks(n, 1024), 256, 0, s>>>(st, x, d, p0, p1, n, ra.rhs_auto);
        launch_res64<RES_TRUE>(s);
        return cudaGetLastError();
    }

    // reset -> init -> while(cond){A; B; if(replace){flush; replace}} -> finalize -> true residual
    // Records the whole solve onto cs, which is already capturing:
    // reset, init, a WHILE node whose body is {pass A, pass B, IF(replace)
    // {flush, replace}}, finalize, true residual.  The loop bodies are
    // captured from helper streams straight into the conditional nodes.
    cudaError_t capture_on(cudaStream_t cs) {
        cudaStream_t bs = nullptr, rs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (e) return e;
        e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
        if (e) {
            cudaStreamDestroy(bs);
            return e;
        }
        auto end_capture = [](cudaStream_t s) {
            cudaStreamCaptureStatus stt;
            if (cudaStreamIsCapturing(s, &stt) == cudaSuccess && stt != cudaStreamCaptureStatusNone) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(s, &tmp);
            }
        };
        // adds a conditional node after the current capture dependencies of s
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
        do {
            cudaStreamCaptureStatus cst;
            cudaGraph_t cap = nullptr;
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap, nullptr, nullptr, nullptr);
            if (e) break;
            cudaGraphConditionalHandle cond;
            e = cudaGraphConditionalHandleCreate(&cond, cap, 1, cudaGraphCondAssignDefault);
            if (e) break;
            set_cond(cond, 0, 1);
            e = launch_setup(cs);
            if (e) break;
            cudaGraph_t body = nullptr;
            e = add_cond(cs, cond, cudaGraphCondTypeWhile, &body);
            if (e) break;
            cudaGraphConditionalHandle rep;
            e = cudaGraphConditionalHandleCreate(&rep, body, 0, cudaGraphCondAssignDefault);
            if (e) break;
            set_cond(cond, rep, 1);
            e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e) break;
            e = launch_a(bs);
            if (e) break;
            e = launch_b(bs);
            if (e) break;
            cudaGraph_t rbody = nullptr;
            e = add_cond(bs, rep, cudaGraphCondTypeIf, &rbody);
            if (e) break;
            e = cudaStreamBeginCaptureToGraph(rs, rbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e) break;
            e = launch_replace(rs);
            if (e) break;
            cudaGraph_t tmp = nullptr;
            e = cudaStreamEndCapture(rs, &tmp);
            if (e) break;
            e = cudaStreamEndCapture(bs, &tmp);
            if (e) break;
            e = launch_final(cs);
        } while (0);
        if (e) {
            end_capture(rs);
            end_capture(bs);
        }
        cudaStreamDestroy(rs);
        cudaStreamDestroy(bs);
        return e;
    }

    // The solve as a graph of its own.
    int capture(cudaGraph_t *out_graph) {
        cudaStream_t cs = nullptr;
        GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (!e) e = capture_on(cs);
        cudaGraph_t graph = nullptr;
        cudaStreamCaptureStatus stt;
        if (cudaStreamIsCapturing(cs, &stt) == cudaSuccess && stt != cudaStreamCaptureStatusNone) {
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (!e) e = e2;
        }
        cudaStreamDestroy(cs);
        if (e) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail_cuda(e, "solve graph capture");
        }
        *out_graph = graph;
        return GBPCG_OK;
    }

    // Host-loop mode (the paper's FP32 variant reads the residual norm back
    // every iteration, Sec. VII): the same kernels launched one iteration at
    // a time, the host reading the device's stop flag after each iteration
    // before it launches the next.
    int run_host_loop(cudaStream_t s) {
        set_cond(0, 0, 0);
        GB_CUDA(launch_setup(s));
        int done = 0;
        GB_CUDA(cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < maxit && !done; ++i) {
            GB_CUDA(launch_a(s));
            GB_CUDA(launch_b(s));
            GB_CUDA(launch_replace(s));
            GB_CUDA(cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
        }
        GB_CUDA(launch_final(s));
        return GBPCG_OK;
    }

    // Profile mode: the same kernels launched one by one on `s`, each pass
    // launch bracketed by CUDA events; the loop polls the device flag every
    // kChunk iterations.  Only launches of real iterations are summed.
    int run_profiled(cudaStream_t s, double pass_ms[2], int launches[2], int ctas[2]) {
        constexpr int kChunk = 32;
        set_cond(0, 0, 0);
        GB_CUDA(launch_setup(s));
        cudaEvent_t ev[kChunk][4];
        for (int i = 0; i < kChunk; ++i)
            for (int j = 0; j < 4; ++j) GB_CUDA(cudaEventCreate(&ev[i][j]));
        pass_ms[0] = pass_ms[1] = 0.0;
        launches[0] = launches[1] = 0;
        ctas[0] = (int)ga.nblocks();
        ctas[1] = (int)gb.nblocks();
        int flags_h[2] = {0, 0};
        int rc = GBPCG_OK;
        for (int base = 0; base < std::max(maxit, 1); base += kChunk) {
            const int cnt = std::min(kChunk, std::max(maxit, 1) - base);
            for (int i = 0; i < cnt; ++i) {
                cudaEventRecord(ev[i][0], s);
                launch_a(s);
                cudaEventRecord(ev[i][1], s);
                cudaEventRecord(ev[i][2], s);
                launch_b(s);
                cudaEventRecord(ev[i][3], s);
                launch_replace(s);
            }
            cudaMemcpyAsync(&flags_h[0], &st->it, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(&flags_h[1], &st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e) { rc = fail_cuda(e, "profiled iteration"); break; }
            const int real = std::min(cnt, flags_h[0] - base);  // iterations completed in this chunk
            for (int i = 0; i < real; ++i) {
                float ta = 0.f, tb = 0.f;
                cudaEventElapsedTime(&ta, ev[i][0], ev[i][1]);
                cudaEventElapsedTime(&tb, ev[i][2], ev[i][3]);
                pass_ms[0] += ta;
                pass_ms[1] += tb;
                launches[0] += 1;
                launches[1] += 1;
            }
            if (flags_h[1]) break;
        }
        for (int i = 0; i < kChunk; ++i)
            for (int j = 0; j < 4; ++j) cudaEventDestroy(ev[i][j]);
        if (rc) return rc;
        GB_CUDA(launch_final(s));
        return GBPCG_OK;
    }
};

// One solve's arguments after validation (b and x already on the device).
struct SolveCall {
    const gbpcg_grid *g;
    int cfg_a, cfg_b;
    const void *b;
    void *x;
    char *ws;
    WsLayout L;
    double tol;
    int maxit;
    int io;                 // gbpcg_dtype of b and x
    float op_scale;         // the operator is op_scale * A (1 normally)
    const double *bscale;   // device scalar multiplying b, or NULL
};

template <typename Op, bool TMA, typename X, typename T>
static int plan_init(SolvePlan<Op, TMA, X, T> &plan, const SolveCall &c, const Op &op) {
    return plan.init(*c.g, op, c.cfg_a, c.cfg_b, static_cast<const X *>(c.b), static_cast<X *>(c.x), c.ws, c.L, c.tol,
                     c.maxit, c.op_scale, c.bscale);
}

// Dispatch over (operator, TMA path, io type); 16-bit storage serves only
// FP32 b and x (the inner solves of iterative refinement).
template <typename T, typename F>
static int dispatch_plan(const SolveCall &c, bool tma, F &&f) {
    const gbpcg_grid &g = *c.g;
    const bool f64 = c.io == GBPCG_F64;
    if (!std::is_same<T, float>::value && f64) return fail_arg("16-bit storage needs FP32 b and x");
    auto go = [&](auto op) -> int {
        if constexpr (std::is_same<T, float>::value) {
            if (tma) return f64 ? f(op, std::true_type{}, double{}) : f(op, std::true_type{}, float{});
            return f64 ? f(op, std::false_type{}, double{}) : f(op, std::false_type{}, float{});
        } else {
            if (tma) return f(op, std::true_type{}, float{});
            return f(op, std::false_type{}, float{});
        }
    };
    if (g.k_block) return go(make_op_table(g, c.op_scale, reinterpret_cast<const float4 *>(c.ws + c.L.tab)));
    return go(make_op_const(g.nx, g.ny, g.nz, c.op_scale));
}

// Graph mode: finds (or captures and instantiates) the solve's graph and
// launches it on s; no synchronisation.
template <typename T>
SolveKey make_key(const SolveCall &c, bool tma) {
    const gbpcg_grid &g = *c.g;
    int dev = 0;
    cudaGetDevice(&dev);
    SolveKey key;
    memset(&key, 0, sizeof(key));
    key.dev = dev; key.nx = g.nx; key.ny = g.ny; key.nz = g.nz;
    key.kb = g.k_block;
    if (g.k_block) { key.kbx = g.kbx; key.kby = g.kby; key.kbz = g.kbz; }
    key.maxit = c.maxit; key.cfg_a = c.cfg_a; key.cfg_b = c.cfg_b; key.tma = tma; key.io = c.io;
    key.storage = std::is_same<T, float>::value ? GBPCG_F32 : std::is_same<T, __half>::value ? GBPCG_F16 : GBPCG_BF16;
    key.op_scale = c.op_scale;
    key.b = c.b; key.x = c.x; key.ws = c.ws; key.bscale = c.bscale; key.tol = c.tol;
    return key;
}

template <typename T>
int solve_launch(const SolveCall &c, bool tma, cudaStream_t s) {
    const SolveKey key = make_key<T>(c, tma);
    cudaGraphExec_t exec = graph_cache_find(key);
    if (!exec) {
        cudaGraph_t graph = nullptr;
        int rc = dispatch_plan<T>(c, tma, [&](auto op, auto tm, auto xt) {
            SolvePlan<decltype(op), decltype(tm)::value, decltype(xt), T> plan;
            if (int r = plan_init(plan, c, op)) return r;
            return plan.capture(&graph);
        });
        if (rc) return rc;
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
        if (e) {
            cudaGraphDestroy(graph);
            return fail_cuda(e, "graph instantiate");
        }
        cudaGraphUpload(ex, s);
        exec = graph_cache_put(key, graph, ex);
    }
    GB_CUDA(cudaGraphLaunch(exec, s));
    return GBPCG_OK;
}

// Several solves as one graph: the capture forks from a root stream into one
// stream per problem, records each problem's whole solve (its own device
// loop and conditions) there and joins back, so one launch runs all of them
// concurrently.  calls[i].x / .b / .ws are the problems' own buffers.
template <typename T>
int batched_capture(const SolveCall *calls, const int *tma, int n, cudaGraph_t *out) {
    cudaStream_t root = nullptr;
    GB_CUDA(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
    std::vector<cudaStream_t> st(n, nullptr);
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && !e; ++i) e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
    for (int i = 0; i <= n && !e; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    bool capturing = false;
    int rc = GBPCG_OK;
    if (!e) e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
    if (!e) {
        capturing = true;
        e = cudaEventRecord(ev[n], root);
    }
    for (int i = 0; i < n && !e && !rc; ++i) {
        e = cudaStreamWaitEvent(st[i], ev[n], 0);
        if (e) break;
        rc = dispatch_plan<T>(calls[i], tma[i] != 0, [&](auto op, auto tm, auto xt) -> int {
            SolvePlan<decltype(op), decltype(tm)::value, decltype(xt), T> plan;
            if (int r = plan_init(plan, calls[i], op)) return r;
            cudaError_t e2 = plan.capture_on(st[i]);
            return e2 ? fail_cuda(e2, "batched capture") : GBPCG_OK;
        });
        if (!rc) e = cudaEventRecord(ev[i], st[i]);
        if (!rc && !e) e = cudaStreamWaitEvent(root, ev[i], 0);
    }
    cudaGraph_t graph = nullptr;
    if (capturing) {
        cudaError_t e2 = cudaStreamEndCapture(root, &graph);
        if (!e) e = e2;
    }
    for (auto s2 : st)
        if (s2) cudaStreamDestroy(s2);
    for (auto v : ev)
        if (v) cudaEventDestroy(v);
    cudaStreamDestroy(root);
    if (rc || e) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : fail_cuda(e, "batched graph capture");
    }
    *out = graph;
    return GBPCG_OK;
}

// Profile mode: the same kernels launched one by one, pass launches timed
// with CUDA events (synchronises s every few iterations).
template <typename T>
int solve_profiled(const SolveCall &c, bool tma, gbpcg_result *res, cudaStream_t s) {
    return dispatch_plan<T>(c, tma, [&](auto op, auto tm, auto xt) {
        SolvePlan<decltype(op), decltype(tm)::value, decltype(xt), T> plan;
        if (int r = plan_init(plan, c, op)) return r;
        return plan.run_profiled(s, res->pass_ms, res->pass_launches, res->pass_ctas);
    });
}

// Host-loop mode (GBPCG_FLAG_HOST_LOOP): one iteration per host round trip.
template <typename T>
int solve_host_loop(const SolveCall &c, bool tma, cudaStream_t s) {
    return dispatch_plan<T>(c, tma, [&](auto op, auto tm, auto xt) {
        SolvePlan<decltype(op), decltype(tm)::value, decltype(xt), T> plan;
        if (int r = plan_init(plan, c, op)) return r;
        return plan.run_host_loop(s);
    });
}

// Many constant-coefficient problems in one persistent kernel (batch.cu).
bool batch_persistent_ok(int nprob, const gbpcg_grid *grids);
size_t batch_persistent_bytes(int nprob, const gbpcg_grid *grids);
int batch_persistent_cfgs();
int batch_persistent_launch(int nprob, const gbpcg_grid *grids, const SolveCall *calls, char *region, int cfg,
                            double tol, int maxit, int io, cudaStream_t s);
int batch_persistent_header(const char *region, int *abort_rounds, cudaStream_t s);

// The split-kernel FP32 solver with host-side scalars (ablation.cu).
size_t split_workspace_size(const gbpcg_grid &g);
int split_solve(const gbpcg_grid &g, const float *b, float *x, const gbpcg_opts &o, gbpcg_result *res,
                cudaStream_t s);

extern template int batched_capture<float>(const SolveCall *, const int *, int, cudaGraph_t *);
extern template int solve_host_loop<float>(const SolveCall &, bool, cudaStream_t);
extern template int solve_launch<float>(const SolveCall &, bool, cudaStream_t);
extern template int solve_launch<__nv_bfloat16>(const SolveCall &, bool, cudaStream_t);
extern template int solve_launch<__half>(const SolveCall &, bool, cudaStream_t);
extern template int solve_profiled<float>(const SolveCall &, bool, gbpcg_result *, cudaStream_t);
extern template int solve_profiled<__nv_bfloat16>(const SolveCall &, bool, gbpcg_result *, cudaStream_t);
extern template int solve_profiled<__half>(const SolveCall &, bool, gbpcg_result *, cudaStream_t);

}  // namespace gb
