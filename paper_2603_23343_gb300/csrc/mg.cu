// Geometric multigrid preconditioner and PCG with it (the paper names
// multigrid as future work in its conclusion; Sec. VII's iteration is kept).
//
// Hierarchy (aggregation): coarse cell I owns the 2 x 2 x 2 fine cells
// 2I + {0,1}^3, P copies a coarse value to its eight fine cells, and the
// coarse operator is the Galerkin product P^T A P.  For a seven-point
// operator in face-weight form, (A u)_c = D_c u_c - sum over interior faces
// w_f u_nb, that product is again one: a coarse face carries the sum of the
// four fine face weights across it and the coarse diagonal is the sum of the
// eight fine diagonals minus twice the twelve face weights inside the
// aggregate.  Level 0 is the solver's operator (weights computed per point,
// nothing stored); coarser levels store (w+x, w+y, w+z, D) per cell.
// Levels are added while every size is even and stays >= 4 (at most 8
// levels).
//
// V-cycle z = M r (level l, right-hand side f; the coarsest level takes
// kMgCoarseSweeps damped Jacobi sweeps from zero in one CTA):
//   u = omega D^-1 f;  f_{l+1} = P^T (f - A u)        (two kernels)
//   e = V-cycle(l + 1)
//   out = u' + omega D^-1 (f - A u'),  u' = u + sigma P e   (one kernel)
// Levels of at most kMgTailCells cells, the coarsest with them, run these
// steps inside one CTA (mg_tail_kernel) instead of a launch per step.
// Pre- and post-smoothing are adjoint, so M is symmetric (positive definite
// for omega < 1, 0 < sigma < 2).  omega = 0.9 and sigma = 1.5 took the
// fewest iterations in a sweep of the oracle at 32^3 and 64^3.
//
// PCG with M: pass A of the Jacobi solver (p_k = z_k + beta p_{k-1} on the
// fly, the deferred x update, p.Ap -> alpha), pass R (r -= alpha A p_k, r.r,
// the convergence test and the replacement trigger), the V-cycle, and r.z
// (-> beta); residual replacements store r = b - A x (FP64) and go through
// the V-cycle again.  One CUDA graph with a device-driven loop.
#include <algorithm>
#include <cstring>
#include <vector>

#include "solver.cuh"

namespace gb {

namespace {

constexpr int kMgMaxLevels = 8;
constexpr int kMgMinCoarse = 4;
constexpr float kMgOmega = 0.9f;
constexpr float kMgSigma = 1.5f;
constexpr int kMgCoarseSweeps = 24;
constexpr int64_t kMgMaxCoarsest = 32768;
constexpr int kMgThreads = 256;
constexpr int kMgCoarseThreads = 1024;
constexpr int64_t kMgTailCells = 4096;  // levels this small run inside the one-CTA tail kernel
constexpr int kMgSmemCells = 4096;      // a coarsest level this small sweeps in shared memory

struct MgLevel {
    int nx, ny, nz;
    float *f;         // right-hand side (level 0: the solver's r)
    float *u;         // pre-smoothed iterate (coarsest: its solution)
    float *w;         // post-smoothed result (level 0: z; coarsest: sweep scratch)
    const float4 *W;  // levels >= 1: (w+x, w+y, w+z, D) per cell
};

struct MgArgs {
    int L;
    MgLevel lv[kMgMaxLevels];
    int block;     // level 0: block coefficients (ob.weights) or constant (ob.cx, cy, cz)
    OpBlock ob;
    const float4 *tab;  // block coefficients: the solver's per-block face table (the same weights, no divisions)
    float rkbx, rkby, rkbz;  // 1 / the block edges (mg_div)
    const SolveState *st;  // inside a solve: every kernel stands down once st->done (NULL outside)
};

// n / d for 0 <= n < 2^22 and d >= 1, with rd = 1/d rounded to FP32:
// (n + 1/2) / d lies at least 1/(2d) from an integer, and the two FP32
// roundings (of rd and of the product) move it by at most
// 2^-23 (n + 1/2) / d < 1/(2d), so truncation gives the exact quotient.
__device__ __forceinline__ int mg_div(int n, float rd) { return (int)(((float)n + 0.5f) * rd); }

// Weights of point (i, j, k) of level l: w[0..5] = faces x-, x+, y-, y+, z-,
// z+ towards interior neighbours (0 across the boundary), and D.
// Which weights a kernel computes: W_ANY decides at run time (level and
// coefficient kind); the level kernels are compiled for one case each, so
// that a Poisson solve's kernels carry none of the table path's registers.
enum MgWeights { W_ANY = 0, W_CONST0 = 1, W_TAB0 = 2, W_STORED = 3 };

template <int WK = W_ANY>
__device__ __forceinline__ void mg_weights(const MgArgs &a, int l, int i, int j, int k, float w[6], float &D) {
    const MgLevel &L = a.lv[l];
    if (WK == W_CONST0 || WK == W_TAB0 || (WK == W_ANY && l == 0)) {
        if (WK == W_TAB0 || (WK == W_ANY && a.block && a.tab)) {
            // the face table holds the harmonic means (or the block's k on the domain boundary):
            // bitwise the weights of OpBlock::weights, without their divisions
            const OpBlock &o = a.ob;
            const int bx = mg_div(i, a.rkbx), by = mg_div(j, a.rkby), bz = mg_div(k, a.rkbz);
            const int ix = i - bx * o.kbx, iy = j - by * o.kby, iz = k - bz * o.kbz;
            const float4 *t = a.tab + 2 * (((int64_t)bz * o.nby + by) * o.nbx + bx);
            const float4 t0 = __ldg(t), t1 = __ldg(t + 1);
            const float kc = t0.x;
            w[0] = o.cx * (ix == 0 ? t0.y : kc);
            w[1] = o.cx * (ix == o.kbx - 1 ? t0.z : kc);
            w[2] = o.cy * (iy == 0 ? t0.w : kc);
            w[3] = o.cy * (iy == o.kby - 1 ? t1.x : kc);
            w[4] = o.cz * (iz == 0 ? t1.y : kc);
            w[5] = o.cz * (iz == o.kbz - 1 ? t1.z : kc);
        } else if (WK == W_ANY && a.block) {
            a.ob.weights(i, j, k, w);
        } else {
            w[0] = w[1] = a.ob.cx;
            w[2] = w[3] = a.ob.cy;
            w[4] = w[5] = a.ob.cz;
        }
        D = ((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]);
        // The level kernels (WK != W_ANY) load stencil inputs outside the grid as zero, so a
        // boundary face's weight multiplies zero there and need not be cleared; the run-time
        // form clears it (its callers index neighbours only where the weight is nonzero).
        if (WK == W_ANY) {
            if (i == 0) w[0] = 0.f;
            if (i == L.nx - 1) w[1] = 0.f;
            if (j == 0) w[2] = 0.f;
            if (j == L.ny - 1) w[3] = 0.f;
            if (k == 0) w[4] = 0.f;
            if (k == L.nz - 1) w[5] = 0.f;
        }
        return;
    }
    const int64_t c = ((int64_t)k * L.ny + j) * L.nx + i;
    const float4 W = __ldg(L.W + c);
    w[1] = W.x;
    w[3] = W.y;
    w[5] = W.z;
    D = W.w;
    w[0] = i > 0 ? __ldg(&L.W[c - 1].x) : 0.f;
    w[2] = j > 0 ? __ldg(&L.W[c - L.nx].y) : 0.f;
    w[4] = k > 0 ? __ldg(&L.W[c - (int64_t)L.nx * L.ny].z) : 0.f;
}

// sum over interior neighbours of w_f v(nb); v(flat index, i, j, k) of the neighbour
template <typename V>
__device__ __forceinline__ float mg_offdiag(const MgLevel &L, int i, int j, int k, int64_t c, const float w[6], V v) {
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    float s = 0.f;
    if (w[0] != 0.f) s = fmaf(w[0], v(c - 1, i - 1, j, k), s);
    if (w[1] != 0.f) s = fmaf(w[1], v(c + 1, i + 1, j, k), s);
    if (w[2] != 0.f) s = fmaf(w[2], v(c - sy, i, j - 1, k), s);
    if (w[3] != 0.f) s = fmaf(w[3], v(c + sy, i, j + 1, k), s);
    if (w[4] != 0.f) s = fmaf(w[4], v(c - sz, i, j, k - 1), s);
    if (w[5] != 0.f) s = fmaf(w[5], v(c + sz, i, j, k + 1), s);
    return s;
}

__device__ __forceinline__ bool mg_stand_down(const MgArgs &a) { return a.st && a.st->done; }

// Launch geometry of the level kernels: a block is bx threads along x times
// by rows along y and marches through zper planes; x, y and z come from the
// block and thread indices (no integer division per point), and there are
// about as many blocks as two waves of resident CTAs.
struct MgLaunch {
    dim3 grid, block;
    int zper;
};
inline MgLaunch mg_launch(int nx, int ny, int nz) {
    const int bx = std::min(kMgThreads, (nx + 31) / 32 * 32);
    const int by = std::max(1, std::min(kMgThreads / bx, ny));
    const int64_t gxy = (int64_t)((nx + bx - 1) / bx) * ((ny + by - 1) / by);
    const int64_t want = (int64_t)device_sm_count() * 16;
    const int gz = (int)std::max<int64_t>(1, std::min<int64_t>(nz, (want + gxy - 1) / gxy));
    const int zper = (nz + gz - 1) / gz;
    return MgLaunch{dim3((unsigned)((nx + bx - 1) / bx), (unsigned)((ny + by - 1) / by), (unsigned)((nz + zper - 1) / zper)),
                    dim3((unsigned)bx, (unsigned)by), zper};
}

// Four consecutive floats (16-byte aligned) <-> registers.
__device__ __forceinline__ void ld4f(const float *p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

// u = omega D^-1 f at level l; V consecutive points per thread (V = 4 needs nx % 4 == 0)
template <int V, int WK>
__global__ void __launch_bounds__(kMgThreads) mg_pre_kernel(const MgArgs a, int l, int zper) {
    if (mg_stand_down(a)) return;
    const MgLevel &L = a.lv[l];
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * V, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    const int k0 = blockIdx.z * zper, k1 = min(L.nz, k0 + zper);
    const float *__restrict__ f = L.f;
    float *__restrict__ u = L.u;
    for (int k = k0; k < k1; ++k) {
        const int64_t c = ((int64_t)k * L.ny + j) * L.nx + i0;
        float fv[V], out[V];
        if constexpr (V == 4) ld4f(f + c, fv);
        else fv[0] = f[c];
#pragma unroll
        for (int m = 0; m < V; ++m) {
            float w[6], D;
            mg_weights<WK>(a, l, i0 + m, j, k, w, D);
            out[m] = fv[m] * __fdividef(kMgOmega, D);
        }
        if constexpr (V == 4) *reinterpret_cast<float4 *>(u + c) = make_float4(out[0], out[1], out[2], out[3]);
        else u[c] = out[0];
    }
}

// The stencil input of V consecutive points of a row and of their neighbours:
// centre values c[V], the x neighbours left of point 0 and right of point
// V-1, the rows above / below and the planes before / after.  Values outside
// the grid read as 0 (their weights are 0 anyway).
template <int V>
struct Nbr {
    float c[V], xl, xr, ym[V], yp[V], zm[V], zp[V];
};
template <int V, typename GetV, typename Get1>
__device__ __forceinline__ void load_nbr(const MgLevel &L, int i0, int j, int k, GetV getv, Get1 get1, Nbr<V> &n) {
    getv(i0, j, k, n.c);
    n.xl = i0 > 0 ? get1(i0 - 1, j, k) : 0.f;
    n.xr = i0 + V < L.nx ? get1(i0 + V, j, k) : 0.f;
#pragma unroll
    for (int m = 0; m < V; ++m) n.ym[m] = n.yp[m] = n.zm[m] = n.zp[m] = 0.f;
    if (j > 0) getv(i0, j - 1, k, n.ym);
    if (j < L.ny - 1) getv(i0, j + 1, k, n.yp);
    if (k > 0) getv(i0, j, k - 1, n.zm);
    if (k < L.nz - 1) getv(i0, j, k + 1, n.zp);
}

// (A v)_m = D v_m - sum of the interior neighbours' w v for point m of a row segment
template <int V>
__device__ __forceinline__ float apply_m(const Nbr<V> &n, int m, const float w[6], float D) {
    const float xm = m == 0 ? n.xl : n.c[m - 1];
    const float xp = m == V - 1 ? n.xr : n.c[m + 1];
    float off = w[0] * xm;
    off = fmaf(w[1], xp, off);
    off = fmaf(w[2], n.ym[m], off);
    off = fmaf(w[3], n.yp[m], off);
    off = fmaf(w[4], n.zm[m], off);
    off = fmaf(w[5], n.zp[m], off);
    return fmaf(D, n.c[m], -off);
}

// f_{l+1} = P^T (f - A u).  V = 1: one thread per coarse cell; V = 2: two
// neighbouring coarse cells per thread, their four fine columns read as one
// 16-byte vector per fine row (needs nx % 4 == 0).
// FROM_F (level 0 with constant coefficients, where D is one number): the
// pre-smoothed u = (omega / D) f is formed from f at every use instead of
// being read, and the pre-smoothing kernel is not run (one multiply per
// value; it rounds once more than omega f / D).
template <int V, int WK, bool FROM_F = false>
__global__ void __launch_bounds__(kMgThreads) mg_restrict_kernel(const MgArgs a, int l, int zper) {
    if (mg_stand_down(a)) return;
    const MgLevel &L = a.lv[l], &C = a.lv[l + 1];
    const int I0 = (blockIdx.x * blockDim.x + threadIdx.x) * V, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I0 >= C.nx || J >= C.ny) return;
    const int K0 = blockIdx.z * zper, K1 = min(C.nz, K0 + zper);
    const float *__restrict__ u = FROM_F ? L.f : L.u;
    const float *__restrict__ f = L.f;
    float *__restrict__ fc = C.f;
    constexpr int FV = 2 * V;  // fine points per fine row
    const float wd = kMgOmega / (2.0f * ((a.ob.cx + a.ob.cy) + a.ob.cz));  // FROM_F: omega / D, D constant
    auto toU = [&](float x) { return FROM_F ? x * wd : x; };
    auto at = [&](int i, int j, int k) { return ((int64_t)k * L.ny + j) * L.nx + i; };
    auto getv = [&](int i, int j, int k, float *v) {
        const int64_t q = at(i, j, k);
        if constexpr (FV == 4) ld4f(u + q, v);
        else { v[0] = u[q]; v[1] = u[q + 1]; }
#pragma unroll
        for (int m = 0; m < FV; ++m) v[m] = toU(v[m]);
    };
    auto get1 = [&](int i, int j, int k) { return toU(u[at(i, j, k)]); };
    for (int K = K0; K < K1; ++K) {
        float sum[V];
#pragma unroll
        for (int m = 0; m < V; ++m) sum[m] = 0.f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const int i0 = 2 * I0, j = 2 * J + dy, k = 2 * K + dz;
                const int64_t c0 = ((int64_t)k * L.ny + j) * L.nx + i0;
                Nbr<FV> n;
                load_nbr<FV>(L, i0, j, k, getv, get1, n);
                float fv[FV];
                if constexpr (FV == 4) ld4f(f + c0, fv);
                else { fv[0] = f[c0]; fv[1] = f[c0 + 1]; }
#pragma unroll
                for (int m = 0; m < FV; ++m) {
                    float w[6], D;
                    mg_weights<WK>(a, l, i0 + m, j, k, w, D);
                    sum[m >> 1] += fv[m] - apply_m<FV>(n, m, w, D);
                }
            }
        const int64_t cc = ((int64_t)K * C.ny + J) * C.nx + I0;
        if constexpr (V == 2) *reinterpret_cast<float2 *>(fc + cc) = make_float2(sum[0], sum[1]);
        else fc[cc] = sum[0];
    }
}

// out = u' + omega D^-1 (f - A u'), u' = u + sigma P e with e the level-(l+1)
// result, formed at every stencil input; V consecutive points per thread.
template <int V, int WK, bool FROM_F = false>
__global__ void __launch_bounds__(kMgThreads)
    mg_post_kernel(const MgArgs a, int l, const float *__restrict__ e, int zper) {
    if (mg_stand_down(a)) return;
    const MgLevel &L = a.lv[l], &C = a.lv[l + 1];
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * V, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    const int k0 = blockIdx.z * zper, k1 = min(L.nz, k0 + zper);
    const float *__restrict__ u = FROM_F ? L.f : L.u;  // FROM_F: u = omega f / D (see mg_restrict_kernel)
    const float wd = kMgOmega / (2.0f * ((a.ob.cx + a.ob.cy) + a.ob.cz));
    const float wd_const = kMgOmega / (((a.ob.cx + a.ob.cx) + (a.ob.cy + a.ob.cy)) + (a.ob.cz + a.ob.cz));
    auto toU = [&](float x) { return FROM_F ? x * wd : x; };
    const float *__restrict__ f = L.f;
    float *__restrict__ out = L.w;
    for (int k = k0; k < k1; ++k) {
        const int64_t c0 = ((int64_t)k * L.ny + j) * L.nx + i0;
        // u' = u + sigma e[parent] at fine points (i, j, k) (V of them from i, i a multiple of V)
        auto fine = [&](int i, int jj, int kk) { return ((int64_t)kk * L.ny + jj) * L.nx + i; };
        auto parent = [&](int i, int jj, int kk) {
            return ((int64_t)(kk >> 1) * C.ny + (jj >> 1)) * C.nx + (i >> 1);
        };
        auto getv = [&](int i, int jj, int kk, float *v) {
            const int64_t q = fine(i, jj, kk), pc = parent(i, jj, kk);
            if constexpr (V == 4) {
                float uv[4];
                ld4f(u + q, uv);
                const float2 ep = __ldg(reinterpret_cast<const float2 *>(e + pc));
                v[0] = fmaf(kMgSigma, ep.x, toU(uv[0]));
                v[1] = fmaf(kMgSigma, ep.x, toU(uv[1]));
                v[2] = fmaf(kMgSigma, ep.y, toU(uv[2]));
                v[3] = fmaf(kMgSigma, ep.y, toU(uv[3]));
            } else {
                v[0] = fmaf(kMgSigma, __ldg(e + pc), toU(u[q]));
            }
        };
        auto get1 = [&](int i, int jj, int kk) {
            return fmaf(kMgSigma, __ldg(e + parent(i, jj, kk)), toU(u[fine(i, jj, kk)]));
        };
        Nbr<V> n;
        load_nbr<V>(L, i0, j, k, getv, get1, n);
        float fv[V], res[V];
        if constexpr (V == 4) ld4f(f + c0, fv);
        else fv[0] = f[c0];
#pragma unroll
        for (int m = 0; m < V; ++m) {
            float w[6], D;
            mg_weights<WK>(a, l, i0 + m, j, k, w, D);
            // omega / D: one number for constant coefficients (hoisted), else the fast division
            const float od = WK == W_CONST0 ? wd_const : __fdividef(kMgOmega, D);
            res[m] = fmaf(od, fv[m] - apply_m<V>(n, m, w, D), n.c[m]);
        }
        if constexpr (V == 4) *reinterpret_cast<float4 *>(out + c0) = make_float4(res[0], res[1], res[2], res[3]);
        else out[c0] = res[0];
    }
}

// coarsest level: kMgCoarseSweeps damped Jacobi sweeps from zero by one CTA;
// the result lands in lv[l].u (sweeps alternate between u and w)
__device__ __forceinline__ void mg_coarse_sweeps(const MgArgs &a, int l) {
    const MgLevel &L = a.lv[l];
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    float *src = L.u, *dst = L.w;
    // the final sweep must land in u: start in w when the sweep count is even
    if (kMgCoarseSweeps % 2 == 0) {
        src = L.w;
        dst = L.u;
    }
    for (int64_t c = threadIdx.x; c < n; c += kMgCoarseThreads) {
        const int i = (int)(c % L.nx);
        const int64_t t = c / L.nx;
        const int j = (int)(t % L.ny), k = (int)(t / L.ny);
        float w[6], D;
        mg_weights(a, l, i, j, k, w, D);
        src[c] = kMgOmega * L.f[c] / D;
    }
    __syncthreads();
    for (int sweep = 1; sweep < kMgCoarseSweeps; ++sweep) {
        for (int64_t c = threadIdx.x; c < n; c += kMgCoarseThreads) {
            const int i = (int)(c % L.nx);
            const int64_t t = c / L.nx;
            const int j = (int)(t % L.ny), k = (int)(t / L.ny);
            float w[6], D;
            mg_weights(a, l, i, j, k, w, D);
            const float off = mg_offdiag(L, i, j, k, c, w, [&](int64_t q, int, int, int) { return src[q]; });
            dst[c] = fmaf(kMgOmega / D, L.f[c] - fmaf(D, src[c], -off), src[c]);
        }
        __syncthreads();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
}

// (i, j, k) of flat cell c of a level (32-bit: the tail's levels are small)
__device__ __forceinline__ void mg_cell(const MgLevel &L, int c, int &i, int &j, int &k) {
    const int t = c / L.nx;
    i = c - t * L.nx;
    k = t / L.ny;
    j = t - k * L.ny;
}

// The coarsest level's sweeps with src / dst in shared memory (n <= kMgSmemCells):
// the same arithmetic as mg_coarse_sweeps; the result is written to lv[l].u
__device__ __forceinline__ void mg_coarse_sweeps_smem(const MgArgs &a, int l, float *sa, float *sb) {
    const MgLevel &L = a.lv[l];
    const int n = L.nx * L.ny * L.nz;
    for (int c = threadIdx.x; c < n; c += kMgCoarseThreads) {
        int i, j, k;
        mg_cell(L, c, i, j, k);
        float w[6], D;
        mg_weights(a, l, i, j, k, w, D);
        sa[c] = kMgOmega * L.f[c] / D;
    }
    __syncthreads();
    float *src = sa, *dst = sb;
    for (int sweep = 1; sweep < kMgCoarseSweeps; ++sweep) {
        for (int c = threadIdx.x; c < n; c += kMgCoarseThreads) {
            int i, j, k;
            mg_cell(L, c, i, j, k);
            float w[6], D;
            mg_weights(a, l, i, j, k, w, D);
            const float off = mg_offdiag(L, i, j, k, c, w, [&](int64_t q, int, int, int) { return src[q]; });
            dst[c] = fmaf(kMgOmega / D, L.f[c] - fmaf(D, src[c], -off), src[c]);
        }
        __syncthreads();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    for (int c = threadIdx.x; c < n; c += kMgCoarseThreads) L.u[c] = src[c];
    __syncthreads();
}

// The small levels l0 .. L-1 of the V-cycle in one CTA (every level but
// possibly the coarsest holds at most kMgTailCells cells; the coarsest at most
// kMgMaxCoarsest, in 32-bit range): pre-smoothing and
// restriction down to the coarsest level, its sweeps, post-smoothing back up
// to l0 (the same steps as the level kernels, with a CTA barrier between
// them instead of a kernel launch: on levels of a few thousand cells the
// launches cost more than the work).  Level l0's result lands in lv[l0].w,
// or in lv[l0].u when l0 is the coarsest level; a one-level hierarchy copies
// it into lv[0].w, the V-cycle's output.
__global__ void __launch_bounds__(kMgCoarseThreads) mg_tail_kernel(const MgArgs a, int l0) {
    if (mg_stand_down(a)) return;
    const int lc = a.L - 1;
    for (int l = l0; l < lc; ++l) {
        const MgLevel &L = a.lv[l], &C = a.lv[l + 1];
        const int n = L.nx * L.ny * L.nz, nc = C.nx * C.ny * C.nz;
        for (int c = threadIdx.x; c < n; c += kMgCoarseThreads) {
            int i, j, k;
            mg_cell(L, c, i, j, k);
            float w[6], D;
            mg_weights(a, l, i, j, k, w, D);
            L.u[c] = kMgOmega * L.f[c] / D;
        }
        __syncthreads();
        for (int cc = threadIdx.x; cc < nc; cc += kMgCoarseThreads) {
            int I, J, K;
            mg_cell(C, cc, I, J, K);
            float sum = 0.f;
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
                        const int c = (k * L.ny + j) * L.nx + i;
                        float w[6], D;
                        mg_weights(a, l, i, j, k, w, D);
                        const float off = mg_offdiag(L, i, j, k, c, w, [&](int64_t q, int, int, int) { return L.u[q]; });
                        sum += L.f[c] - fmaf(D, L.u[c], -off);
                    }
            C.f[cc] = sum;
        }
        __syncthreads();
    }
    __shared__ float s_sweep[2][kMgSmemCells];
    if ((int64_t)a.lv[lc].nx * a.lv[lc].ny * a.lv[lc].nz <= kMgSmemCells)
        mg_coarse_sweeps_smem(a, lc, s_sweep[0], s_sweep[1]);
    else
        mg_coarse_sweeps(a, lc);
    for (int l = lc - 1; l >= l0; --l) {
        const MgLevel &L = a.lv[l], &C = a.lv[l + 1];
        const float *e = (l + 1 == lc) ? C.u : C.w;
        const int n = L.nx * L.ny * L.nz;
        // u' = u + sigma P e at a fine cell
        auto up = [&](int64_t q, int i, int j, int k) {
            return fmaf(kMgSigma, e[((int64_t)(k >> 1) * C.ny + (j >> 1)) * C.nx + (i >> 1)], L.u[q]);
        };
        for (int c = threadIdx.x; c < n; c += kMgCoarseThreads) {
            int i, j, k;
            mg_cell(L, c, i, j, k);
            float w[6], D;
            mg_weights(a, l, i, j, k, w, D);
            const float uc = up(c, i, j, k);
            const float off = mg_offdiag(L, i, j, k, c, w, up);
            L.w[c] = fmaf(kMgOmega / D, L.f[c] - fmaf(D, uc, -off), uc);
        }
        __syncthreads();
    }
    if (lc == 0) {
        const MgLevel &L = a.lv[0];
        const int n = L.nx * L.ny * L.nz;
        for (int c = threadIdx.x; c < n; c += kMgCoarseThreads) L.w[c] = L.u[c];
    }
}

// Galerkin coarsening of level l into level l + 1 (one thread per coarse cell)
__global__ void __launch_bounds__(kMgThreads) mg_galerkin_kernel(const MgArgs a, int l, float4 *Wc, int zper) {
    const MgLevel &C = a.lv[l + 1];
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= C.nx || J >= C.ny) return;
    const int K0 = blockIdx.z * zper, K1 = min(C.nz, K0 + zper);
    for (int K = K0; K < K1; ++K) {
        float sx = 0.f, sy = 0.f, sz = 0.f, sD = 0.f, inner = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    float w[6], D;
                    mg_weights(a, l, 2 * I + dx, 2 * J + dy, 2 * K + dz, w, D);
                    sD += D;
                    if (dx == 1) sx += w[1]; else inner += w[1];
                    if (dy == 1) sy += w[3]; else inner += w[3];
                    if (dz == 1) sz += w[5]; else inner += w[5];
                }
        Wc[((int64_t)K * C.ny + J) * C.nx + I] = make_float4(sx, sy, sz, sD - 2.0f * inner);
    }
}

// r.z; last CTA: beta (the first time, only r.z), breakdown, the loop condition
__global__ void __launch_bounds__(kMgThreads)
    mg_rz_kernel(int64_t n, const float *__restrict__ r, const float *__restrict__ z, SolveState *st, double *partials,
                 int init, cudaGraphConditionalHandle cond, int use_cond) {
    if (st->done) return;
    float acc[1] = {0.f};
    for (int64_t i = (int64_t)blockIdx.x * kMgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kMgThreads)
        acc[0] = fmaf(r[i], z[i], acc[0]);
    double part[1], tot[1];
    block_sum<1, kMgThreads>(acc, part);
    if (!grid_sum_last<1, kMgThreads>(part, partials, &st->ticket[1], tot) || threadIdx.x != 0) return;
    const double rz = tot[0];
    if (!isfinite(rz) || !(rz > 0.0)) {
        st->done = 1;
        st->status = GBPCG_BREAKDOWN;
    } else {
        if (!init) st->beta = rz / st->rzm;
        st->rz = rz;
        st->rzm = rz;
    }
    if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// ---------------------------------------------------------- host side --

struct MgGeom {
    int L;
    int nx[kMgMaxLevels], ny[kMgMaxLevels], nz[kMgMaxLevels];
};

MgGeom mg_geom(const gbpcg_grid &g) {
    MgGeom m;
    m.L = 1;
    m.nx[0] = g.nx; m.ny[0] = g.ny; m.nz[0] = g.nz;
    while (m.L < kMgMaxLevels) {
        const int l = m.L - 1;
        const int a = m.nx[l], b = m.ny[l], c = m.nz[l];
        if (a % 2 || b % 2 || c % 2 || a / 2 < kMgMinCoarse || b / 2 < kMgMinCoarse || c / 2 < kMgMinCoarse) break;
        m.nx[m.L] = a / 2; m.ny[m.L] = b / 2; m.nz[m.L] = c / 2;
        ++m.L;
    }
    return m;
}

// workspace pieces beyond the Jacobi solver's: r, level 0's u, and per coarse
// level f, u, w and the weights
struct MgLayout {
    WsLayout base;
    size_t r, u0, lev[kMgMaxLevels][4];
    size_t total;
};

MgLayout mg_layout(const gbpcg_grid &g, int io) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    MgLayout M;
    M.base = ws_layout_n(n, GBPCG_F32, io, false, block_count(g));
    size_t o = M.base.total;
    M.r = o; o += round256(n * 4);
    M.u0 = o; o += round256(n * 4);
    const MgGeom G = mg_geom(g);
    for (int l = 1; l < G.L; ++l) {
        const size_t m = (size_t)G.nx[l] * G.ny[l] * G.nz[l];
        for (int v = 0; v < 3; ++v) {
            M.lev[l][v] = o;
            o += round256(m * 4);
        }
        M.lev[l][3] = o;
        o += round256(m * 16);
    }
    M.total = o;
    return M;
}

MgArgs mg_args(const gbpcg_grid &g, char *ws, const MgLayout &M, float *f0, float *z, const SolveState *st) {
    const MgGeom G = mg_geom(g);
    MgArgs a;
    memset(&a, 0, sizeof(a));
    a.L = G.L;
    for (int l = 0; l < G.L; ++l) {
        MgLevel &L = a.lv[l];
        L.nx = G.nx[l]; L.ny = G.ny[l]; L.nz = G.nz[l];
        if (l == 0) {
            L.f = f0;
            L.u = reinterpret_cast<float *>(ws + M.u0);
            L.w = z;
            L.W = nullptr;
        } else {
            L.f = reinterpret_cast<float *>(ws + M.lev[l][0]);
            L.u = reinterpret_cast<float *>(ws + M.lev[l][1]);
            L.w = reinterpret_cast<float *>(ws + M.lev[l][2]);
            L.W = reinterpret_cast<const float4 *>(ws + M.lev[l][3]);
        }
    }
    a.block = g.k_block ? 1 : 0;
    a.tab = g.k_block ? reinterpret_cast<const float4 *>(ws + M.base.tab) : nullptr;
    if (g.k_block) {
        a.rkbx = 1.0f / (float)g.kbx;
        a.rkby = 1.0f / (float)g.kby;
        a.rkbz = 1.0f / (float)g.kbz;
    }
    if (g.k_block) {
        a.ob = make_op_block(g);
    } else {
        memset(&a.ob, 0, sizeof(a.ob));
        auto c = [](int m) { double h = 1.0 / (m + 1); return (float)(1.0 / (h * h)); };
        a.ob.cx = c(g.nx); a.ob.cy = c(g.ny); a.ob.cz = c(g.nz);
    }
    a.st = st;
    return a;
}

unsigned mg_grid(int64_t n) {
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + kMgThreads - 1) / kMgThreads, (int64_t)device_sm_count() * 8));
}

// the coarse operators (once per solve)
cudaError_t mg_setup(const MgArgs &a, cudaStream_t s) {
    for (int l = 0; l + 1 < a.L; ++l) {
        const MgLevel &C = a.lv[l + 1];
        const MgLaunch g = mg_launch(C.nx, C.ny, C.nz);
        mg_galerkin_kernel<<<g.grid, g.block, 0, s>>>(a, l, const_cast<float4 *>(C.W), g.zper);
    }
    return cudaGetLastError();
}

// z = M f0 (a.lv[0].f -> a.lv[0].w)
cudaError_t mg_vcycle(const MgArgs &a, cudaStream_t s) {
    // levels whose rows split into 16-byte vectors take four points per thread (and their
    // restriction two coarse cells per thread)
    auto vec = [&](int l) { return a.lv[l].nx % 4 == 0; };
    // levels from l0 down (at most kMgTailCells cells each) run in one CTA
    int l0 = a.L - 1;
    while (l0 > 0 && (int64_t)a.lv[l0 - 1].nx * a.lv[l0 - 1].ny * a.lv[l0 - 1].nz <= kMgTailCells) --l0;
    // the kernels of one level, compiled for its kind of weights
    auto down = [&](auto wk_tag, int l) {
        constexpr int WK = decltype(wk_tag)::value;
        const MgLevel &L = a.lv[l], &C = a.lv[l + 1];
        if (vec(l) && WK == W_CONST0) {
            // constant coefficients: u = omega f / D is formed inside restriction and post-smoothing
            const MgLaunch gc = mg_launch(C.nx / 2, C.ny, C.nz);
            mg_restrict_kernel<2, WK, true><<<gc.grid, gc.block, 0, s>>>(a, l, gc.zper);
        } else if (vec(l)) {
            const MgLaunch gf = mg_launch(L.nx / 4, L.ny, L.nz), gc = mg_launch(C.nx / 2, C.ny, C.nz);
            mg_pre_kernel<4, WK><<<gf.grid, gf.block, 0, s>>>(a, l, gf.zper);
            mg_restrict_kernel<2, WK><<<gc.grid, gc.block, 0, s>>>(a, l, gc.zper);
        } else {
            const MgLaunch gf = mg_launch(L.nx, L.ny, L.nz), gc = mg_launch(C.nx, C.ny, C.nz);
            mg_pre_kernel<1, WK><<<gf.grid, gf.block, 0, s>>>(a, l, gf.zper);
            mg_restrict_kernel<1, WK><<<gc.grid, gc.block, 0, s>>>(a, l, gc.zper);
        }
    };
    auto up = [&](auto wk_tag, int l) {
        constexpr int WK = decltype(wk_tag)::value;
        const MgLevel &L = a.lv[l];
        const float *e = (l + 1 == a.L - 1) ? a.lv[l + 1].u : a.lv[l + 1].w;
        if (vec(l) && WK == W_CONST0) {
            const MgLaunch gf = mg_launch(L.nx / 4, L.ny, L.nz);
            mg_post_kernel<4, WK, true><<<gf.grid, gf.block, 0, s>>>(a, l, e, gf.zper);
        } else if (vec(l)) {
            const MgLaunch gf = mg_launch(L.nx / 4, L.ny, L.nz);
            mg_post_kernel<4, WK><<<gf.grid, gf.block, 0, s>>>(a, l, e, gf.zper);
        } else {
            const MgLaunch gf = mg_launch(L.nx, L.ny, L.nz);
            mg_post_kernel<1, WK><<<gf.grid, gf.block, 0, s>>>(a, l, e, gf.zper);
        }
    };
    using Const0 = std::integral_constant<int, W_CONST0>;
    using Tab0 = std::integral_constant<int, W_TAB0>;
    using Stored = std::integral_constant<int, W_STORED>;
    for (int l = 0; l < l0; ++l) {
        if (l > 0) down(Stored{}, l);
        else if (a.block) down(Tab0{}, 0);
        else down(Const0{}, 0);
    }
    mg_tail_kernel<<<1, kMgCoarseThreads, 0, s>>>(a, l0);
    for (int l = l0 - 1; l >= 0; --l) {
        if (l > 0) up(Stored{}, l);
        else if (a.block) up(Tab0{}, 0);
        else up(Const0{}, 0);
    }
    return cudaGetLastError();
}

int check_mg_grid(const gbpcg_grid *g) {
    if (int rc = check_grid(g)) return rc;
    const MgGeom G = mg_geom(*g);
    const int l = G.L - 1;
    if ((int64_t)G.nx[l] * G.ny[l] * G.nz[l] > kMgMaxCoarsest)
        return fail_arg("multigrid: the grid does not coarsen below 32768 cells (each size must be even, "
                        "down to >= 4, often enough)");
    if (g->nx % 4) return fail_arg("multigrid solves need nx a multiple of 4 (16-byte rows)");
    if (g->ny > 65535 || g->nz > 65535) return fail_arg("multigrid: ny and nz must be at most 65535");
    return GBPCG_OK;
}

// One MG-PCG solve recorded as a graph: the Jacobi solver's plan for pass A,
// the replacement and the finalize, plus pass R, the V-cycle and r.z.
template <typename Op>
struct MgSolve {
    SolvePlan<Op, true, double, float> sp;
    PassMaps mr;
    PassArgs ar;
    MgArgs mg;
    float *r, *z;
    int64_t n;

    cudaError_t launch_r(cudaStream_t s) {
        return GB_CFG_DISPATCH(sp.cfg_b, float, K_PASSR, true, Op, K::launch(mr, ar, sp.op, sp.gb.grid(), s));
    }
    void launch_rz(cudaStream_t s, int init) {
        mg_rz_kernel<<<mg_grid(n), kMgThreads, 0, s>>>(n, r, z, sp.st, sp.partials, init, sp.cond_loop, sp.use_cond);
    }

    int capture(cudaGraph_t *out) {
        cudaStream_t cs = nullptr, bs = nullptr, rs = nullptr;
        GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (!e) e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
        auto add_cond = [&](cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            cudaGraph_t *body_out) -> cudaError_t {
            cudaStreamCaptureStatus cst;
            cudaGraph_t cap = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            cudaError_t e2 = cudaStreamGetCaptureInfo(st, &cst, nullptr, &cap, &deps, nullptr, &ndeps);
            if (e2) return e2;
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = h;
            cp.conditional.type = type;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            e2 = cudaGraphAddNode(&node, cap, deps, nullptr, ndeps, &cp);
            if (e2) return e2;
            *body_out = cp.conditional.phGraph_out[0];
            return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        };
        cudaGraph_t graph = nullptr;
        bool cap_main = false, cap_b = false, cap_r = false;
        do {
            if (e) break;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e) break;
            cap_main = true;
            cudaStreamCaptureStatus cst;
            cudaGraph_t cap = nullptr;
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap, nullptr, nullptr, nullptr);
            if (e) break;
            cudaGraphConditionalHandle cond;
            e = cudaGraphConditionalHandleCreate(&cond, cap, 1, cudaGraphCondAssignDefault);
            if (e) break;
            sp.set_cond(cond, 0, 1);
            ar.cond = cond;
            ar.use_cond = 1;
            e = sp.launch_setup(cs);  // reset, max |b|, r0 = b - A x0 stored as r
            if (e) break;
            e = mg_setup(mg, cs);
            if (e) break;
            e = mg_vcycle(mg, cs);
            if (e) break;
            launch_rz(cs, 1);
            cudaGraph_t body = nullptr;
            e = add_cond(cs, cond, cudaGraphCondTypeWhile, &body);
            if (e) break;
            cudaGraphConditionalHandle rep;
            e = cudaGraphConditionalHandleCreate(&rep, body, 0, cudaGraphCondAssignDefault);
            if (e) break;
            sp.set_cond(cond, rep, 1);
            ar.cond_replace = rep;
            e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e) break;
            cap_b = true;
            e = sp.launch_a(bs);
            if (e) break;
            e = launch_r(bs);
            if (e) break;
            cudaGraph_t rbody = nullptr;
            e = add_cond(bs, rep, cudaGraphCondTypeIf, &rbody);
            if (e) break;
            e = cudaStreamBeginCaptureToGraph(rs, rbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e) break;
            cap_r = true;
            e = sp.launch_replace(rs);  // flush, r = b - A x (FP64) stored as r
            if (e) break;
            cudaGraph_t tmp = nullptr;
            e = cudaStreamEndCapture(rs, &tmp);
            cap_r = false;
            if (e) break;
            e = mg_vcycle(mg, bs);
            if (e) break;
            launch_rz(bs, 0);
            e = cudaStreamEndCapture(bs, &tmp);
            cap_b = false;
            if (e) break;
            e = sp.launch_final(cs);
            if (e) break;
            e = cudaStreamEndCapture(cs, &graph);
            cap_main = false;
        } while (0);
        cudaGraph_t tmp = nullptr;
        if (cap_r) cudaStreamEndCapture(rs, &tmp);
        if (cap_b) cudaStreamEndCapture(bs, &tmp);
        if (cap_main) {
            cudaStreamEndCapture(cs, &tmp);
            if (tmp) cudaGraphDestroy(tmp);
        }
        if (rs) cudaStreamDestroy(rs);
        if (bs) cudaStreamDestroy(bs);
        cudaStreamDestroy(cs);
        if (e) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail_cuda(e, "multigrid solve graph capture");
        }
        *out = graph;
        return GBPCG_OK;
    }
};

template <typename Op>
int mg_solve_op(const gbpcg_grid &g, const Op &op, const double *b, double *x, const gbpcg_opts &o, char *ws,
                const MgLayout &M, gbpcg_result *res, cudaStream_t s) {
    MgSolve<Op> P;
    int ca = 0, cb = 0;
    {
        const int narrow = g.nx <= 32 ? CFG_32x16 : g.nx <= 64 ? CFG_64x16 : -1;
        ca = narrow >= 0 ? narrow : (g.nx > 192 && g.nx <= 256) ? CFG_256x4 : CFG_128x8;
        cb = narrow >= 0 ? narrow : CFG_128x8;
    }
    if (int rc = P.sp.init(g, op, ca, cb, b, x, ws, M.base, o.tol, o.maxit, 1.0, nullptr)) return rc;
    P.n = (int64_t)g.nx * g.ny * g.nz;
    P.r = reinterpret_cast<float *>(ws + M.r);
    P.z = P.sp.z;
    // the FP64 residuals store r itself, in the r vector
    P.sp.ra.store_r = 1;
    P.sp.ra.z = P.r;
    // pass R: halo p_k (as pass B), centre and output r
    P.mr = P.sp.mb;
    if (make_pass_map<float>(&P.mr.c0, cb, false, P.r, g.nx, g.ny, g.nz)) return GBPCG_ERR_CUDA;
    P.ar = P.sp.ab;
    P.ar.c0 = P.r;
    P.ar.o0[0] = P.ar.o0[1] = P.r;
    P.ar.o1 = P.r;
    (void)GB_CFG_DISPATCH(cb, float, K_PASSR, true, Op, K::prepare());
    P.mg = mg_args(g, ws, M, P.r, P.z, P.sp.st);
    cudaGraph_t graph = nullptr;
    if (int rc = P.capture(&graph)) return rc;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return fail_cuda(e, "multigrid graph instantiate");
    struct ExecGuard { cudaGraphExec_t g; ~ExecGuard() { cudaGraphExecDestroy(g); } } eg{exec};
    cudaGraphUpload(exec, s);
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    GB_CUDA(cudaEventRecord(e0, s));
    GB_CUDA(cudaGraphLaunch(exec, s));
    GB_CUDA(cudaEventRecord(e1, s));
    SolveState hs;
    GB_CUDA(cudaMemcpyAsync(&hs, P.sp.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    res->iters = hs.it;
    res->status = hs.status;
    res->rel_res_recursive = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
    res->rel_res_true = hs.bb_true > 0 ? sqrt(hs.rr_true / hs.bb_true) : 0.0;
    res->time_ms = ms;
    res->replacements = hs.n_replace;
    res->pass_launches[0] = P.mg.L;  // levels of the hierarchy
    if (hs.status == GBPCG_TIMEOUT) set_error("a bounded device wait timed out during the solve");
    return hs.status;
}

}  // namespace

}  // namespace gb

using namespace gb;

extern "C" {

int gbpcg_mg_workspace_size(const gbpcg_grid *grid, size_t *bytes) {
    clear_error();
    if (int rc = check_mg_grid(grid)) return rc;
    if (!bytes) return fail_arg("bytes is NULL");
    *bytes = mg_layout(*grid, GBPCG_F64).total;
    return GBPCG_OK;
}

int gbpcg_mg_vcycle(const gbpcg_grid *grid, const float *r, float *z, void *workspace, size_t workspace_bytes,
                    int32_t *levels, gbpcg_stream stream) {
    clear_error();
    if (int rc = check_mg_grid(grid)) return rc;
    if (!r || !z || r == z) return fail_arg("r and z must be distinct device arrays");
    const MgLayout M = mg_layout(*grid, GBPCG_F64);
    if (!workspace || workspace_bytes < M.total || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return fail_arg("workspace: gbpcg_mg_workspace_size() bytes, 256-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const MgArgs a = mg_args(*grid, ws, M, const_cast<float *>(r), z, nullptr);
    if (grid->k_block) {  // the per-block face table the level-0 weights come from
        const int nbx = (grid->nx + grid->kbx - 1) / grid->kbx, nby = (grid->ny + grid->kby - 1) / grid->kby,
                  nbz = (grid->nz + grid->kbz - 1) / grid->kbz;
        const int64_t nb = (int64_t)nbx * nby * nbz;
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 4096));
        build_face_table<<<blocks, 256, 0, s>>>(grid->k_block, nbx, nby, nbz, const_cast<float4 *>(a.tab));
    }
    GB_CUDA(mg_setup(a, s));
    GB_CUDA(mg_vcycle(a, s));
    if (levels) *levels = a.L;
    return GBPCG_OK;
}

int gbpcg_mg_pcg_solve(const gbpcg_grid *grid, const double *b, double *x, const gbpcg_opts *opts,
                       gbpcg_result *result, gbpcg_stream stream) {
    NvtxRange range("gbpcg_mg_pcg_solve");
    clear_error();
    if (int rc = check_mg_grid(grid)) return rc;
    if (!opts || !b || !x || !result) return fail_arg("NULL argument");
    if (!(opts->tol >= 0.0) || opts->maxit < 0) return fail_arg("tol must be >= 0 and maxit >= 0");
    if (opts->precond != GBPCG_PRECOND_MG || opts->io_dtype != GBPCG_F64 || opts->storage != GBPCG_F32 || opts->flags)
        return fail_arg("multigrid solves take precond MG, FP64 b and x, FP32 vectors, no flags");
    if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15u)
        return fail_arg("b and x must be 16-byte aligned");
    const MgLayout M = mg_layout(*grid, GBPCG_F64);
    if (!opts->workspace || opts->workspace_bytes < M.total || (reinterpret_cast<uintptr_t>(opts->workspace) & 255u))
        return fail_arg("workspace: gbpcg_mg_workspace_size() bytes, 256-byte aligned");
    memset(result, 0, sizeof(*result));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(opts->workspace);
    const gbpcg_grid &g = *grid;
    if (g.k_block)
        return mg_solve_op(g, make_op_table(g, 1.0f, reinterpret_cast<const float4 *>(ws + M.base.tab)), b, x, *opts,
                           ws, M, result, s);
    return mg_solve_op(g, make_op_const(g.nx, g.ny, g.nz), b, x, *opts, ws, M, result, s);
}

}  // extern "C"
