// Z-marching stencil engine: the data path shared by the stencil apply and
// the fused PCG passes.
//
// Each CTA owns a TX x TY tile of the (x, y) plane and marches through a
// contiguous range of z planes [k0, k1).  Plane m of every input array
// arrives in shared memory as one box: the "halo" arrays with one extra row
// above/below and XH extra columns left/right (XH = 16 bytes of elements, so
// the box's x origin stays 16-byte aligned as TMA requires), the "center"
// arrays without halo.  Boxes reaching outside the grid are zero-filled by
// the TMA unit, which is exactly the zero Dirichlet boundary (the paper's
// explicit zero fill, Sec. VI-C, costs nothing here).  An S-stage ring of
// boxes is kept in flight, each stage completed by one mbarrier.
//
// The seven-point operator at plane k needs the input at planes k-1, k, k+1
// in the thread's own column (kept in registers as a 3-deep queue) and the
// four in-plane neighbours (read from the plane-k box).  One thread computes
// one 16-byte vector of a row: four FP32 or eight 16-bit x points.
//
// Pass kinds (Sec. VII's PCG split into two data passes plus setup):
//   K_STENCIL  q = A p
//   K_PASSA    p_k = z_k + beta_{k-1} p_{k-1} formed on the fly for every
//              stencil input (no D needed: z, not r, is the stored vector);
//              d += alpha_{k-1} p_{k-1} (deferred update of the previous
//              iteration into the correction vector d, see solver.cuh); stores
//              p_k; sum p_k . A p_k -> alpha_k
//   K_PASSB    q = A p_k recomputed (cheaper than storing it),
//              r = D z - alpha_k q, z = D^-1 r; stores z; sums r.r, r.z
//              -> beta_k, the convergence test and the residual-replacement
//              trigger
//   K_PASSR    (preconditioners other than Jacobi, which keep r itself)
//              q = A p_k recomputed, r -= alpha_k q; stores r; sums r.r
//              -> the convergence test and the replacement trigger (beta
//              follows once the preconditioner has been applied to r)
#pragma once

#include <type_traits>

#include "common.cuh"

namespace gb {

enum PassKind { K_STENCIL = 0, K_PASSA = 2, K_PASSB = 3, K_PASSR = 7 };

// Device-resident solver scalars (one per solve).
struct __align__(16) SolveState {
    double rz;      // r_k . z_k
    double pq;      // p_k . A p_k
    double alpha;   // alpha_k
    double beta;    // beta_{k-1}
    double rr;      // ||r_k||^2 (recursive)
    double bb;      // ||b||^2
    double tol2;    // tol^2
    double rr_true; // ||b - A x||^2 (FP64 stencil, compensated FP32 sum of squares)
    double bb_true; // ||b||^2, FP64
    int it;         // completed iterations
    int maxit;
    int done;       // 1: stop iterating
    int status;     // gbpcg_status
    int pending;    // 1: x still lacks alpha_{it-1} p_{it-1}
    int zero_x;     // 1: b == 0, x must be zeroed
    int timeout;    // a bounded wait gave up somewhere
    int replace;    // 1: flush d into x and replace r by b - A x (FP64) now
    double rr_rep;  // ||r||^2 at the last residual replacement
    double rr_conf; // ||b - A x||^2 at the last confirmation (recursive residual had met tol)
    int n_replace;  // residual replacements done
    int true_known; // 1: rr_true, bb_true already hold b - A x of the final x
    unsigned long long rhs_bits;  // max |b| as the bit pattern of a non-negative double
    double rzm;     // r.M r of the last residual (preconditioners other than Jacobi)
    unsigned int ticket[8];
};

// Power of two s that brings max |b| into [0.5, 1) when it lies outside
// [2^-21, 2^20), else 1.  The solver works on s b and s x (exact scalings):
// the FP32 iteration vectors and their FP32 partial sums then stay far from
// underflow and overflow whatever the scale of b.
__device__ __forceinline__ double rhs_scale(unsigned long long bits) {
    const double m = __longlong_as_double((long long)bits);
    if (!(m > 0.0) || !isfinite(m)) return 1.0;
    int e = 0;
    frexp(m, &e);
    if (e >= -20 && e <= 20) return 1.0;
    return ldexp(1.0, -e);
}

// A residual replacement is triggered whenever ||r|| has dropped by this
// factor squared since the last one (two decades of residual norm), and
// when the recursive residual meets the tolerance.  Every decade measured
// the same iterations and true residuals at 256^3 and 512^3 with twice the
// replacements (each an FP64-bound b - A x on GB300).
constexpr double kReplaceDrop2 = 1e-4;

// Constant-coefficient operator: face weights 1/h_d^2.
struct NoCache {};

struct OpConst {
    static constexpr bool kConst = true;
    using Cache = NoCache;
    float cx, cy, cz;
    float d;      // diagonal 2 (cx + cy + cz)
    float inv_d;  // 1 / d
    // q = (A u)_c from the centre and its six neighbours; dg = diagonal
    __device__ __forceinline__ void apply(float c, float xm, float xp, float ym, float yp, float zm, float zp, int,
                                          int, int, float &q, float &dg) const {
        q = fmaf(d, c, -fmaf(cx, xm + xp, fmaf(cy, ym + yp, cz * (zm + zp))));
        dg = d;
    }
    template <int V>
    __device__ __forceinline__ void applyv(Cache &, const float c[V], float xl, float xr, const float ym[V],
                                           const float yp[V], const float zm[V], const float zp[V], int gx, int gy,
                                           int k, int nx, int ny, float q[V], float dg[V], float rdg[V]) const;
};

// Block-constant coefficient k (one float per kbx*kby*kbz block): face
// weight k_f / h_d^2 with k_f the harmonic mean across a block face, the
// cell's own k inside a block and on the domain boundary.
struct OpBlock {
    static constexpr bool kConst = false;
    using Cache = NoCache;
    float inv_d;  // unused
    const float *kb;
    int nx, ny, nz, nbx, nby, kbx, kby, kbz;
    float cx, cy, cz;
    __device__ __forceinline__ float K(int bx, int by, int bz) const {
        return __ldg(kb + ((size_t)bz * nby + by) * nbx + bx);
    }
    __device__ __forceinline__ static float hm(float a, float b) { return 2.0f * a * b / (a + b); }
    __device__ __forceinline__ void weights(int i, int j, int k, float w[6]) const {
        const int bx = i / kbx, by = j / kby, bz = k / kbz;
        const int ix = i - bx * kbx, iy = j - by * kby, iz = k - bz * kbz;
        const float kc = K(bx, by, bz);
        w[0] = cx * ((ix == 0 && i > 0) ? hm(kc, K(bx - 1, by, bz)) : kc);
        w[1] = cx * ((ix == kbx - 1 && i < nx - 1) ? hm(kc, K(bx + 1, by, bz)) : kc);
        w[2] = cy * ((iy == 0 && j > 0) ? hm(kc, K(bx, by - 1, bz)) : kc);
        w[3] = cy * ((iy == kby - 1 && j < ny - 1) ? hm(kc, K(bx, by + 1, bz)) : kc);
        w[4] = cz * ((iz == 0 && k > 0) ? hm(kc, K(bx, by, bz - 1)) : kc);
        w[5] = cz * ((iz == kbz - 1 && k < nz - 1) ? hm(kc, K(bx, by, bz + 1)) : kc);
    }
    __device__ __forceinline__ void apply(float c, float xm, float xp, float ym, float yp, float zm, float zp, int i,
                                          int j, int k, float &q, float &dg) const {
        float w[6];
        weights(i, j, k, w);
        q = w[0] * (c - xm) + w[1] * (c - xp) + w[2] * (c - ym) + w[3] * (c - yp) + w[4] * (c - zm) + w[5] * (c - zp);
        dg = ((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]);
    }
    template <int V>
    __device__ __forceinline__ void applyv(Cache &, const float c[V], float xl, float xr, const float ym[V],
                                           const float yp[V], const float zm[V], const float zp[V], int gx, int gy,
                                           int k, int nx_, int ny_, float q[V], float dg[V], float rdg[V]) const;
};

// 1/x by the hardware's approximate reciprocal (PTX rcp.approx.ftz.f32: at
// most one unit in the last place off, for the normal positive diagonals it
// is given).  The Jacobi step z = r * rcp(D) is then a fixed diagonal scaling
// of r, as a preconditioner must be; the FP64 residual steps divide exactly,
// which differs from it by the same unit in the last place.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The operator at one thread's V consecutive x points: c = centre values,
// xl / xr = the x neighbours left of point 0 and right of point V-1, y and
// z neighbours per point.  Point positions past the grid edge (masked lanes)
// are clamped into the grid before any coefficient lookup.  rdg receives the
// reciprocal of each diagonal (the Jacobi step multiplies by it; the
// compiler drops it where a pass does not use it).
template <int V, typename Op>
__device__ __forceinline__ void applyv_pointwise(const Op &op, const float c[V], float xl, float xr, const float ym[V],
                                                 const float yp[V], const float zm[V], const float zp[V], int gx,
                                                 int gy, int k, int nx, int ny, float q[V], float dg[V],
                                                 float rdg[V]) {
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const float xm = i == 0 ? xl : c[i - 1];
        const float xp = i == V - 1 ? xr : c[i + 1];
        op.apply(c[i], xm, xp, ym[i], yp[i], zm[i], zp[i], min(gx + i, nx - 1), min(gy, ny - 1), k, q[i], dg[i]);
        rdg[i] = Op::kConst ? op.inv_d : rcp_approx(dg[i]);
    }
}

template <int V>
__device__ __forceinline__ void OpConst::applyv(Cache &, const float c[V], float xl, float xr, const float ym[V],
                                                const float yp[V], const float zm[V], const float zp[V], int gx,
                                                int gy, int k, int nx, int ny, float q[V], float dg[V],
                                                float rdg[V]) const {
    applyv_pointwise<V>(*this, c, xl, xr, ym, yp, zm, zp, gx, gy, k, nx, ny, q, dg, rdg);
}
template <int V>
__device__ __forceinline__ void OpBlock::applyv(Cache &, const float c[V], float xl, float xr, const float ym[V],
                                                const float yp[V], const float zm[V], const float zp[V], int gx,
                                                int gy, int k, int nx_, int ny_, float q[V], float dg[V],
                                                float rdg[V]) const {
    applyv_pointwise<V>(*this, c, xl, xr, ym, yp, zm, zp, gx, gy, k, nx_, ny_, q, dg, rdg);
}

// Block-constant coefficient through a per-block face table built once per
// solve (build_face_table in solver.cuh): for block b, tab[2b] = {k, k_x-,
// k_x+, k_y-}, tab[2b+1] = {k_y+, k_z-, k_z+, 0}, each face value the
// harmonic mean with the neighbouring block or, on the domain boundary, k
// itself.  One lookup serves a thread's four points when kbx is a multiple
// of 4; the weights are bitwise those of OpBlock.
struct OpTable {
    static constexpr bool kConst = false;
    float inv_d;  // unused
    const float4 *tab;
    int nx, ny, nz, nbx, nby, kbx, kby, kbz;
    int grouped4, grouped8;  // kbx % 4 == 0 / kbx % 8 == 0: a thread's 4 / 8 points share one block
    float cx, cy, cz;
    __device__ __forceinline__ void lookup(int bx, int by, int bz, float4 &t0, float4 &t1) const {
        const float4 *t = tab + 2 * (((size_t)bz * nby + by) * nbx + bx);
        t0 = __ldg(t);
        t1 = __ldg(t + 1);
    }
    __device__ __forceinline__ void apply(float c, float xm, float xp, float ym, float yp, float zm, float zp, int i,
                                          int j, int k, float &q, float &dg) const {
        const int bx = i / kbx, by = j / kby, bz = k / kbz;
        const int ix = i - bx * kbx, iy = j - by * kby, iz = k - bz * kbz;
        float4 t0, t1;
        lookup(bx, by, bz, t0, t1);
        const float kc = t0.x;
        const float w0 = cx * (ix == 0 ? t0.y : kc), w1 = cx * (ix == kbx - 1 ? t0.z : kc);
        const float w2 = cy * (iy == 0 ? t0.w : kc), w3 = cy * (iy == kby - 1 ? t1.x : kc);
        const float w4 = cz * (iz == 0 ? t1.y : kc), w5 = cz * (iz == kbz - 1 ? t1.z : kc);
        q = w0 * (c - xm) + w1 * (c - xp) + w2 * (c - ym) + w3 * (c - yp) + w4 * (c - zm) + w5 * (c - zp);
        dg = ((w0 + w1) + (w2 + w3)) + (w4 + w5);
    }
    // A thread's block column (bx, by, x/y offsets) is fixed; its table entry
    // changes only when the march crosses a z block, so the weights derived
    // from it are kept in registers and recomputed then.  The z block and
    // offset follow the march plane by plane (no integer division per plane).
    struct Cache {
        int bz = -1, bx = 0, by = 0, ix0 = 0, iy = 0, iz = 0, k = -2;
        float kc, kzm, kzp;       // block k and its -z / +z face values
        float w2, w3, wi, wf, wl; // y- / y+ weights; interior, point 0 (-x) and point V-1 (+x) x weights
    };
    template <int V>
    __device__ __forceinline__ void applyv(Cache &cc, const float c[V], float xl, float xr, const float ym[V],
                                           const float yp[V], const float zm[V], const float zp[V], int gx, int gy,
                                           int k, int nx_, int ny_, float q[V], float dg[V], float rdg[V]) const {
        if (!(V == 4 ? grouped4 : grouped8)) {
            applyv_pointwise<V>(*this, c, xl, xr, ym, yp, zm, zp, gx, gy, k, nx_, ny_, q, dg, rdg);
            return;
        }
        int bz, iz;
        if (cc.bz >= 0 && k == cc.k + 1) {
            bz = cc.bz;
            iz = cc.iz + 1;
            if (iz == kbz) { iz = 0; ++bz; }
        } else if (cc.bz >= 0 && k == cc.k - 1) {
            bz = cc.bz;
            iz = cc.iz - 1;
            if (iz < 0) { iz = kbz - 1; --bz; }
        } else {
            bz = k / kbz;
            iz = k - bz * kbz;
        }
        cc.k = k;
        cc.iz = iz;
        if (bz != cc.bz) {
            if (cc.bz < 0) {
                const int i0 = min(gx, (nx - 1) & ~(V - 1)), j = min(gy, ny - 1);  // gx is a multiple of V
                cc.bx = i0 / kbx;
                cc.by = j / kby;
                cc.ix0 = i0 - cc.bx * kbx;
                cc.iy = j - cc.by * kby;
            }
            cc.bz = bz;
            float4 t0, t1;
            lookup(cc.bx, cc.by, bz, t0, t1);
            const float kc = t0.x;
            cc.kc = kc;
            cc.kzm = t1.y;
            cc.kzp = t1.z;
            cc.w2 = cy * (cc.iy == 0 ? t0.w : kc);
            cc.w3 = cy * (cc.iy == kby - 1 ? t1.x : kc);
            // kbx and ix0 are multiples of V: only point 0 can sit on a block's -x face and only
            // point V-1 on its +x face; the others have x weights cx k on both sides
            cc.wi = cx * kc;
            cc.wf = cx * (cc.ix0 == 0 ? t0.y : kc);
            cc.wl = cx * (cc.ix0 + V - 1 == kbx - 1 ? t0.z : kc);
        }
        const float w4 = cz * (iz == 0 ? cc.kzm : cc.kc), w5 = cz * (iz == kbz - 1 ? cc.kzp : cc.kc);
        const float wyz = (cc.w2 + cc.w3) + (w4 + w5);
        // three diagonals cover the V points (and three reciprocals, rcp_approx)
        const float di = (cc.wi + cc.wi) + wyz, d0 = (cc.wf + cc.wi) + wyz, dl = (cc.wi + cc.wl) + wyz;
        const float ri = rcp_approx(di), r0 = rcp_approx(d0), rl = rcp_approx(dl);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float xm = i == 0 ? xl : c[i - 1];
            const float xp = i == V - 1 ? xr : c[i + 1];
            const float w0 = i == 0 ? cc.wf : cc.wi, w1 = i == V - 1 ? cc.wl : cc.wi;
            // (A u)_c = sum of w_f (u_c - u_f): for smooth u the differences are small and
            // nearly exact, where dg u_c - sum w_f u_f would cancel at the scale of dg u_c
            float sq = w0 * (c[i] - xm);
            sq = fmaf(w1, c[i] - xp, sq);
            sq = fmaf(cc.w2, c[i] - ym[i], sq);
            sq = fmaf(cc.w3, c[i] - yp[i], sq);
            sq = fmaf(w4, c[i] - zm[i], sq);
            q[i] = fmaf(w5, c[i] - zp[i], sq);
            dg[i] = i == 0 ? d0 : i == V - 1 ? dl : di;
            rdg[i] = i == 0 ? r0 : i == V - 1 ? rl : ri;
        }
    }
};

struct __align__(128) PassMaps {
    CUtensorMap h0[2];  // halo array 0 (two candidates, chosen by iteration parity)
    CUtensorMap h1[2];  // halo array 1
    CUtensorMap c0;     // center array
};

struct PassArgs {
    int nx, ny, nz;
    int tiles_x, zchunk;
    int zparts;  // CTAs sharing one z chunk, each marching one part of it (0 or 1: whole chunks)
    const void *h0[2];
    const void *h1[2];
    const void *c0;
    void *o0[2];
    void *o1;
    SolveState *st;
    double *partials;
    cudaGraphConditionalHandle cond;          // WHILE condition of the iteration loop
    cudaGraphConditionalHandle cond_replace;  // IF condition of the residual replacement
    int use_cond;
    float scale;  // stencil apply: output multiplier (1 normally)
    int l2hint;   // pass A: p_{k-1} and d marked evict-first in L2 (march_tile)
};

constexpr uint32_t round128(uint32_t v) { return (v + 127u) & ~127u; }

// Tiles of width 256 span a whole grid row (nx <= 256): they need no x halo,
// so their boxes are whole rows, contiguous in memory.
template <int TX>
constexpr bool full_row() { return TX == 256; }

// Type of the centre array and of the second output: pass A's correction
// vector d is FP32 whatever the storage type of z and p (16-bit d rounds at
// the scale of |d|, and A amplifies that noise far beyond a 16-bit solve's
// residual on fine grids); elsewhere it is the storage type.
template <typename T, int KIND>
using CenterT = typename std::conditional<KIND == K_PASSA, float, T>::type;

template <typename T, int TX, int TY, int KIND>
struct Geometry {
    static constexpr int V = 16 / (int)sizeof(T);  // points per thread: one 16-byte vector of T
    static constexpr int NT = TX / V * TY;
    static constexpr int XH = full_row<TX>() ? 0 : 16 / (int)sizeof(T);
    static constexpr int HX = TX + 2 * XH, HY = TY + 2;
    static constexpr int NH = KIND == K_PASSA ? 2 : 1;
    static constexpr int NC = KIND == K_STENCIL ? 0 : 1;
    static constexpr int NV = KIND == K_PASSA ? 1 : KIND == K_PASSB ? 2 : KIND == K_PASSR ? 1 : 0;
    static constexpr uint32_t HBYTES = HX * HY * sizeof(T);
    static constexpr uint32_t CBYTES = TX * TY * sizeof(CenterT<T, KIND>);
    static constexpr uint32_t HB = round128(HBYTES), CB = round128(CBYTES);
    static constexpr uint32_t SB = NH * HB + NC * CB;
};

template <typename T, int TX, int TY, int S, int KIND>
constexpr size_t zmarch_smem_bytes() {
    return (size_t)S * Geometry<T, TX, TY, KIND>::SB;
}

// Copies one box (w x h at (xs, ys, m)) into shared memory with plain loads,
// zero outside the grid.  Used when the arrays do not meet TMA's alignment.
template <typename T, int NT>
__device__ __forceinline__ void manual_box(const T *src, T *dst, int nx, int ny, int nz, int xs,
                                           int ys, int m, int w, int h) {
    for (int e = threadIdx.x; e < w * h; e += NT) {
        const int r = e / w, c = e - r * w;
        const int gx = xs + c, gy = ys + r;
        T v = from_f<T>(0.0f);
        if (m >= 0 && m < nz && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
            v = src[((size_t)m * ny + gy) * nx + gx];
        dst[e] = v;
    }
}

// The pointers and tensor maps one pass reads and writes for one problem.
template <typename T, int KIND>
struct MarchIO {
    using TC = CenterT<T, KIND>;
    const T *H0, *H1;
    const TC *C0;
    T *O0;
    TC *O1;
    const CUtensorMap *M0, *M1, *MC;
    bool l2hint = false;  // pass A: p_{k-1} and d leave L2 first (see march_tile)
};

// The solver scalars a pass reads when it starts (iteration k = it).
struct MarchScalars {
    int it;
    float alpha;       // pass B: alpha_k
    float beta;        // pass A: beta_{k-1}
    float alpha_prev;  // pass A: alpha_{k-1}, for the deferred d update
    bool first;        // pass A: k == 0 (p_0 = z_0, no p_{k-1} to load)
    bool do_x;         // pass A: d still lacks alpha_{k-1} p_{k-1}
};

// SP is `const SolveState *`, or `const volatile SolveState *` in a
// persistent kernel, where another SM may have written the scalars during
// the same launch.  (Volatile accesses cost an L2 round trip each, which on
// the serial last-CTA step of every pass shows up in the pass time, so the
// single-problem passes use plain ones: their scalars were written by an
// earlier launch.)  The same holds for the finish steps below.
template <int KIND, typename SP>
__device__ __forceinline__ MarchScalars read_scalars(SP st) {
    MarchScalars sc{};
    if constexpr (KIND == K_PASSA || KIND == K_PASSB || KIND == K_PASSR) sc.it = st->it;
    if constexpr (KIND == K_PASSA) {
        sc.first = (sc.it == 0);
        sc.beta = (float)st->beta;
        sc.alpha_prev = (float)st->alpha;
        sc.do_x = st->pending != 0;
    }
    if constexpr (KIND == K_PASSB || KIND == K_PASSR) sc.alpha = (float)st->alpha;
    return sc;
}

// ZFILL (an ablation of Sec. VI-C, off in every solver path): after each
// TMA box lands, tiles that touch the domain boundary also zero the
// out-of-grid part of the box explicitly, the work the paper's kernels do by
// hand; here the TMA unit has already written those zeros, so the variant
// measures what explicit zero filling would cost.
//
// One CTA marches one tile (x0, y0) through planes [k0, k1) and adds its
// points' partial sums into acc.  Loads go round an S-stage ring whose
// stages and mbarrier phases continue from `ring` (the loads the CTA issued
// before: a persistent CTA marches many tiles through one ring); the
// function returns the number of loads this march issued.  A wait that runs
// out sets *s_timeout; the march then stops, waits (bounded) for its copies
// still in flight and returns.
template <typename T, int TX, int TY, int S, int KIND, bool TMA, typename Op, bool ZFILL>
__device__ __forceinline__ uint32_t march_tile(unsigned char *smem, uint64_t *full, volatile int *s_timeout,
                                               uint32_t ring, const MarchIO<T, KIND> &io, const Op &op, int nx,
                                               int ny, int nz, int x0, int y0, int k0, int k1, const MarchScalars &sc,
                                               float (&acc)[Geometry<T, TX, TY, KIND>::NV > 0
                                                                ? Geometry<T, TX, TY, KIND>::NV
                                                                : 1]) {
    static_assert(S >= 2, "a stage is refilled only after the step that reads it as the output plane");
    using G = Geometry<T, TX, TY, KIND>;
    using TC = CenterT<T, KIND>;
    constexpr int NT = G::NT, XH = G::XH, HX = G::HX, NH = G::NH, V = G::V;
    constexpr uint32_t HB = G::HB, SB = G::SB;
    if (k0 >= k1) return 0;

    const int lx = threadIdx.x % (TX / V), ly = threadIdx.x / (TX / V);
    const int gx = x0 + V * lx, gy = y0 + ly;
    bool ok[V];
#pragma unroll
    for (int i = 0; i < V; ++i) ok[i] = gy < ny && gx + i < nx;

    const bool first = sc.first, do_x = sc.do_x;
    const float alpha = sc.alpha, beta = sc.beta, alpha_prev = sc.alpha_prev;
    const bool load_h1 = NH == 2 && !first;
    const bool load_c = G::NC == 1 && !(KIND == K_PASSA && !do_x);
    uint64_t dpol = 0;
    if (KIND == K_PASSA && TMA && io.l2hint) dpol = l2_policy_evict_first();

    // Planes are visited in march order: step t = 0..tl loads plane pl(t),
    // forward pl(t) = k0 - 1 + t, reverse pl(t) = k1 - t (the first and the
    // last loaded planes are halo planes); step t >= 2 outputs plane pl(t-1).
    // Pass B marches down so it starts on the planes pass A touched last,
    // which are still in L2; the next pass A, marching up, starts where pass
    // B ended.
    constexpr bool REV = KIND == K_PASSB || KIND == K_PASSR;
    const int tl = k1 - k0 + 1;
    auto plane = [&](int t) { return REV ? k1 - t : k0 - 1 + t; };
    auto stage = [&](int t) { return (int)((ring + (uint32_t)t) % S); };
    auto parity = [&](int t) { return (uint32_t)(((ring + (uint32_t)t) / S) & 1u); };

    auto issue = [&](int t) {
        const int m = plane(t);
        const int s = stage(t);
        unsigned char *base = smem + (size_t)s * SB;
        const bool cen = load_c && t >= 1 && t < tl;
        if constexpr (TMA) {
            if (threadIdx.x == 0) {
                const uint32_t bytes = G::HBYTES + (load_h1 ? G::HBYTES : 0u) + (cen ? G::CBYTES : 0u);
                mbar_arrive_expect_tx(&full[s], bytes);
                tma_load_3d(base, io.M0, &full[s], x0 - XH, y0 - 1, m);
                if (KIND == K_PASSA && io.l2hint) {
                    // pass A's p_{k-1} (overwritten next iteration) and d (read again only by the
                    // next pass A) leave L2 first: pass B reads what pass A read and wrote besides
                    // (z_k, p_k).  Measured: a gain where that data nearly fits in L2 (256^3: pass
                    // A 58.2 -> 56.7 us, pass B 41.0 -> 39.1 us), a loss on grids far larger
                    // (512^3 pass A 440 -> 461 us) and in the persistent batch, so the solver
                    // sets it by grid size.
                    const uint64_t pol = l2_policy_evict_first();
                    if (load_h1) tma_load_3d_hint(base + HB, io.M1, &full[s], x0 - XH, y0 - 1, m, pol);
                    if (cen) tma_load_3d_hint(base + NH * HB, io.MC, &full[s], x0, y0, m, pol);
                } else {
                    if (load_h1) tma_load_3d(base + HB, io.M1, &full[s], x0 - XH, y0 - 1, m);
                    if (cen) tma_load_3d(base + NH * HB, io.MC, &full[s], x0, y0, m);
                }
            }
        } else {
            manual_box<T, NT>(io.H0, reinterpret_cast<T *>(base), nx, ny, nz, x0 - XH, y0 - 1, m, HX, TY + 2);
            if (load_h1)
                manual_box<T, NT>(io.H1, reinterpret_cast<T *>(base + HB), nx, ny, nz, x0 - XH, y0 - 1, m, HX,
                                  TY + 2);
            if (cen) manual_box<TC, NT>(io.C0, reinterpret_cast<TC *>(base + NH * HB), nx, ny, nz, x0, y0, m, TX, TY);
            __syncthreads();
        }
    };

    // stencil-input value at (row, col) of a stage box
    auto in_val = [&](const unsigned char *base, int idx) -> float {
        float v = to_f(reinterpret_cast<const T *>(base)[idx]);
        if constexpr (KIND == K_PASSA) {
            if (!first) v = fmaf(beta, to_f(reinterpret_cast<const T *>(base + HB)[idx]), v);
        }
        return v;
    };
    auto in_valv = [&](const unsigned char *base, int idx, float v[V]) {
        ldv<T, V>(reinterpret_cast<const T *>(base) + idx, v);
        if constexpr (KIND == K_PASSA) {
            if (!first) {
                float p[V];
                ldv<T, V>(reinterpret_cast<const T *>(base + HB) + idx, p);
#pragma unroll
                for (int i = 0; i < V; ++i) v[i] = fmaf(beta, p[i], v[i]);
            }
        }
    };

    int issued_hi = -1;
    int consumed = -1;
    for (int t = 0; t <= tl && t < S; ++t) {
        issue(t);
        issued_hi = t;
    }
    // The three planes around the output plane live in q0, q1, q2; each step
    // loads the next plane over the oldest, and the roles (below, centre,
    // above) rotate with the step instead of the values moving: the march
    // loop is unrolled three times, one copy per rotation (below).
    float q0[V], q1[V], q2[V];
#pragma unroll
    for (int i = 0; i < V; ++i) q0[i] = q1[i] = q2[i] = 0.f;
    typename Op::Cache opc;
    const int cidx = (ly + 1) * HX + XH + V * lx;  // this thread's first point in a halo box
    // one march step t; qa, qb, qc = planes pl(t-2), pl(t-1), pl(t) (qc loaded here); false: stop
    auto step = [&](int t, float (&qa)[V], float (&qb)[V], float (&qc)[V]) -> bool {
        const int s = stage(t);
        const unsigned char *base = smem + (size_t)s * SB;
        if constexpr (TMA) {
            if (!mbar_wait_bounded(&full[s], parity(t))) *s_timeout = 1;
        }
        consumed = t;
        if constexpr (ZFILL) {
            const int m = plane(t);
            const bool edge = m < 0 || m >= nz || x0 - XH < 0 || x0 + TX + XH > nx || y0 - 1 < 0 ||
                              y0 + TY + 1 > ny;
            if (edge) {
                T *hb = reinterpret_cast<T *>(smem + (size_t)s * SB);
                for (int e = threadIdx.x; e < HX * G::HY; e += NT) {
                    const int r = e / HX, c = e - r * HX;
                    const int bx = x0 - XH + c, by = y0 - 1 + r;
                    if (m < 0 || m >= nz || bx < 0 || bx >= nx || by < 0 || by >= ny) hb[e] = from_f<T>(0.0f);
                }
                // generic-proxy writes before the TMA refills this stage
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            __syncthreads();
        }
        in_valv(base, cidx, qc);
        if (t >= 2) {
            // ---- output plane k = pl(t-1) from its own stage ----
            const int k = plane(t - 1);
            const unsigned char *bk = smem + (size_t)stage(t - 1) * SB;
            float ym[V], yp[V];
            in_valv(bk, cidx - HX, ym);
            in_valv(bk, cidx + HX, yp);
            // whole-row tiles: the x neighbours past either end of the row are
            // boundary zeros (the box holds no x halo)
            const float xl = (full_row<TX>() && lx == 0) ? 0.0f : in_val(bk, cidx - 1);
            const float xr = (full_row<TX>() && lx == TX / V - 1) ? 0.0f : in_val(bk, cidx + V);
            float q[V], dg[V], rdg[V];
            op.template applyv<V>(opc, qb, xl, xr, ym, yp, REV ? qc : qa, REV ? qa : qc, gx, gy, k, nx, ny, q,
                                  dg, rdg);
            const size_t g = ((size_t)k * ny + gy) * nx + gx;
            const TC *cen = reinterpret_cast<const TC *>(bk + NH * HB) + ly * TX + V * lx;
            float out0[V], out1[V];
            bool st1 = false;
            if constexpr (KIND == K_STENCIL) {
                (void)alpha;
#pragma unroll
                for (int i = 0; i < V; ++i) out0[i] = q[i] * sc.alpha;  // alpha carries the output scale
            } else if constexpr (KIND == K_PASSA) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    out0[i] = qb[i];
                    if (ok[i]) acc[0] = fmaf(qb[i], q[i], acc[0]);
                }
                if (do_x) {
                    float xv[V], po[V];
                    ldv<TC, V>(cen, xv);
                    ldv<T, V>(reinterpret_cast<const T *>(bk + HB) + cidx, po);
#pragma unroll
                    for (int i = 0; i < V; ++i) out1[i] = fmaf(alpha_prev, po[i], xv[i]);
                    st1 = true;
                }
            } else if constexpr (KIND == K_PASSR) {
                float rv[V];
                ldv<TC, V>(cen, rv);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const float r = fmaf(-alpha, q[i], rv[i]);
                    out0[i] = r;
                    if (ok[i]) acc[0] = fmaf(r, r, acc[0]);
                }
            } else {  // K_PASSB
                float zv[V];
                ldv<TC, V>(cen, zv);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const float r = fmaf(-alpha, q[i], dg[i] * zv[i]);
                    const float z = r * rdg[i];  // D^-1 r
                    out0[i] = z;
                    if (ok[i]) {
                        acc[0] = fmaf(r, r, acc[0]);
                        acc[1] = fmaf(r, z, acc[1]);
                    }
                }
            }
            if (ok[0] && ok[V - 1] && TMA) {
                stv<T, V>(io.O0 + g, out0);
                if constexpr (KIND == K_PASSA && std::is_same<TC, float>::value) {
                    if (st1 && io.l2hint) {  // d: evict first (above)
#pragma unroll
                        for (int i = 0; i < V; i += 4) st4f_hint(io.O1 + g + i, out1 + i, dpol);
                    } else if (st1) {
                        stv<TC, V>(io.O1 + g, out1);
                    }
                } else {
                    if (st1) stv<TC, V>(io.O1 + g, out1);
                }
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (ok[i]) {
                        io.O0[g + i] = from_f<T>(out0[i]);
                        if (st1) io.O1[g + i] = from_f<TC>(out1[i]);
                    }
            }
        }
        __syncthreads();
        if (*s_timeout) return false;
        if (t >= 1 && t - 1 + S <= tl) {
            issue(t - 1 + S);
            issued_hi = t - 1 + S;
        }
        return true;
    };
    // The 16-bit pass A is bound by memory bandwidth, and the threefold
    // copy costs it registers (occupancy): it moves the values instead.
    constexpr bool ROTATE = !(KIND == K_PASSA && sizeof(T) == 2);
    if constexpr (ROTATE) {
        for (int t = 0; t <= tl;) {
            if (!step(t, q1, q2, q0) || ++t > tl) break;
            if (!step(t, q2, q0, q1) || ++t > tl) break;
            if (!step(t, q0, q1, q2) || ++t > tl) break;
        }
    } else {
        for (int t = 0; t <= tl; ++t) {
#pragma unroll
            for (int i = 0; i < V; ++i) { q0[i] = q1[i]; q1[i] = q2[i]; }
            if (!step(t, q0, q1, q2)) break;
        }
    }
    if constexpr (TMA) {
        if (*s_timeout) {
            // give copies still in flight a bounded chance to land before exit
            for (int t = consumed + 1; t <= issued_hi; ++t) mbar_wait_bounded(&full[stage(t)], parity(t));
        }
    }
    return (uint32_t)(issued_hi + 1);
}

// Pass A's last-CTA step: alpha_k = rz / pq, or BREAKDOWN.
template <typename SP>
__device__ __forceinline__ void passa_finish(SP st, double pq, bool tmo) {
    st->pq = pq;
    st->pending = 0;
    st->replace = 0;
    if (!(pq > 0.0) || !isfinite(pq)) { st->done = 1; st->status = GBPCG_BREAKDOWN; }
    else st->alpha = st->rz / pq;
    if (tmo) { st->done = 1; st->status = GBPCG_TIMEOUT; st->replace = 0; }
}

// Pass B's last-CTA step: beta_k, the convergence test and the residual-
// replacement trigger.
template <typename SP>
__device__ __forceinline__ void passb_finish(SP st, int it, double rr, double rz, bool tmo) {
    st->it = it + 1;
    st->rr = rr;
    st->pending = 1;
    if (!isfinite(rr) || !isfinite(rz) || !(rz > 0.0)) { st->done = 1; st->status = GBPCG_BREAKDOWN; }
    else if (rr <= st->tol2 * st->bb || rr <= kReplaceDrop2 * st->rr_rep) {
        // flush d into x and recompute r = b - A x in FP64 before deciding
        // (the replacement pass sets beta and the flags); 2 marks a
        // confirmation of convergence
        st->replace = rr <= st->tol2 * st->bb ? 2 : 1;
    } else if (it + 1 >= st->maxit) { st->done = 1; st->status = GBPCG_NOT_CONVERGED; }
    else { st->beta = rz / st->rz; st->rz = rz; }
    if (tmo) { st->done = 1; st->status = GBPCG_TIMEOUT; st->replace = 0; }
}

// Pass R's last-CTA step: the convergence test and the replacement trigger
// on the recursive residual (beta is formed after the preconditioner).
template <typename SP>
__device__ __forceinline__ void passr_finish(SP st, int it, double rr, bool tmo) {
    st->it = it + 1;
    st->rr = rr;
    st->pending = 1;
    if (!isfinite(rr)) { st->done = 1; st->status = GBPCG_BREAKDOWN; }
    else if (rr <= st->tol2 * st->bb || rr <= kReplaceDrop2 * st->rr_rep) st->replace = rr <= st->tol2 * st->bb ? 2 : 1;
    else if (it + 1 >= st->maxit) { st->done = 1; st->status = GBPCG_NOT_CONVERGED; }
    if (tmo) { st->done = 1; st->status = GBPCG_TIMEOUT; st->replace = 0; }
}

template <typename T, int TX, int TY, int S, int KIND, bool TMA, typename Op, bool ZFILL = false>
__global__ void __launch_bounds__(TX / (16 / sizeof(T)) * TY)
    zmarch_kernel(const __grid_constant__ PassMaps maps, const PassArgs a, const Op op) {
    using G = Geometry<T, TX, TY, KIND>;
    using TC = CenterT<T, KIND>;
    constexpr int NT = G::NT, NV = G::NV;

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ int s_timeout;

    SolveState *st = a.st;
    if constexpr (KIND == K_PASSA || KIND == K_PASSB || KIND == K_PASSR) {
        if (st->done) return;  // uniform across the grid
    }
    MarchScalars sc = read_scalars<KIND>(st);
    if constexpr (KIND == K_STENCIL) sc.alpha = a.scale;
    const int it = sc.it;

    int sh0 = 0, sh1 = 0, so0 = 0;
    if constexpr (KIND == K_PASSA) { sh1 = (it + 1) & 1; so0 = it & 1; }
    if constexpr (KIND == K_PASSB || KIND == K_PASSR) sh0 = it & 1;
    MarchIO<T, KIND> io;
    // selects between fixed parameter slots: a run-time index into the
    // kernel's parameter arrays would copy them to local memory in every thread
    io.H0 = static_cast<const T *>(sh0 ? a.h0[1] : a.h0[0]);
    io.H1 = static_cast<const T *>(sh1 ? a.h1[1] : a.h1[0]);
    io.C0 = static_cast<const TC *>(a.c0);
    io.O0 = static_cast<T *>(so0 ? a.o0[1] : a.o0[0]);
    io.O1 = static_cast<TC *>(a.o1);
    io.M0 = sh0 ? &maps.h0[1] : &maps.h0[0];
    io.M1 = sh1 ? &maps.h1[1] : &maps.h1[0];
    io.MC = &maps.c0;
    io.l2hint = a.l2hint != 0;

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tile = blockIdx.x;
    const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
    int k0, k1;  // this CTA's planes [k0, k1): part blockIdx.y % zparts of chunk blockIdx.y / zparts
    {
        const int parts = max(a.zparts, 1);
        const int c = (int)blockIdx.y / parts, part = (int)blockIdx.y - c * parts;
        const int c0 = c * a.zchunk, c1 = min(nz, c0 + a.zchunk), sub = (a.zchunk + parts - 1) / parts;
        k0 = min(c1, c0 + part * sub);
        k1 = min(c1, k0 + sub);
    }

    float acc[NV > 0 ? NV : 1];
#pragma unroll
    for (int i = 0; i < (NV > 0 ? NV : 1); ++i) acc[i] = 0.f;

    if (threadIdx.x == 0) {
        s_timeout = 0;
        if constexpr (TMA) {
            for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
            fence_mbar_init();
        }
    }
    __syncthreads();

    march_tile<T, TX, TY, S, KIND, TMA, Op, ZFILL>(smem, full, &s_timeout, 0u, io, op, nx, ny, nz, x0, y0, k0, k1,
                                                   sc, acc);
    if constexpr (TMA) {
        if (s_timeout && threadIdx.x == 0) atomicExch(&st->timeout, 1);
    }

    if constexpr (NV > 0) {
        double part[NV], tot[NV];
        block_sum<NV, NT>(acc, part);
        if (grid_sum_last<NV, NT>(part, a.partials, &st->ticket[KIND], tot) && threadIdx.x == 0) {
            __threadfence();
            const bool tmo = atomicAdd(&st->timeout, 0) != 0;
            if constexpr (KIND == K_PASSA) passa_finish(st, tot[0], tmo);
            else if constexpr (KIND == K_PASSR) passr_finish(st, it, tot[0], tmo);
            else passb_finish(st, it, tot[0], tot[NV - 1], tmo);
            if (a.use_cond) {
                cudaGraphSetConditional(a.cond, st->done ? 0u : 1u);
                cudaGraphSetConditional(a.cond_replace, st->replace ? 1u : 0u);
            }
        }
    }
}

}  // namespace gb
