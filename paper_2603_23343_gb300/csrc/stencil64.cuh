// FP64 evaluation of the 7-point operator at one grid point, shared by the
// FP64 stencil entry point, the solver's residuals b - A x and the outer
// residual of mixed-precision refinement.
//
// Operator (the seven-point stencil of Sec. VI / VII): (A u)_c = sum over the six faces f of
// w_f (u_c - u_f), with zero Dirichlet values outside the grid; w_f = 1/h_d^2
// for constant coefficients, and for per-block coefficients 1/h_d^2 times the
// block's k inside a block and times the harmonic mean of the two blocks' k
// on a face between blocks (the domain boundary keeps the block's own k).
//
// GB300 executes FP64 arithmetic at a small fraction of its FP32 rate, so
// these helpers spend FP64 operations only where the accuracy of b - A x
// needs them: the differences of nearby values and their weighted sum.
#pragma once

#include "common.cuh"

namespace gb {

struct Coef64 {
    double cx, cy, cz;  // 1/h_d^2 (times the operator scale)
    const float *kb;    // per-block coefficients, x fastest (unused for constant coefficients)
    int kbx, kby, kbz;  // block edges in grid points
};

// The centre value and its six neighbours (zero outside the grid).
struct Nbr64 {
    double c, xm, xp, ym, yp, zm, zp;
};

// CG: load through L2 only (ld.global.cg), for x written earlier in the same
// launch by other SMs; otherwise the read-only path (ld.global.nc), which is
// valid only for data no thread writes during the launch.
template <typename X, bool CG = false>
__device__ __forceinline__ Nbr64 load_nbr64(const X *__restrict__ x, int64_t g, int i, int j, int k, int nx, int ny,
                                            int nz) {
    const int64_t pl = (int64_t)nx * ny;
    auto L = [&](int64_t o) { return CG ? (double)__ldcg(x + o) : (double)__ldg(x + o); };
    Nbr64 u;
    u.c = L(g);
    u.xm = i > 0 ? L(g - 1) : 0.0;
    u.xp = i < nx - 1 ? L(g + 1) : 0.0;
    u.ym = j > 0 ? L(g - nx) : 0.0;
    u.yp = j < ny - 1 ? L(g + nx) : 0.0;
    u.zm = k > 0 ? L(g - pl) : 0.0;
    u.zp = k < nz - 1 ? L(g + pl) : 0.0;
    return u;
}

// Face weights {x-, x+, y-, y+, z-, z+} at grid point (i, j, k).
template <bool BLOCK>
__device__ __forceinline__ void face_weights64(double w[6], int i, int j, int k, int nx, int ny, int nz,
                                               const Coef64 &cf) {
    w[0] = w[1] = cf.cx;
    w[2] = w[3] = cf.cy;
    w[4] = w[5] = cf.cz;
    if constexpr (BLOCK) {
        const int nbx = (nx + cf.kbx - 1) / cf.kbx, nby = (ny + cf.kby - 1) / cf.kby;
        auto K = [&](int p, int q, int r) { return (double)__ldg(cf.kb + ((int64_t)r * nby + q) * nbx + p); };
        auto hm = [](double u, double v) { return 2.0 * u * v / (u + v); };
        const int bx = i / cf.kbx, by = j / cf.kby, bz = k / cf.kbz;
        const int ix = i - bx * cf.kbx, iy = j - by * cf.kby, iz = k - bz * cf.kbz;
        const double kc = K(bx, by, bz);
        w[0] = cf.cx * ((ix == 0 && i > 0) ? hm(kc, K(bx - 1, by, bz)) : kc);
        w[1] = cf.cx * ((ix == cf.kbx - 1 && i < nx - 1) ? hm(kc, K(bx + 1, by, bz)) : kc);
        w[2] = cf.cy * ((iy == 0 && j > 0) ? hm(kc, K(bx, by - 1, bz)) : kc);
        w[3] = cf.cy * ((iy == cf.kby - 1 && j < ny - 1) ? hm(kc, K(bx, by + 1, bz)) : kc);
        w[4] = cf.cz * ((iz == 0 && k > 0) ? hm(kc, K(bx, by, bz - 1)) : kc);
        w[5] = cf.cz * ((iz == cf.kbz - 1 && k < nz - 1) ? hm(kc, K(bx, by, bz + 1)) : kc);
    }
}

// FP64 face weights of every coefficient block, 9 doubles per block (x
// fastest): {cx k, cx k_x-, cx k_x+, cy k, cy k_y-, cy k_y+, cz k, cz k_z-,
// cz k_z+}, with k the block's coefficient and k_f the harmonic mean with the
// neighbouring block across face f (k itself on the domain boundary) -- the
// values face_weights64<true> derives per point, computed once per block so
// that the per-point FP64 divisions disappear.
constexpr int kTab64 = 9;

__device__ __forceinline__ void face_table64_block(double *t, const float *__restrict__ kb, int bx, int by, int bz,
                                                   int nbx, int nby, int nbz, const Coef64 &cf) {
    auto K = [&](int p, int q, int r) { return (double)__ldg(kb + ((int64_t)r * nby + q) * nbx + p); };
    auto hm = [](double u, double v) { return 2.0 * u * v / (u + v); };
    const double kc = K(bx, by, bz);
    t[0] = cf.cx * kc;
    t[1] = cf.cx * (bx > 0 ? hm(kc, K(bx - 1, by, bz)) : kc);
    t[2] = cf.cx * (bx < nbx - 1 ? hm(kc, K(bx + 1, by, bz)) : kc);
    t[3] = cf.cy * kc;
    t[4] = cf.cy * (by > 0 ? hm(kc, K(bx, by - 1, bz)) : kc);
    t[5] = cf.cy * (by < nby - 1 ? hm(kc, K(bx, by + 1, bz)) : kc);
    t[6] = cf.cz * kc;
    t[7] = cf.cz * (bz > 0 ? hm(kc, K(bx, by, bz - 1)) : kc);
    t[8] = cf.cz * (bz < nbz - 1 ? hm(kc, K(bx, by, bz + 1)) : kc);
}

// Face weights at (i, j, k) from the block table: a point on a block face
// takes the face's entry, every other point the block's own.  Equal, value
// for value, to face_weights64<true>: a point with ix == 0 has i > 0 exactly
// when bx > 0, and one with ix == kbx - 1 has i < nx - 1 exactly when
// bx < nbx - 1.
__device__ __forceinline__ void face_weights64_tab(double w[6], int i, int j, int k, int nx, int ny,
                                                   const double *__restrict__ tab, const Coef64 &cf) {
    const int nbx = (nx + cf.kbx - 1) / cf.kbx, nby = (ny + cf.kby - 1) / cf.kby;
    const int bx = i / cf.kbx, by = j / cf.kby, bz = k / cf.kbz;
    const int ix = i - bx * cf.kbx, iy = j - by * cf.kby, iz = k - bz * cf.kbz;
    const double *t = tab + kTab64 * (((int64_t)bz * nby + by) * nbx + bx);
    w[0] = __ldg(t + (ix == 0 ? 1 : 0));
    w[1] = __ldg(t + (ix == cf.kbx - 1 ? 2 : 0));
    w[2] = __ldg(t + (iy == 0 ? 4 : 3));
    w[3] = __ldg(t + (iy == cf.kby - 1 ? 5 : 3));
    w[4] = __ldg(t + (iz == 0 ? 7 : 6));
    w[5] = __ldg(t + (iz == cf.kbz - 1 ? 8 : 6));
}

// (A u)_c.  With equal weights on opposite faces (constant coefficients) the
// pairs are taken together, w ((2 u_c - u_-) - u_+): ten FP64 operations
// instead of twelve, each difference still exact for nearby values.
template <bool BLOCK>
__device__ __forceinline__ double apply64(const Nbr64 &u, const double w[6]) {
    if constexpr (!BLOCK) {
        const double c2 = u.c + u.c;
        double q = w[0] * ((c2 - u.xm) - u.xp);
        q = fma(w[2], (c2 - u.ym) - u.yp, q);
        return fma(w[4], (c2 - u.zm) - u.zp, q);
    } else {
        double q = w[0] * (u.c - u.xm);
        q = fma(w[1], u.c - u.xp, q);
        q = fma(w[2], u.c - u.ym, q);
        q = fma(w[3], u.c - u.yp, q);
        q = fma(w[4], u.c - u.zm, q);
        return fma(w[5], u.c - u.zp, q);
    }
}

// Diagonal of A at the point, rounded to FP32 (the preconditioner D).
__device__ __forceinline__ float diag64(const double w[6]) {
    return (float)(((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]));
}

}  // namespace gb
