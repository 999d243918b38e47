/*
 * FP64 CPU oracle for the Jacobi-preconditioned conjugate-gradient solver of
 * arxiv 2603.23343 ("Numerical Kernels on a Spatial Accelerator: A Study of
 * Tenstorrent Wormhole"), Sec. VII: a 3D seven-point finite-difference
 * operator with zero Dirichlet boundaries, applied matrix-free, Jacobi
 * (diagonal) preconditioning, conjugate-gradient iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Everything is plain loops in double precision, written to be checked
 * against the mathematics by eye:
 *   grid     interior points (i, j, k), 0 <= i < nx, fastest; index
 *            (k*ny + j)*nx + i; spacing h_d = 1/(n_d + 1) on the unit cube;
 *            u = 0 on every point outside the interior (zero Dirichlet).
 *   Poisson  (A u)_c = sum_d (2 u_c - u_{c-e_d} - u_{c+e_d}) / h_d^2
 *            (the seven-point stencil of Sec. VI / VII; for a cube this is
 *            (6 u_c - sum of the six neighbours) / h^2).
 *   var-k    (A u)_c = sum_d sum_{+-} k_f (u_c - u_nb) / h_d^2, k constant
 *            on blocks of kbx*kby*kbz points; k_f is the harmonic mean of
 *            the two cells' k on an interior face and the cell's own k on a
 *            boundary face (ghost value 0 one spacing away).
 *   Jacobi   z = D^{-1} r with D the diagonal of A (Sec. VII: the
 *            preconditioner is an element-wise scaling).
 *   PCG      Hestenes-Stiefel preconditioned CG (Sec. VII composes the
 *            stencil, the dot product of Sec. V and the element-wise
 *            updates of Sec. IV into it).
 *
 * The paper gives no stencil scale, stopping norm or tolerance; the choices
 * above (1/h^2 scale, relative recursive 2-norm residual, harmonic-mean
 * faces) are the readings the whole project uses.
 *
 * Parallel loops (OpenMP, when compiled with it) only split independent
 * output points; every sum is taken in one fixed order (per-chunk partials
 * added in chunk order) so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 3
#define ORC_BREAKDOWN 4

#define IDX(i, j, k) ((((int64_t)(k)) * ny + (j)) * nx + (i))
#define SUM_CHUNK 4096

/* Threads the parallel loops use (1 without OpenMP); reported beside timings. */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
#else
int orc_threads(void) { return 1; }
#endif

static double inv_h2(int n) {
    double h = 1.0 / (double)(n + 1);
    return 1.0 / (h * h);
}

/* --------------------------------------------------------------- sums -- */

/* x . y, summed in chunks of SUM_CHUNK consecutive entries; chunk totals are
 * then added in chunk order (a fixed order, independent of threads). */
double orc_dot(int64_t n, const double *x, const double *y) {
    if (n <= 0) return 0.0;
    int64_t nc = (n + SUM_CHUNK - 1) / SUM_CHUNK;
    double *part = (double *)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t a = c * SUM_CHUNK, e = a + SUM_CHUNK < n ? a + SUM_CHUNK : n;
        double s = 0.0;
        for (int64_t i = a; i < e; ++i) s += x[i] * y[i];
        part[c] = s;
    }
    double s = 0.0;
    for (int64_t c = 0; c < nc; ++c) s += part[c];
    free(part);
    return s;
}

/* y <- alpha * x + y */
void orc_axpy(int64_t n, double alpha, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) y[i] = alpha * x[i] + y[i];
}

/* ----------------------------------------------------------- operators -- */

/* Seven-point Poisson operator, out = A u (u = 0 outside the interior). */
void orc_apply_poisson(int nx, int ny, int nz, const double *u, double *out) {
    const double cx = inv_h2(nx), cy = inv_h2(ny), cz = inv_h2(nz);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double c = u[IDX(i, j, k)];
                double xm = i > 0 ? u[IDX(i - 1, j, k)] : 0.0;
                double xp = i < nx - 1 ? u[IDX(i + 1, j, k)] : 0.0;
                double ym = j > 0 ? u[IDX(i, j - 1, k)] : 0.0;
                double yp = j < ny - 1 ? u[IDX(i, j + 1, k)] : 0.0;
                double zm = k > 0 ? u[IDX(i, j, k - 1)] : 0.0;
                double zp = k < nz - 1 ? u[IDX(i, j, k + 1)] : 0.0;
                out[IDX(i, j, k)] = cx * (2.0 * c - xm - xp) + cy * (2.0 * c - ym - yp) +
                                    cz * (2.0 * c - zm - zp);
            }
}

/* Coefficient of the cell holding point (i, j, k). */
static double kcell(const double *kb, int nbx, int nby, int kbx, int kby, int kbz, int i, int j,
                    int k) {
    return kb[((int64_t)(k / kbz) * nby + (j / kby)) * nbx + (i / kbx)];
}

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

/* Face coefficient between point c and its neighbour at offset (di,dj,dk);
 * the cell's own coefficient when the neighbour lies outside the grid. */
static double kface(const double *kb, int nx, int ny, int nz, int nbx, int nby, int kbx, int kby,
                    int kbz, int i, int j, int k, int di, int dj, int dk) {
    double kc = kcell(kb, nbx, nby, kbx, kby, kbz, i, j, k);
    int a = i + di, b = j + dj, c = k + dk;
    if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) return kc;
    return harmonic(kc, kcell(kb, nbx, nby, kbx, kby, kbz, a, b, c));
}

/* Variable-coefficient operator out = -div(k grad u), cell-centred finite
 * volumes on blocks of constant k. */
void orc_apply_varcoeff(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz,
                        const double *u, double *out) {
    const int nbx = (nx + kbx - 1) / kbx, nby = (ny + kby - 1) / kby;
    const double cx = inv_h2(nx), cy = inv_h2(ny), cz = inv_h2(nz);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double c = u[IDX(i, j, k)];
                double xm = i > 0 ? u[IDX(i - 1, j, k)] : 0.0;
                double xp = i < nx - 1 ? u[IDX(i + 1, j, k)] : 0.0;
                double ym = j > 0 ? u[IDX(i, j - 1, k)] : 0.0;
                double yp = j < ny - 1 ? u[IDX(i, j + 1, k)] : 0.0;
                double zm = k > 0 ? u[IDX(i, j, k - 1)] : 0.0;
                double zp = k < nz - 1 ? u[IDX(i, j, k + 1)] : 0.0;
#define KF(di, dj, dk) kface(kb, nx, ny, nz, nbx, nby, kbx, kby, kbz, i, j, k, di, dj, dk)
                double s = cx * (KF(-1, 0, 0) * (c - xm) + KF(1, 0, 0) * (c - xp)) +
                           cy * (KF(0, -1, 0) * (c - ym) + KF(0, 1, 0) * (c - yp)) +
                           cz * (KF(0, 0, -1) * (c - zm) + KF(0, 0, 1) * (c - zp));
                out[IDX(i, j, k)] = s;
            }
}

/* Diagonal of A (kb == NULL: Poisson). */
void orc_diag(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz, double *d) {
    const double cx = inv_h2(nx), cy = inv_h2(ny), cz = inv_h2(nz);
    const int nbx = kb ? (nx + kbx - 1) / kbx : 0, nby = kb ? (ny + kby - 1) / kby : 0;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (!kb) {
                    d[IDX(i, j, k)] = 2.0 * (cx + cy + cz);
                } else {
                    d[IDX(i, j, k)] = cx * (KF(-1, 0, 0) + KF(1, 0, 0)) +
                                      cy * (KF(0, -1, 0) + KF(0, 1, 0)) +
                                      cz * (KF(0, 0, -1) + KF(0, 0, 1));
                }
            }
#undef KF
}

/* out = A u for either operator. */
void orc_apply(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz,
               const double *u, double *out) {
    if (kb)
        orc_apply_varcoeff(nx, ny, nz, kb, kbx, kby, kbz, u, out);
    else
        orc_apply_poisson(nx, ny, nz, u, out);
}

/* r = b - A x */
void orc_residual(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz,
                  const double *b, const double *x, double *r) {
    int64_t n = (int64_t)nx * ny * nz;
    orc_apply(nx, ny, nz, kb, kbx, kby, kbz, x, r);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
}

/* ------------------------------------------------------------------ PCG -- */

/*
 * Preconditioned CG, Hestenes-Stiefel form, Jacobi preconditioner
 * (precond = 0) or none (precond = -1, z = r):
 *
 *   r = b - A x;  z = M^{-1} r;  p = z;  rz = r.z;  bn = ||b||
 *   if ||r||/bn <= tol: stop with 0 iterations
 *   repeat:  q = A p;  alpha = rz / (p.q);  x += alpha p;  r -= alpha q;
 *            it += 1;  stop if ||r||/bn <= tol or it == maxit
 *            z = M^{-1} r;  rz' = r.z;  beta = rz'/rz;  p = z + beta p;  rz = rz'
 *
 * b = 0 gives x = 0 and 0 iterations.  p.q <= 0 or a non-finite scalar is a
 * breakdown.  hist (length >= maxit+1, may be NULL) receives ||r_k||/||b||
 * for k = 0 .. iters.  Returns ORC_OK, ORC_NOT_CONVERGED or ORC_BREAKDOWN.
 */
int orc_pcg(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz, const double *b,
            double *x, double tol, int maxit, int precond, double *hist, int *iters_out,
            double *relres_out) {
    const int64_t n = (int64_t)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    int status = ORC_NOT_CONVERGED, it = 0;
    double rel = 0.0;

    orc_diag(nx, ny, nz, kb, kbx, kby, kbz, d);
    const double bn = sqrt(orc_dot(n, b, b));
    if (bn == 0.0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        if (hist) hist[0] = 0.0;
        status = ORC_OK;
        goto done;
    }
    orc_residual(nx, ny, nz, kb, kbx, kby, kbz, b, x, r);
    for (int64_t i = 0; i < n; ++i) z[i] = precond == 0 ? r[i] / d[i] : r[i];
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = orc_dot(n, r, z);
    rel = sqrt(orc_dot(n, r, r)) / bn;
    if (hist) hist[0] = rel;
    if (rel <= tol) {
        status = ORC_OK;
        goto done;
    }
    while (it < maxit) {
        orc_apply(nx, ny, nz, kb, kbx, kby, kbz, p, q);
        double pq = orc_dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rz / pq;
        orc_axpy(n, alpha, p, x);
        orc_axpy(n, -alpha, q, r);
        it += 1;
        rel = sqrt(orc_dot(n, r, r)) / bn;
        if (hist) hist[it] = rel;
        if (rel <= tol) {
            status = ORC_OK;
            break;
        }
        if (it == maxit) break;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) z[i] = precond == 0 ? r[i] / d[i] : r[i];
        double rz_new = orc_dot(n, r, z);
        double beta = rz_new / rz;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    free(r);
    free(z);
    free(p);
    free(q);
    free(d);
    return status;
}

/* ------------------------------------------------ general sparse (CSR) -- */

/* y = A x for A in compressed sparse row form: row i holds the entries
 * row_ptr[i] .. row_ptr[i+1]-1 with columns col[e] and values val[e];
 * y_i = sum over the row's entries of val[e] x[col[e]], in entry order. */
void orc_csr_apply(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, const double *x,
                   double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += val[e] * x[col[e]];
        y[i] = s;
    }
}

/* Jacobi-PCG for a CSR matrix: the iteration of orc_pcg (Sec. VII) with the
 * matrix-free operator replaced by orc_csr_apply and D by the matrix's
 * diagonal entries (summed when a row repeats its diagonal column). */
int orc_csr_pcg(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, const double *b,
                double *x, double tol, int maxit, double *hist, int *iters_out, double *relres_out) {
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    int status = ORC_NOT_CONVERGED, it = 0;
    double rel = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        d[i] = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] == i) d[i] += val[e];
    }
    const double bn = sqrt(orc_dot(n, b, b));
    if (bn == 0.0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        if (hist) hist[0] = 0.0;
        status = ORC_OK;
        goto done;
    }
    orc_csr_apply(n, row_ptr, col, val, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    for (int64_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = orc_dot(n, r, z);
    rel = sqrt(orc_dot(n, r, r)) / bn;
    if (hist) hist[0] = rel;
    if (rel <= tol) {
        status = ORC_OK;
        goto done;
    }
    while (it < maxit) {
        orc_csr_apply(n, row_ptr, col, val, p, q);
        double pq = orc_dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rz / pq;
        orc_axpy(n, alpha, p, x);
        orc_axpy(n, -alpha, q, r);
        it += 1;
        rel = sqrt(orc_dot(n, r, r)) / bn;
        if (hist) hist[it] = rel;
        if (rel <= tol) {
            status = ORC_OK;
            break;
        }
        if (it == maxit) break;
        for (int64_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
        double rz_new = orc_dot(n, r, z);
        double beta = rz_new / rz;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    free(r);
    free(z);
    free(p);
    free(q);
    free(d);
    return status;
}

/* ||b - A x|| / ||b|| evaluated in FP64 (every solve's result is checked with it). */
double orc_true_relres(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz,
                       const double *b, const double *x) {
    const int64_t n = (int64_t)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    orc_residual(nx, ny, nz, kb, kbx, kby, kbz, b, x, r);
    double rn = sqrt(orc_dot(n, r, r)), bn = sqrt(orc_dot(n, b, b));
    free(r);
    return bn > 0.0 ? rn / bn : rn;
}

/*
 * Iterative refinement (Wilkinson; Moler, J. ACM 14, 1967) around an inner
 * Jacobi-PCG solve, everything in FP64 here:
 *   r = b - A x;  while ||r||/||b|| > tol and step < max_outer:
 *       s = max|r|;  solve A d = r/s to relative tolerance inner_tol (d0 = 0);
 *       x += s d;  r = b - A x
 * Returns the number of outer steps; *relres_out = final ||r||/||b||.
 */
int orc_refine(int nx, int ny, int nz, const double *kb, int kbx, int kby, int kbz,
               const double *b, double *x, double tol, int max_outer, double inner_tol,
               int inner_maxit, double *relres_out, int *inner_iters_total) {
    const int64_t n = (int64_t)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *rs = (double *)malloc(sizeof(double) * (size_t)n);
    double *dd = (double *)malloc(sizeof(double) * (size_t)n);
    const double bn = sqrt(orc_dot(n, b, b));
    int step = 0, total = 0;
    double rel = 0.0;
    orc_residual(nx, ny, nz, kb, kbx, kby, kbz, b, x, r);
    rel = bn > 0.0 ? sqrt(orc_dot(n, r, r)) / bn : 0.0;
    while (rel > tol && step < max_outer) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s = fabs(r[i]) > s ? fabs(r[i]) : s;
        for (int64_t i = 0; i < n; ++i) {
            rs[i] = r[i] / s;
            dd[i] = 0.0;
        }
        int it = 0;
        double irel = 0.0;
        orc_pcg(nx, ny, nz, kb, kbx, kby, kbz, rs, dd, inner_tol, inner_maxit, 0, NULL, &it,
                &irel);
        total += it;
        orc_axpy(n, s, dd, x);
        orc_residual(nx, ny, nz, kb, kbx, kby, kbz, b, x, r);
        rel = sqrt(orc_dot(n, r, r)) / bn;
        step += 1;
    }
    if (relres_out) *relres_out = rel;
    if (inner_iters_total) *inner_iters_total = total;
    free(r);
    free(rs);
    free(dd);
    return step;
}
