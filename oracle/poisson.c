/*
 * Oracle: the Poisson solve of the gravity step, by the textbook conjugate gradient (CG)
 * and by the preconditioned pipelined conjugate gradient (PPCG) that Sec. 2.3 puts in
 * its place (TEST INFRASTRUCTURE ONLY).
 *
 * Linear system.  A x = b on a box of nx*ny*nz cells, vectors indexed i + nx (j + ny k).
 * A = 6 I - N, where (N v)_c sums v over the face neighbours of cell c that lie inside the
 * box: the 7-point discrete Laplacian times -h^2 with homogeneous Dirichlet boundaries
 * (the caller folds the boundary values and h^2 4 pi G rho into b).  A is symmetric
 * positive definite.
 *
 * Preconditioner (Sec. 2.3).  u = M^-1 r is the 7-point stencil with centre 13/12 and the
 * six face neighbours 1/6 (the "incomplete Poisson" approximate inverse K K^T,
 * K = I - L D^-1, with the fill-in outside the 7-point pattern dropped, written for
 * 3-D).  The stencil is the same in every cell; a neighbour outside the box contributes
 * nothing.  PRECOND_NONE makes M^-1 the identity, which turns PPCG into pipelined CG.
 *
 * Convergence measure (Eq. 3): eps_i = sqrt((r_i . u_i) / (r_0 . u_0)) with u_i = M^-1 r_i
 * (u = r without a preconditioner).  Both solvers stop at the first i >= 1 with
 * eps_i <= tol, or after maxit iterations; eps[0..iters] receives the history and
 * *iters the number of updates of x made.  When r_0 . u_0 = 0 the initial guess solves
 * the system: *iters = 0 and eps[0] = 0.
 *
 * or_cg is the preconditioned CG of Hestenes & Stiefel (two inner products per
 * iteration, each needed before the next vector update).  or_ppcg is the preconditioned
 * pipelined CG of Ghysels & Vanroose (2014), their Algorithm 4, the solver Sec. 2.3
 * adopts: the two inner products of an iteration are computed together and do not wait
 * on the preconditioner and operator applications of the same iteration, at the price of
 * four extra recurrences (z = A q, q = M^-1 s, s = A p, w = A u in exact arithmetic).
 * In exact arithmetic both produce the same iterates.
 *
 * Every loop is a plain sequential loop in FP64; inner products sum in index order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* sum of v over the face neighbours of cell (i,j,k) inside the box */
static double nb_sum(const double *v, int nx, int ny, int nz, int i, int j, int k)
{
    int64_t sy = nx, sz = (int64_t)nx * ny;
    int64_t c = i + sy * j + sz * k;
    double s = 0.0;
    if (i > 0) s += v[c - 1];
    if (i < nx - 1) s += v[c + 1];
    if (j > 0) s += v[c - sy];
    if (j < ny - 1) s += v[c + sy];
    if (k > 0) s += v[c - sz];
    if (k < nz - 1) s += v[c + sz];
    return s;
}

void or_poisson_apply_A(int nx, int ny, int nz, const double *x, double *y)
{
    int64_t c = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++, c++)
                y[c] = 6.0 * x[c] - nb_sum(x, nx, ny, nz, i, j, k);
}

void or_poisson_apply_Minv(int nx, int ny, int nz, int precond, const double *r, double *u)
{
    int64_t n = (int64_t)nx * ny * nz, c = 0;
    if (precond == OR_PRECOND_NONE) {
        memcpy(u, r, (size_t)n * sizeof(double));
        return;
    }
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++, c++)
                u[c] = (13.0 / 12.0) * r[c] + nb_sum(r, nx, ny, nz, i, j, k) / 6.0;
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t c = 0; c < n; c++) s += a[c] * b[c];
    return s;
}

static int check_args(int nx, int ny, int nz, int precond, const double *b, double *x, double tol, int maxit,
                      double *eps, int *iters)
{
    if (nx < 1 || ny < 1 || nz < 1 || !b || !x || !eps || !iters || maxit < 0 || !(tol >= 0.0)) return OR_EINVAL;
    if (precond != OR_PRECOND_NONE && precond != OR_PRECOND_IP) return OR_EINVAL;
    return OR_OK;
}

/* r = b - A x */
static void residual(int nx, int ny, int nz, const double *b, const double *x, double *r)
{
    int64_t n = (int64_t)nx * ny * nz;
    or_poisson_apply_A(nx, ny, nz, x, r);
    for (int64_t c = 0; c < n; c++) r[c] = b[c] - r[c];
}

int or_cg(int nx, int ny, int nz, int precond, const double *b, double *x, double tol, int maxit,
          double *eps, int *iters)
{
    int st = check_args(nx, ny, nz, precond, b, x, tol, maxit, eps, iters);
    if (st != OR_OK) return st;
    int64_t n = (int64_t)nx * ny * nz;
    double *r = malloc(n * sizeof(double)), *u = malloc(n * sizeof(double));
    double *p = malloc(n * sizeof(double)), *s = malloc(n * sizeof(double));
    residual(nx, ny, nz, b, x, r);
    or_poisson_apply_Minv(nx, ny, nz, precond, r, u);
    double gamma0 = dot(n, r, u), gamma = gamma0;
    *iters = 0;
    eps[0] = gamma0 > 0.0 ? 1.0 : 0.0;
    st = gamma0 > 0.0 ? OR_ENOCONV : OR_OK;
    memcpy(p, u, n * sizeof(double));
    for (int i = 0; i < maxit && gamma0 > 0.0; i++) {
        or_poisson_apply_A(nx, ny, nz, p, s);          /* s = A p */
        double ps = dot(n, p, s);
        if (!(ps > 0.0)) { st = OR_EBREAKDOWN; break; }
        double alpha = gamma / ps;
        for (int64_t c = 0; c < n; c++) {
            x[c] += alpha * p[c];
            r[c] -= alpha * s[c];
        }
        or_poisson_apply_Minv(nx, ny, nz, precond, r, u);
        double gnew = dot(n, r, u);
        *iters = i + 1;
        eps[i + 1] = sqrt(gnew / gamma0);
        if (eps[i + 1] <= tol) { st = OR_OK; break; }
        double beta = gnew / gamma;
        gamma = gnew;
        for (int64_t c = 0; c < n; c++) p[c] = u[c] + beta * p[c];
    }
    free(r); free(u); free(p); free(s);
    return st;
}

int or_ppcg(int nx, int ny, int nz, int precond, const double *b, double *x, double tol, int maxit,
            double *eps, int *iters)
{
    int st = check_args(nx, ny, nz, precond, b, x, tol, maxit, eps, iters);
    if (st != OR_OK) return st;
    int64_t n = (int64_t)nx * ny * nz;
    double *v = malloc(10 * n * sizeof(double));
    double *r = v, *u = v + n, *w = v + 2 * n, *m = v + 3 * n, *nn = v + 4 * n;
    double *z = v + 5 * n, *q = v + 6 * n, *s = v + 7 * n, *p = v + 8 * n;
    residual(nx, ny, nz, b, x, r);                    /* r_0 = b - A x_0 */
    or_poisson_apply_Minv(nx, ny, nz, precond, r, u); /* u_0 = M^-1 r_0 */
    or_poisson_apply_A(nx, ny, nz, u, w);             /* w_0 = A u_0 */
    double gamma0 = 0.0, gamma_old = 0.0, alpha_old = 0.0;
    *iters = 0;
    st = OR_ENOCONV;
    for (int i = 0;; i++) {
        double gamma = dot(n, r, u), delta = dot(n, w, u);
        if (i == 0) {
            gamma0 = gamma;
            eps[0] = gamma0 > 0.0 ? 1.0 : 0.0;
            if (!(gamma0 > 0.0)) { st = OR_OK; break; }
        } else {
            eps[i] = sqrt(gamma / gamma0);
            if (eps[i] <= tol) { st = OR_OK; break; }
        }
        if (i == maxit) break;
        or_poisson_apply_Minv(nx, ny, nz, precond, w, m);  /* m_i = M^-1 w_i */
        or_poisson_apply_A(nx, ny, nz, m, nn);             /* n_i = A m_i */
        double alpha, beta;
        if (i == 0) {
            beta = 0.0;
            alpha = gamma / delta;
        } else {
            beta = gamma / gamma_old;
            alpha = gamma / (delta - beta * gamma / alpha_old);
        }
        if (!(alpha > 0.0) || !isfinite(alpha)) { st = OR_EBREAKDOWN; break; }
        for (int64_t c = 0; c < n; c++) {
            if (i == 0) {
                z[c] = nn[c]; q[c] = m[c]; s[c] = w[c]; p[c] = u[c];
            } else {
                z[c] = nn[c] + beta * z[c];
                q[c] = m[c] + beta * q[c];
                s[c] = w[c] + beta * s[c];
                p[c] = u[c] + beta * p[c];
            }
            x[c] += alpha * p[c];
            r[c] -= alpha * s[c];
            u[c] -= alpha * q[c];
            w[c] -= alpha * z[c];
        }
        gamma_old = gamma;
        alpha_old = alpha;
        *iters = i + 1;
    }
    free(v);
    return st;
}
