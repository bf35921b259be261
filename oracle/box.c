/*
 * Oracle: one Godunov step on a single uniform box of N^3 cells of size 1/N
 * (TEST INFRASTRUCTURE ONLY).
 *
 * The same scheme as hydro.c (MUSCL-Hancock, MinMod, HLLC or exact solver, FP64), written
 * as plain loops over a cell-indexed grid: cell (i,j,k) at index i + N (j + N k).  Ghost
 * cells two deep follow the same boundary rule as the octree (periodic wrap, or outflow
 * clamping of the integer coordinate), and every ghost cell's slopes and predicted state
 * are computed from its own (clamped) neighbours, exactly as a stencil cell of the
 * octree oracle.  For power-of-two N it is the octree oracle's step on a complete tree.
 * Used for batches of independent boxes whose sizes need not be powers of two.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

#define NV OR_NVAR

static int64_t bc_index(int64_t c, int64_t n, int periodic)
{
    if (c >= 0 && c < n) return c;
    if (periodic) return ((c % n) + n) % n;
    return c < 0 ? 0 : n - 1;
}

static void predict_cell(const double *W, double D[3][NV], double gamma, double lam, double *Wt)
{
    double r = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
    double h = 0.5 * lam;
    Wt[0] = r - h * (u * D[0][0] + r * D[0][1] + v * D[1][0] + r * D[1][2] + w * D[2][0] + r * D[2][3]);
    Wt[1] = u - h * (u * D[0][1] + v * D[1][1] + w * D[2][1] + D[0][4] / r);
    Wt[2] = v - h * (u * D[0][2] + v * D[1][2] + w * D[2][2] + D[1][4] / r);
    Wt[3] = w - h * (u * D[0][3] + v * D[1][3] + w * D[2][3] + D[2][4] / r);
    Wt[4] = p - h * (u * D[0][4] + v * D[1][4] + w * D[2][4] + gamma * p * (D[0][1] + D[1][2] + D[2][3]));
}

int or_box_courant(int64_t N, const or_params *p, const double *u, double *dt)
{
    int64_t nc = N * N * N;
    double dx = 1.0 / (double)N, best = INFINITY;
    for (int64_t c = 0; c < nc; c++) {
        double U[NV], W[NV];
        for (int v = 0; v < NV; v++) U[v] = u[(int64_t)v * nc + c];
        or_cons_to_prim(U, p->gamma, p->rho_floor, p->p_floor, W);
        double cs = sqrt(p->gamma * W[4] / W[0]);
        double sig = (fabs(W[1]) + cs) + (fabs(W[2]) + cs) + (fabs(W[3]) + cs);
        double r = dx / sig;
        if (r < best) best = r;
    }
    *dt = p->cfl * best;
    return OR_OK;
}

/* u, u_new: [5][N^3].  bc[6] as for the octree.  dt given by the caller. */
int or_box_step(int64_t N, const int32_t *bc, const or_params *p, const double *u, double *u_new, double dt)
{
    const int64_t E = N + 4, nc = N * N * N, ne = E * E * E;   /* extended grid, index i+2 */
    const int per[3] = { bc[0] == OR_BC_PERIODIC, bc[2] == OR_BC_PERIODIC, bc[4] == OR_BC_PERIODIC };
    const double lam = dt * (double)N;
    double *W = malloc(sizeof(double) * NV * ne);
    double *Wf = malloc(sizeof(double) * 3 * 2 * NV * ne);      /* [d][side][v][cell] */
    int st = OR_OK;
#define XI(i, j, k) ((i) + E * ((j) + E * (k)))
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < E; k++)
        for (int64_t j = 0; j < E; j++)
            for (int64_t i = 0; i < E; i++) {
                int64_t ci = bc_index(i - 2, N, per[0]), cj = bc_index(j - 2, N, per[1]), ck = bc_index(k - 2, N, per[2]);
                int64_t c = ci + N * (cj + N * ck);
                double U[NV], Wc[NV];
                for (int v = 0; v < NV; v++) U[v] = u[(int64_t)v * nc + c];
                or_cons_to_prim(U, p->gamma, p->rho_floor, p->p_floor, Wc);
                for (int v = 0; v < NV; v++) W[(int64_t)v * ne + XI(i, j, k)] = Wc[v];
            }
    const int64_t step[3] = { 1, E, E * E };
    #pragma omp parallel for schedule(static)
    for (int64_t k = 1; k < E - 1; k++)
        for (int64_t j = 1; j < E - 1; j++)
            for (int64_t i = 1; i < E - 1; i++) {
                int64_t s = XI(i, j, k);
                double Wc[NV], D[3][NV], Wt[NV];
                for (int v = 0; v < NV; v++) Wc[v] = W[(int64_t)v * ne + s];
                for (int d = 0; d < 3; d++)
                    for (int v = 0; v < NV; v++)
                        D[d][v] = or_slope(p->limiter, W[(int64_t)v * ne + s] - W[(int64_t)v * ne + s - step[d]],
                                           W[(int64_t)v * ne + s + step[d]] - W[(int64_t)v * ne + s]);
                predict_cell(Wc, D, p->gamma, lam, Wt);
                for (int d = 0; d < 3; d++)
                    for (int side = 0; side < 2; side++) {
                        double *o = Wf + ((int64_t)(d * 2 + side) * NV) * ne;
                        for (int v = 0; v < NV; v++)
                            o[(int64_t)v * ne + s] = side ? Wt[v] + 0.5 * D[d][v] : Wt[v] - 0.5 * D[d][v];
                        if (o[s] < p->rho_floor) o[s] = p->rho_floor;
                        if (o[(int64_t)4 * ne + s] < p->p_floor) o[(int64_t)4 * ne + s] = p->p_floor;
                    }
            }
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; k++)
        for (int64_t j = 0; j < N; j++)
            for (int64_t i = 0; i < N; i++) {
                int64_t s = XI(i + 2, j + 2, k + 2);
                double dU[NV] = { 0, 0, 0, 0, 0 };
                for (int d = 0; d < 3; d++) {
                    int perm[3] = { d + 1, d == 0 ? 2 : 1, d == 2 ? 2 : 3 };
                    for (int side = 0; side < 2; side++) {
                        int64_t n = side ? s + step[d] : s - step[d];
                        int64_t a = side ? s : n, b = side ? n : s;
                        const double *L = Wf + ((int64_t)(d * 2 + 1) * NV) * ne, *R = Wf + ((int64_t)(d * 2 + 0) * NV) * ne;
                        double WL[NV], WR[NV], Fn[NV], F[NV];
                        WL[0] = L[a]; WR[0] = R[b];
                        for (int q = 0; q < 3; q++) { WL[1 + q] = L[(int64_t)perm[q] * ne + a]; WR[1 + q] = R[(int64_t)perm[q] * ne + b]; }
                        WL[4] = L[(int64_t)4 * ne + a]; WR[4] = R[(int64_t)4 * ne + b];
                        int rs = or_riemann_flux(WL, WR, p, Fn);
                        if (rs != OR_OK) {
                            #pragma omp critical
                            { if (st == OR_OK) st = rs; }
                        }
                        F[0] = Fn[0]; F[4] = Fn[4];
                        for (int q = 0; q < 3; q++) F[perm[q]] = Fn[1 + q];
                        for (int v = 0; v < NV; v++) dU[v] = side ? dU[v] - F[v] : dU[v] + F[v];
                    }
                }
                int64_t c = i + N * (j + N * k);
                for (int v = 0; v < NV; v++) u_new[(int64_t)v * nc + c] = u[(int64_t)v * nc + c] + lam * dU[v];
            }
#undef XI
    free(W);
    free(Wf);
    return st;
}
