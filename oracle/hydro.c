/*
 * Oracle: one Godunov step on the octree (TEST INFRASTRUCTURE ONLY).
 *
 * The paper names the steps (Table 1: godunov_fine, newdt_fine) but prints no scheme;
 * this file writes out the readings used throughout the project:
 *   - one global time step for every level (Sec. 2.3, the w(l+1) = w(l) "single time
 *     step" option next to Eq. 1);
 *   - per oct, a 6^3 ghosted stencil of level-l cells around the oct.  A stencil cell
 *     that does not exist at level l is interpolated from its level l-1 father C:
 *       U = U_C + sum_d s_d * 1/4 * minmod(U_C - U_{C-e_d}, U_{C+e_d} - U_C)
 *     on conserved variables, s_d = +1 for the upper child along d, -1 for the lower;
 *     a neighbour of C missing at level l-1 takes the value of the deepest existing
 *     cell containing it (injection);
 *   - boundaries: periodic wraps, outflow clamps the integer cell coordinate at the
 *     cell's own level (zero gradient);
 *   - MUSCL-Hancock in primitive variables (Toro 2009, Sec. 14.4): MinMod slopes of
 *     undivided differences (or, on request, the monotonized central limiter of van
 *     Leer 1977), the half-step predictor written out in or_predict below,
 *     face states W~ +- Delta/2 with rho and p floored;
 *   - Riemann problem at each face in the face-normal frame (HLLC or exact);
 *   - conservative FP64 update U += dt/dx * sum_d (F_{d,-} - F_{d,+});
 *     a face whose other side is a refined cell of the same level carries no flux at
 *     this level: the finer level supplies it (refluxing);
 *     a face whose other side is a coarse leaf (an interpolated stencil cell) is applied
 *     to the fine cell and its flux summed, over the four fine faces of that oct side,
 *     into a register that later corrects the coarse cell by
 *       U_C -/+= dt/dx_C * 1/4 * sum F   (minus when C lies on the low side of the face);
 *   - restriction: a refined cell becomes the mean of its eight children, level by
 *     level from the finest up;
 *   - CFL step (newdt_fine): dt = C_cfl * min over leaf cells of dx / sum_d (|u_d| + c).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define NV OR_NVAR
static double dx_of(int l) { return ldexp(1.0, -l); }

/* boundary at level l for a cell coordinate: wrap (periodic) or clamp (outflow) */
static int64_t bc_wrap_clamp(const or_tree *t, int axis, int l, int64_t c)
{
    int64_t n = (int64_t)1 << l;
    if (c >= 0 && c < n) return c;
    int face = 2 * axis + (c >= n ? 1 : 0);
    if (t->bc[face] == OR_BC_PERIODIC) return ((c % n) + n) % n;
    return c < 0 ? 0 : n - 1;
}

static int64_t cell_id(const or_tree *t, int l, int64_t X, int64_t Y, int64_t Z)
{
    int64_t o = or_lookup(t, l, X >> 1, Y >> 1, Z >> 1);
    return o < 0 ? -1 : o * 8 + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1);
}

static void load(const double *u, int64_t ncell, int64_t cid, double *U)
{
    for (int v = 0; v < NV; v++) U[v] = u[(int64_t)v * ncell + cid];
}

/* value used for a neighbour of an interpolated coarse cell: deepest existing cell at
   level <= l containing the level-l cell (X,Y,Z) (after the boundary rule at level l) */
static int coarse_value(const or_tree *t, const double *u, int l, int64_t X, int64_t Y, int64_t Z, double *U)
{
    X = bc_wrap_clamp(t, 0, l, X); Y = bc_wrap_clamp(t, 1, l, Y); Z = bc_wrap_clamp(t, 2, l, Z);
    for (int lev = l; lev >= 1; lev--) {
        int sh = l - lev;
        int64_t cid = cell_id(t, lev, X >> sh, Y >> sh, Z >> sh);
        if (cid >= 0) { load(u, t->noct * 8, cid, U); return OR_OK; }
    }
    return OR_EUNBALANCED;
}

/* Value of the level-l cell (X,Y,Z); returns its id, -1 if it was interpolated from its
   father, or -2 if even the father is missing (an unbalanced tree). */
static int64_t cell_value(const or_tree *t, const double *u, int l, int64_t X, int64_t Y, int64_t Z, double *U)
{
    X = bc_wrap_clamp(t, 0, l, X); Y = bc_wrap_clamp(t, 1, l, Y); Z = bc_wrap_clamp(t, 2, l, Z);
    int64_t cid = cell_id(t, l, X, Y, Z);
    if (cid >= 0) { load(u, t->noct * 8, cid, U); return cid; }
    int64_t CX = X >> 1, CY = Y >> 1, CZ = Z >> 1;
    int64_t C = cell_id(t, l - 1, CX, CY, CZ);
    if (C < 0) return -2;
    double UC[NV], Um[3][NV], Up[3][NV];
    load(u, t->noct * 8, C, UC);
    for (int d = 0; d < 3; d++) {
        int64_t P[3] = { CX, CY, CZ }, M[3] = { CX, CY, CZ };
        P[d] += 1; M[d] -= 1;
        if (coarse_value(t, u, l - 1, M[0], M[1], M[2], Um[d]) != OR_OK) return -2;
        if (coarse_value(t, u, l - 1, P[0], P[1], P[2], Up[d]) != OR_OK) return -2;
    }
    int64_t pos[3] = { X & 1, Y & 1, Z & 1 };
    for (int v = 0; v < NV; v++) {
        double r = UC[v];
        for (int d = 0; d < 3; d++) {
            double m = or_minmod(UC[v] - Um[d][v], Up[d][v] - UC[v]);
            r = r + (pos[d] ? 0.25 * m : -0.25 * m);
        }
        U[v] = r;
    }
    return -1;
}

#define S3(i, j, k) ((i) + 6 * ((j) + 6 * (k)))

int or_oct_stencil(const or_tree *t, const double *u, int64_t oct, double *stencil)
{
    int l = t->lvl[oct];
    for (int k = 0; k < 6; k++)
        for (int j = 0; j < 6; j++)
            for (int i = 0; i < 6; i++) {
                double U[NV];
                int64_t r = cell_value(t, u, l, 2 * (int64_t)t->ix[oct] - 2 + i, 2 * (int64_t)t->iy[oct] - 2 + j,
                                       2 * (int64_t)t->iz[oct] - 2 + k, U);
                if (r == -2) return OR_EUNBALANCED;
                for (int v = 0; v < NV; v++) stencil[v * 216 + S3(i, j, k)] = U[v];
            }
    return OR_OK;
}

/* MUSCL-Hancock half-step predictor (Toro 2009, Sec. 14.4) in primitive variables,
   with D[d][v] the undivided MinMod slope along d and lam = dt/dx. */
static void or_predict(const double *W, double D[3][NV], double gamma, double lam, double *Wt)
{
    double r = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
    double h = 0.5 * lam;
    Wt[0] = r - h * (u * D[0][0] + r * D[0][1] + v * D[1][0] + r * D[1][2] + w * D[2][0] + r * D[2][3]);
    Wt[1] = u - h * (u * D[0][1] + v * D[1][1] + w * D[2][1] + D[0][4] / r);
    Wt[2] = v - h * (u * D[0][2] + v * D[1][2] + w * D[2][2] + D[1][4] / r);
    Wt[3] = w - h * (u * D[0][3] + v * D[1][3] + w * D[2][3] + D[2][4] / r);
    Wt[4] = p - h * (u * D[0][4] + v * D[1][4] + w * D[2][4] + gamma * p * (D[0][1] + D[1][2] + D[2][3]));
}

typedef struct {
    double U[NV][216];                /* stencil, conserved */
    double W[NV][216];                /* stencil, primitive */
    double Wf[3][2][NV][216];         /* face states: [d][0] low face, [d][1] high face */
    int64_t cid[216];                 /* id of each stencil cell, -1 if interpolated */
} oct_work;

/* Godunov update of one oct's eight cells (all of them, refined or not: refined cells are
   overwritten by the restriction that follows). */
static int oct_update(const or_tree *t, const or_params *p, int64_t oct, const double *u_old, double *u_new,
                      double *reg, double dt, oct_work *wk)
{
    int l = t->lvl[oct];
    int64_t ncell = t->noct * 8;
    double lam = dt / dx_of(l);
    int st = OR_OK;
    for (int k = 0; k < 6; k++)
        for (int j = 0; j < 6; j++)
            for (int i = 0; i < 6; i++) {
                double U[NV];
                int64_t r = cell_value(t, u_old, l, 2 * (int64_t)t->ix[oct] - 2 + i, 2 * (int64_t)t->iy[oct] - 2 + j,
                                       2 * (int64_t)t->iz[oct] - 2 + k, U);
                if (r == -2) return OR_EUNBALANCED;
                wk->cid[S3(i, j, k)] = r;
                for (int v = 0; v < NV; v++) wk->U[v][S3(i, j, k)] = U[v];
            }
    for (int s = 0; s < 216; s++) {
        double U[NV], W[NV];
        for (int v = 0; v < NV; v++) U[v] = wk->U[v][s];
        or_cons_to_prim(U, p->gamma, p->rho_floor, p->p_floor, W);
        for (int v = 0; v < NV; v++) wk->W[v][s] = W[v];
    }
    const int step[3] = { 1, 6, 36 };
    for (int k = 1; k < 5; k++)
        for (int j = 1; j < 5; j++)
            for (int i = 1; i < 5; i++) {
                int s = S3(i, j, k);
                double W[NV], D[3][NV], Wt[NV];
                for (int v = 0; v < NV; v++) W[v] = wk->W[v][s];
                for (int d = 0; d < 3; d++)
                    for (int v = 0; v < NV; v++)
                        D[d][v] = or_slope(p->limiter, wk->W[v][s] - wk->W[v][s - step[d]],
                                           wk->W[v][s + step[d]] - wk->W[v][s]);
                or_predict(W, D, p->gamma, lam, Wt);
                for (int d = 0; d < 3; d++)
                    for (int side = 0; side < 2; side++) {
                        for (int v = 0; v < NV; v++)
                            wk->Wf[d][side][v][s] = side ? Wt[v] + 0.5 * D[d][v] : Wt[v] - 0.5 * D[d][v];
                        if (wk->Wf[d][side][0][s] < p->rho_floor) wk->Wf[d][side][0][s] = p->rho_floor;
                        if (wk->Wf[d][side][4][s] < p->p_floor) wk->Wf[d][side][4][s] = p->p_floor;
                    }
            }
    /* the oct's cells are stencil indices 2,3 on every axis */
    for (int c = 0; c < 8; c++) {
        int ci = 2 + (c & 1), cj = 2 + ((c >> 1) & 1), ck = 2 + ((c >> 2) & 1);
        int s = S3(ci, cj, ck);
        double dU[NV] = { 0, 0, 0, 0, 0 };
        for (int d = 0; d < 3; d++) {
            for (int side = 0; side < 2; side++) {
                int n = side ? s + step[d] : s - step[d];       /* neighbour across the face */
                int a = side ? s : n, b = side ? n : s;         /* left, right cells */
                double WL[NV], WR[NV], F[NV], Fn[NV];
                /* rotate to the face-normal frame: normal velocity first */
                int perm[3] = { d + 1, d == 0 ? 2 : 1, d == 2 ? 2 : 3 };
                WL[0] = wk->Wf[d][1][0][a]; WR[0] = wk->Wf[d][0][0][b];
                for (int q = 0; q < 3; q++) { WL[1 + q] = wk->Wf[d][1][perm[q]][a]; WR[1 + q] = wk->Wf[d][0][perm[q]][b]; }
                WL[4] = wk->Wf[d][1][4][a]; WR[4] = wk->Wf[d][0][4][b];
                int rs = or_riemann_flux(WL, WR, p, Fn);
                if (rs != OR_OK && st == OR_OK) st = rs;
                F[0] = Fn[0]; F[4] = Fn[4];
                for (int q = 0; q < 3; q++) F[perm[q]] = Fn[1 + q];
                int64_t ncid = wk->cid[n];
                if (ncid >= 0 && t->son[ncid] >= 0) continue;  /* refined neighbour: no flux here */
                for (int v = 0; v < NV; v++) dU[v] = side ? dU[v] - F[v] : dU[v] + F[v];
                (void)a; (void)b;
            }
        }
        int64_t cell = oct * 8 + c;
        for (int v = 0; v < NV; v++) u_new[(int64_t)v * ncell + cell] = u_old[(int64_t)v * ncell + cell] + lam * dU[v];
    }
    /* flux register: oct sides whose neighbours are interpolated (coarse leaf) cells */
    if (reg) {
        for (int f = 0; f < 6; f++) {
            int d = f / 2, side = f & 1;
            int64_t C = t->nbor[6 * oct + f];
            if (C < 0 || t->son[C] >= 0) continue;   /* outside an outflow boundary, or refined */
            double sum[NV] = { 0, 0, 0, 0, 0 };
            for (int c = 0; c < 8; c++) {
                int pc[3] = { c & 1, (c >> 1) & 1, (c >> 2) & 1 };
                if (pc[d] != side) continue;
                int s = S3(2 + pc[0], 2 + pc[1], 2 + pc[2]);
                int n = side ? s + step[d] : s - step[d];
                int a = side ? s : n, b = side ? n : s;
                double WL[NV], WR[NV], Fn[NV], F[NV];
                int perm[3] = { d + 1, d == 0 ? 2 : 1, d == 2 ? 2 : 3 };
                WL[0] = wk->Wf[d][1][0][a]; WR[0] = wk->Wf[d][0][0][b];
                for (int q = 0; q < 3; q++) { WL[1 + q] = wk->Wf[d][1][perm[q]][a]; WR[1 + q] = wk->Wf[d][0][perm[q]][b]; }
                WL[4] = wk->Wf[d][1][4][a]; WR[4] = wk->Wf[d][0][4][b];
                or_riemann_flux(WL, WR, p, Fn);
                F[0] = Fn[0]; F[4] = Fn[4];
                for (int q = 0; q < 3; q++) F[perm[q]] = Fn[1 + q];
                for (int v = 0; v < NV; v++) sum[v] += F[v];
            }
            for (int v = 0; v < NV; v++) reg[(oct * 6 + f) * NV + v] = sum[v];
        }
    }
    return st;
}

int or_level_update(const or_tree *t, const or_params *p, int level, const double *u_old, double *u_new,
                    double *reg, double dt)
{
    if (level < 1 || level > OR_MAXLEV) return OR_EINVAL;
    int st = OR_OK;
    int64_t o0 = t->lvl_off[level], o1 = t->lvl_off[level + 1];
    #pragma omp parallel
    {
        oct_work *wk = malloc(sizeof(oct_work));
        int lst = OR_OK;
        #pragma omp for schedule(static)
        for (int64_t o = o0; o < o1; o++) {
            int r = oct_update(t, p, o, u_old, u_new, reg, dt, wk);
            if (r != OR_OK && lst == OR_OK) lst = r;
        }
        #pragma omp critical
        { if (lst != OR_OK && (st == OR_OK || lst == OR_EUNBALANCED)) st = lst; }
        free(wk);
    }
    return st;
}

/* the Godunov update of octs [o0, o1) only (same arithmetic as or_level_update) */
int or_octs_update(const or_tree *t, const or_params *p, int64_t o0, int64_t o1, const double *u_old, double *u_new,
                   double *reg, double dt)
{
    int st = OR_OK;
    #pragma omp parallel
    {
        oct_work *wk = malloc(sizeof(oct_work));
        int lst = OR_OK;
        #pragma omp for schedule(static)
        for (int64_t o = o0; o < o1; o++) {
            int r = oct_update(t, p, o, u_old, u_new, reg, dt, wk);
            if (r != OR_OK && lst == OR_OK) lst = r;
        }
        #pragma omp critical
        { if (lst != OR_OK && st == OR_OK) st = lst; }
        free(wk);
    }
    return st;
}

int or_reflux_restrict(const or_tree *t, const or_params *p, int level, const double *reg, double *u_new, double dt)
{
    (void)p;
    int64_t ncell = t->noct * 8;
    double lam = dt / dx_of(level);
    int64_t o0 = t->lvl_off[level], o1 = t->lvl_off[level + 1];
    if (level >= t->levelmin && reg) {
        for (int64_t o = o0; o < o1; o++)
            for (int c = 0; c < 8; c++) {
                int64_t C = o * 8 + c;
                if (t->son[C] >= 0) continue;   /* only leaf cells are corrected */
                int64_t X[3] = { 2 * (int64_t)t->ix[o] + (c & 1), 2 * (int64_t)t->iy[o] + ((c >> 1) & 1),
                                 2 * (int64_t)t->iz[o] + ((c >> 2) & 1) };
                for (int f = 0; f < 6; f++) {
                    int d = f / 2, side = f & 1;
                    int64_t P[3] = { X[0], X[1], X[2] };
                    P[d] += side ? 1 : -1;
                    int64_t n = (int64_t)1 << level;
                    if (P[d] < 0 || P[d] >= n) {
                        if (t->bc[f] != OR_BC_PERIODIC) continue;   /* outflow boundary face */
                        P[d] = ((P[d] % n) + n) % n;
                    }
                    int64_t nb = cell_id(t, level, P[0], P[1], P[2]);
                    if (nb < 0 || t->son[nb] < 0) continue;
                    int64_t fo = t->son[nb];
                    int opp = 2 * d + (1 - side);
                    for (int v = 0; v < NV; v++) {
                        double corr = 0.25 * reg[(fo * 6 + opp) * NV + v];
                        u_new[(int64_t)v * ncell + C] = side ? u_new[(int64_t)v * ncell + C] - lam * corr
                                                             : u_new[(int64_t)v * ncell + C] + lam * corr;
                    }
                }
            }
    }
    for (int64_t o = o0; o < o1; o++)
        for (int c = 0; c < 8; c++) {
            int64_t s = t->son[8 * o + c];
            if (s < 0) continue;
            for (int v = 0; v < NV; v++) {
                double sum = 0.0;
                for (int q = 0; q < 8; q++) sum += u_new[(int64_t)v * ncell + s * 8 + q];
                u_new[(int64_t)v * ncell + o * 8 + c] = 0.125 * sum;
            }
        }
    return OR_OK;
}

int or_courant(const or_tree *t, const or_params *p, const double *u, double *dt)
{
    int64_t ncell = t->noct * 8;
    double best = INFINITY;
    for (int64_t o = t->lvl_off[t->levelmin]; o < t->noct; o++) {
        double dx = dx_of(t->lvl[o]);
        for (int c = 0; c < 8; c++) {
            int64_t cid = o * 8 + c;
            if (t->son[cid] >= 0) continue;
            double U[NV], W[NV];
            load(u, ncell, cid, U);
            or_cons_to_prim(U, p->gamma, p->rho_floor, p->p_floor, W);
            double cs = sqrt(p->gamma * W[4] / W[0]);
            double sig = (fabs(W[1]) + cs) + (fabs(W[2]) + cs) + (fabs(W[3]) + cs);
            double r = dx / sig;
            if (r < best) best = r;
        }
    }
    *dt = p->cfl * best;
    return OR_OK;
}

int or_step(const or_tree *t, const or_params *p, const double *u_old, double *u_new, double *dt_out, int nthreads)
{
    (void)nthreads;
    double dt;
    or_courant(t, p, u_old, &dt);
    if (dt_out) *dt_out = dt;
    size_t regn = (size_t)t->noct * 6 * NV;
    double *reg = calloc(regn, sizeof(double));
    int st = OR_OK;
    for (int l = t->levelmin; l <= t->levelmax; l++) {
        int r = or_level_update(t, p, l, u_old, u_new, reg, dt);
        if (r != OR_OK && st == OR_OK) st = r;
    }
    for (int l = t->levelmax - 1; l >= 1; l--) or_reflux_restrict(t, p, l, reg, u_new, dt);
    free(reg);
    return st;
}

int or_init_from_prim(const or_tree *t, const or_params *p, const double *w, double *u)
{
    int64_t ncell = t->noct * 8;
    for (int64_t cid = 0; cid < ncell; cid++) {
        double W[NV], U[NV];
        for (int v = 0; v < NV; v++) W[v] = w[(int64_t)v * ncell + cid];
        or_prim_to_cons(W, p->gamma, U);
        for (int v = 0; v < NV; v++) u[(int64_t)v * ncell + cid] = U[v];
    }
    for (int l = t->levelmax - 1; l >= 1; l--) or_reflux_restrict(t, p, l, NULL, u, 0.0);
    return OR_OK;
}

int or_prim_of_state(const or_tree *t, const or_params *p, const double *u, double *w)
{
    int64_t ncell = t->noct * 8;
    for (int64_t cid = 0; cid < ncell; cid++) {
        double W[NV], U[NV];
        for (int v = 0; v < NV; v++) U[v] = u[(int64_t)v * ncell + cid];
        or_cons_to_prim(U, p->gamma, p->rho_floor, p->p_floor, W);
        for (int v = 0; v < NV; v++) w[(int64_t)v * ncell + cid] = W[v];
    }
    return OR_OK;
}

/* the value of level-l cell (X,Y,Z): its own state, or the interpolation from its father
   used for ghost cells when it does not exist (returns -1 then, < -1 if unbalanced) */
int64_t or_cell_value(const or_tree *t, const double *u, int l, int64_t X, int64_t Y, int64_t Z, double *U)
{
    return cell_value(t, u, l, X, Y, Z, U);
}
