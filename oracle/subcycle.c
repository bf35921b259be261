/*
 * Oracle: one coarse step with level sub-cycling, dt(l+1) = dt(l)/2 (TEST
 * INFRASTRUCTURE ONLY).
 *
 * Sec. 2.3 (the weights next to Eq. 1) contrasts sub-cycled levels, where level l+1 makes
 * two steps for every step of level l, with one time step for all levels; the paper
 * prints no scheme for it.  The readings written out here:
 *   - time steps: dt_l = dt_base 2^-(l - levelmin), so dt_l / dx_l is the same on every
 *     level; dt_base is the largest step every leaf accepts at its own level,
 *       dt_base = C_cfl * min over leaves of 2^(l - levelmin) dx_l / sum_d (|u_d| + c);
 *   - order (coarse first): level c is advanced by dt_c from the state at its time T,
 *     then level c+1 makes two steps of dt_c / 2.  The first reads level-c ghosts at T.
 *     For the second, the leaves of level c hold the mean of their values at T and at
 *     T + dt_c, a linear interpolation in time at T + dt_c/2, plus the first fine step's
 *     reflux correction: the coarse prediction carries no flux at the faces next to
 *     refined cells, and the fine flux of the first step stands in for it over the half
 *     step (uniform flow then stays uniform).  The refined cells of level c hold the
 *     mean of their children after the first fine step;
 *   - refluxing: a coarse face next to a refined cell carries no flux at level c; after
 *     each fine step the coarse leaf takes -/+ dt_{c+1} / dx_c * 1/4 * (sum of the four
 *     fine fluxes of that step), so the fine fluxes are applied with the fine time step
 *     over both steps and the totals are conserved;
 *   - restriction: after each fine step the refined cells of level c become the mean of
 *     their children; at the end of the step the levels below levelmin are restricted.
 * With a single level this is the step of or_step.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define NV OR_NVAR

int or_courant_levels(const or_tree *t, const or_params *p, const double *u, double *dt_base)
{
    int64_t ncell = t->noct * 8;
    double best = INFINITY;
    for (int64_t o = t->lvl_off[t->levelmin]; o < t->noct; o++) {
        int l = t->lvl[o];
        double dx = ldexp(1.0, -l);
        for (int c = 0; c < 8; c++) {
            int64_t cid = o * 8 + c;
            if (t->son[cid] >= 0) continue;
            double U[NV], W[NV];
            for (int v = 0; v < NV; v++) U[v] = u[(int64_t)v * ncell + cid];
            or_cons_to_prim(U, p->gamma, p->rho_floor, p->p_floor, W);
            double cs = sqrt(p->gamma * W[4] / W[0]);
            double sig = (fabs(W[1]) + cs) + (fabs(W[2]) + cs) + (fabs(W[3]) + cs);
            double r = ldexp(dx / sig, l - t->levelmin);
            if (r < best) best = r;
        }
    }
    *dt_base = p->cfl * best;
    return OR_OK;
}

typedef struct {
    const or_tree *t;
    const or_params *p;
    double *U, *N, *reg;
    double dt[OR_MAXLEV + 2];
    int st;
} sc_ctx;

static void copy_level(const or_tree *t, int l, const double *src, double *dst)
{
    int64_t ncell = t->noct * 8, c0 = t->lvl_off[l] * 8, c1 = t->lvl_off[l + 1] * 8;
    for (int v = 0; v < NV; v++)
        memcpy(dst + (int64_t)v * ncell + c0, src + (int64_t)v * ncell + c0, (size_t)(c1 - c0) * sizeof(double));
}

static void lerp_leaves(const or_tree *t, int l, double *U, const double *N)
{
    int64_t ncell = t->noct * 8;
    for (int64_t cell = t->lvl_off[l] * 8; cell < t->lvl_off[l + 1] * 8; cell++) {
        if (t->son[cell] >= 0) continue;
        for (int v = 0; v < NV; v++) {
            int64_t i = (int64_t)v * ncell + cell;
            U[i] = 0.5 * (U[i] + N[i]);
        }
    }
}

static void advance(sc_ctx *x, int c)
{
    const or_tree *t = x->t;
    int r = or_level_update(t, x->p, c, x->U, x->N, x->reg, x->dt[c]);
    if (r != OR_OK && x->st == OR_OK) x->st = r;
    if (c < t->levelmax) {
        advance(x, c + 1);
        /* ghosts for the second fine step: the time interpolation of the coarse leaves,
           plus the first fine step's correction (the coarse prediction has no flux at the
           faces next to refined cells), and refined cells restricted from the fine level */
        lerp_leaves(t, c, x->U, x->N);
        or_reflux_restrict(t, x->p, c, x->reg, x->U, x->dt[c + 1]);
        or_reflux_restrict(t, x->p, c, x->reg, x->N, x->dt[c + 1]);
        advance(x, c + 1);
        or_reflux_restrict(t, x->p, c, x->reg, x->N, x->dt[c + 1]);
    }
    copy_level(t, c, x->N, x->U);
}

int or_step_subcycled(const or_tree *t, const or_params *p, double *u, double *dt_out)
{
    if (!t || !p || !u) return OR_EINVAL;
    int64_t ncell = t->noct * 8;
    sc_ctx x;
    x.t = t;
    x.p = p;
    x.st = OR_OK;
    double dtb;
    or_courant_levels(t, p, u, &dtb);
    for (int l = 0; l < OR_MAXLEV + 2; l++) x.dt[l] = l >= t->levelmin ? ldexp(dtb, -(l - t->levelmin)) : dtb;
    x.U = u;
    x.N = malloc((size_t)ncell * NV * sizeof(double));
    memcpy(x.N, u, (size_t)ncell * NV * sizeof(double));
    x.reg = calloc((size_t)t->noct * 6 * NV, sizeof(double));
    advance(&x, t->levelmin);
    for (int l = t->levelmin - 1; l >= 1; l--) or_reflux_restrict(t, p, l, NULL, x.U, 0.0);
    free(x.N);
    free(x.reg);
    if (dt_out) *dt_out = dtb;
    return x.st;
}
