/*
 * Oracle: refinement of the octree between steps, refine_fine of Table 1 (TEST
 * INFRASTRUCTURE ONLY).
 *
 * The paper names the routine but not its rules; the readings written out here:
 *   - criterion (quasi-Lagrangian, the rule of the clump workload): a cell at level l
 *     with levelmin <= l < lmax is refined iff its mass rho * dx_l^3 exceeds mass_thr,
 *     where rho is the cell's own density (a refined cell holds the mean of its
 *     children).  Cells above levelmin are always refined (levels 1..levelmin stay
 *     complete); cells at lmax or deeper never are;
 *   - 2:1 balance: a refined cell's 26 neighbours must exist, so, level by level from the
 *     finest up, every refined cell at level l also refines the level-(l-1) cells that
 *     contain its neighbours (2 per axis, its own father among them).  A neighbour beyond
 *     an outflow face needs nothing; periodic faces wrap;
 *   - a cell exists in the new tree iff its father is refined (levels 1..levelmin always),
 *     so the new oct list is the root oct plus the child oct of every refined cell;
 *     octs whose father is no longer refined are dropped (derefinement), several levels
 *     at once if needed;
 *   - state: a cell present in both trees keeps its conserved state (a derefined cell
 *     keeps the restricted mean it already holds); a new cell is the interpolation of its
 *     father used for ghost cells,
 *       U = U_C + sum_d s_d * 1/4 * minmod(U_C - U_{C-e_d}, U_{C+e_d} - U_C),
 *     whose eight children sum to 8 U_C, so the total mass, momentum and energy of the
 *     leaves are unchanged up to rounding.
 * Refinement grows by at most one level per call: only cells of the old tree are tested.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "oracle.h"

static int64_t wrap_or_skip(const or_tree *t, int axis, int l, int64_t c, int *skip)
{
    int64_t n = (int64_t)1 << l;
    *skip = 0;
    if (c >= 0 && c < n) return c;
    if (t->bc[2 * axis + (c >= n)] == OR_BC_PERIODIC) return ((c % n) + n) % n;
    *skip = 1;
    return c;
}

static void cell_coords(const or_tree *t, int64_t cell, int64_t X[3])
{
    int64_t o = cell >> 3;
    int c = (int)(cell & 7);
    X[0] = 2 * (int64_t)t->ix[o] + (c & 1);
    X[1] = 2 * (int64_t)t->iy[o] + ((c >> 1) & 1);
    X[2] = 2 * (int64_t)t->iz[o] + ((c >> 2) & 1);
}

int or_refine_flags(const or_tree *t, const double *u, double mass_thr, int lmax, uint8_t *flag)
{
    if (!t || !u || !flag || lmax < t->levelmin || lmax > OR_MAXLEV) return OR_EINVAL;
    int64_t ncell = t->noct * 8;
    /* the criterion */
    for (int64_t cell = 0; cell < ncell; cell++) {
        int l = t->lvl[cell >> 3];
        if (l < t->levelmin) flag[cell] = 1;
        else if (l >= lmax) flag[cell] = 0;
        else {
            double dx = ldexp(1.0, -l);
            flag[cell] = u[cell] * (dx * dx * dx) > mass_thr;
        }
    }
    /* 2:1 balance, finest level first */
    for (int l = t->levelmax; l > t->levelmin; l--) {
        for (int64_t cell = t->lvl_off[l] * 8; cell < t->lvl_off[l + 1] * 8; cell++) {
            if (!flag[cell]) continue;
            int64_t X[3];
            cell_coords(t, cell, X);
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    for (int c = 0; c < 2; c++) {
                        /* the parents of the neighbours X-1, X, X+1 along each axis are
                           (X-1)>>1 and (X+1)>>1 (one of them is X>>1) */
                        int64_t T[3] = { (X[0] + (a ? 1 : -1)) >> 1, (X[1] + (b ? 1 : -1)) >> 1,
                                         (X[2] + (c ? 1 : -1)) >> 1 };
                        int skip = 0, s;
                        for (int d = 0; d < 3; d++) {
                            T[d] = wrap_or_skip(t, d, l - 1, T[d], &s);
                            skip |= s;
                        }
                        if (skip) continue;
                        int64_t o = or_lookup(t, l - 1, T[0] >> 1, T[1] >> 1, T[2] >> 1);
                        if (o < 0) return OR_EUNBALANCED;   /* the old tree breaks the 2:1 rule */
                        flag[o * 8 + (T[0] & 1) + 2 * (T[1] & 1) + 4 * (T[2] & 1)] = 1;
                    }
        }
    }
    /* a cell whose father is not refined does not exist in the new tree (after the
       balance pass every refined cell's father is refined, so this changes nothing) */
    for (int l = t->levelmin + 1; l <= t->levelmax; l++)
        for (int64_t cell = t->lvl_off[l] * 8; cell < t->lvl_off[l + 1] * 8; cell++)
            if (!flag[t->father[cell >> 3]]) flag[cell] = 0;
    return OR_OK;
}

int or_refine_list(const or_tree *t, const double *u, double mass_thr, int lmax, int32_t *lxyz, int64_t cap,
                   int64_t *n_out)
{
    if (!lxyz || !n_out) return OR_EINVAL;
    int64_t ncell = t ? t->noct * 8 : 0;
    uint8_t *flag = malloc(ncell > 0 ? (size_t)ncell : 1);
    int st = or_refine_flags(t, u, mass_thr, lmax, flag);
    if (st != OR_OK) { free(flag); return st; }
    int64_t n = 0;
    if (cap < 1) { free(flag); return OR_EINVAL; }
    lxyz[0] = 1; lxyz[1] = 0; lxyz[2] = 0; lxyz[3] = 0;    /* the root oct */
    n = 1;
    for (int64_t cell = 0; cell < ncell; cell++) {
        if (!flag[cell]) continue;
        if (n >= cap) { free(flag); return OR_EINVAL; }
        int64_t X[3];
        cell_coords(t, cell, X);
        lxyz[4 * n + 0] = t->lvl[cell >> 3] + 1;
        lxyz[4 * n + 1] = (int32_t)X[0];
        lxyz[4 * n + 2] = (int32_t)X[1];
        lxyz[4 * n + 3] = (int32_t)X[2];
        n++;
    }
    free(flag);
    *n_out = n;
    return OR_OK;
}

/* hydro.c: the value of level-l cell (X,Y,Z), interpolated from its father if missing */
int64_t or_cell_value(const or_tree *t, const double *u, int l, int64_t X, int64_t Y, int64_t Z, double *U);

int or_remap(const or_tree *t_old, const double *u_old, const or_tree *t_new, double *u_new)
{
    if (!t_old || !u_old || !t_new || !u_new) return OR_EINVAL;
    int64_t ncell = t_new->noct * 8;
    for (int64_t cell = 0; cell < ncell; cell++) {
        int64_t X[3];
        cell_coords(t_new, cell, X);
        double U[OR_NVAR];
        int64_t r = or_cell_value(t_old, u_old, t_new->lvl[cell >> 3], X[0], X[1], X[2], U);
        if (r < -1) return OR_EUNBALANCED;
        for (int v = 0; v < OR_NVAR; v++) u_new[(int64_t)v * ncell + cell] = U[v];
    }
    return OR_OK;
}
