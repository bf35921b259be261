/*
 * Plain FP64 CPU oracle for the AMR Godunov hydro hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or calls
 * this code; only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no source with the CUDA path.
 *
 * The paper (RAMSES-yOMP, arXiv 2411.14631) names the routines of this path only in
 * Table 1 (godunov_fine: the hydro solver; newdt_fine: time stepping; refine_fine:
 * refinement) and the fully threaded octree (Sec. 1); it does not print the scheme.
 * The scheme is therefore written out from the published methods it rests on:
 *   - the octree and its neighbour relations: Khokhlov 1998 / Teyssier 2002 (Sec. 1),
 *   - the Peano-Hilbert key (Sec. 1): Skilling 2004, "Programming the Hilbert curve",
 *   - MUSCL-Hancock in primitive variables with MinMod slopes: Toro 2009, Sec. 14.4,
 *   - HLLC: Toro, Spruce & Speares 1994; Toro 2009, Sec. 10.4,
 *   - the exact Riemann solver: Toro 2009, Ch. 4,
 *   - one global time step for all levels: the "single time step" option of Eq. 1's
 *     weighting discussion (Sec. 2.3).
 * Every floating-point quantity is FP64.  Compiled with -ffp-contract=off.
 */
#ifndef HYDRO_ORACLE_H
#define HYDRO_ORACLE_H
#include <stdint.h>

#define OR_MAXLEV 21
#define OR_NVAR 5

enum { OR_OK = 0, OR_EINVAL = -1, OR_EUNBALANCED = -2, OR_ENONPHYSICAL = -6, OR_ENOCONV = -7,
       OR_EBREAKDOWN = -8 };
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1 };
enum { OR_HLLC = 0, OR_EXACT = 1 };
/* nb27 entry for a father-level position outside an outflow boundary */
#define OR_OUTSIDE ((int32_t)0x80000000)

typedef struct {
    int32_t levelmin, levelmax;   /* levelmax = deepest level present */
    int32_t bc[6];                /* faces -x,+x,-y,+y,-z,+z */
    int64_t noct;
    int64_t lvl_off[OR_MAXLEV + 2];
    int32_t *lvl, *ix, *iy, *iz;  /* oct level and oct coordinates (oct units) */
    uint64_t *key;                /* Hilbert key with 3*(lvl-1) bits */
    int32_t *son;                 /* [noct*8]  child oct of each cell, or -1 */
    int32_t *father;              /* [noct]    father cell id, -1 at level 1 */
    int32_t *nbor;                /* [noct*6]  father-level face neighbour cell, -1 outside */
    int32_t *nb27;                /* [noct*27] same-level neighbour oct, -(1+coarse cell), or OR_OUTSIDE */
    int64_t *lex;                 /* oct ids sorted by (lvl, ix, iy, iz) for lookups */
} or_tree;

enum { OR_LIMITER_MINMOD = 0, OR_LIMITER_MC = 1 };

typedef struct {
    double gamma, cfl, rho_floor, p_floor;
    int32_t riemann;              /* OR_HLLC or OR_EXACT */
    int32_t limiter;              /* slopes of the reconstruction: OR_LIMITER_MINMOD or OR_LIMITER_MC */
} or_params;

uint64_t or_hilbert_key(int bits, uint32_t x, uint32_t y, uint32_t z);

int  or_tree_build(int32_t levelmin, const int32_t *bc, const int32_t *lxyz, int64_t n, or_tree **out);
void or_tree_free(or_tree *t);
int64_t or_tree_noct(const or_tree *t);
void or_tree_export(const or_tree *t, int32_t *lvl, int32_t *ix, int32_t *iy, int32_t *iz, uint64_t *key,
                    int32_t *son, int32_t *father, int32_t *nbor, int32_t *nb27, int64_t *lvl_off);
int64_t or_lookup(const or_tree *t, int l, int64_t x, int64_t y, int64_t z);

/* single-state pieces */
double or_minmod(double a, double b);
double or_mc(double a, double b);
double or_slope(int limiter, double a, double b);
void or_cons_to_prim(const double *U, double gamma, double rho_floor, double p_floor, double *W);
void or_prim_to_cons(const double *W, double gamma, double *U);
void or_flux_normal(const double *W, double gamma, double *F);
void or_hllc(const double *WL, const double *WR, double gamma, double *F);
int  or_exact_star(const double *WL, const double *WR, double gamma, double tol, int maxit,
                   double *pstar, double *ustar, int *iters);
int  or_exact_sample(const double *WL, const double *WR, double gamma, double pstar, double ustar,
                     double S, double *W);
int  or_riemann_flux(const double *WL, const double *WR, const or_params *p, double *F);

/* per-oct pieces and whole steps; state arrays are u[var*ncell + cell], cell = oct*8 + c */
int or_oct_stencil(const or_tree *t, const double *u, int64_t oct, double *stencil /*[5][6][6][6]*/);
int or_courant(const or_tree *t, const or_params *p, const double *u, double *dt);
int or_level_update(const or_tree *t, const or_params *p, int level, const double *u_old, double *u_new,
                    double *reg /*[noct][6][5]*/, double dt);
int or_octs_update(const or_tree *t, const or_params *p, int64_t o0, int64_t o1, const double *u_old, double *u_new,
                   double *reg, double dt);
int or_reflux_restrict(const or_tree *t, const or_params *p, int level, const double *reg, double *u_new, double dt);
int or_step(const or_tree *t, const or_params *p, const double *u_old, double *u_new, double *dt_out, int nthreads);
int or_init_from_prim(const or_tree *t, const or_params *p, const double *w, double *u);
int or_prim_of_state(const or_tree *t, const or_params *p, const double *u, double *w);

/* one uniform box of N^3 cells of size 1/N, state [5][N^3] with cell i + N (j + N k) */
int or_box_courant(int64_t N, const or_params *p, const double *u, double *dt);
int or_box_step(int64_t N, const int32_t *bc, const or_params *p, const double *u, double *u_new, double dt);

/* learned Riemann surrogate (FP64 reference of the network) */
int64_t or_mlp_nparams(void);
void or_mlp_features(const double *WL, const double *WR, double gamma, double *x /*[7]*/, double *ref /*[3]*/);
void or_mlp_forward(const double *theta, const double *x, int64_t n, double *y, double *act /*nullable*/);
void or_mlp_backward(const double *theta, const double *x, const double *dy, int64_t n, double *act, double *grad);
void or_adam_step(double *th, double *m, double *v, const double *grad, int64_t n, double lr,
                  double beta1, double beta2, double eps, int64_t t);

/* one coarse step with level sub-cycling, dt(l+1) = dt(l)/2 (subcycle.c); u in place */
int or_courant_levels(const or_tree *t, const or_params *p, const double *u, double *dt_base);
int or_step_subcycled(const or_tree *t, const or_params *p, double *u, double *dt_out);

/* refinement between steps (refine.c) */
int or_refine_flags(const or_tree *t, const double *u, double mass_thr, int lmax, uint8_t *flag /*[8 noct]*/);
int or_refine_list(const or_tree *t, const double *u, double mass_thr, int lmax, int32_t *lxyz /*[cap][4]*/,
                   int64_t cap, int64_t *n_out);
int or_remap(const or_tree *t_old, const double *u_old, const or_tree *t_new, double *u_new);
int64_t or_cell_value(const or_tree *t, const double *u, int l, int64_t X, int64_t Y, int64_t Z, double *U);

/* Poisson solve on a box of nx*ny*nz cells, vectors indexed i + nx (j + ny k) (poisson.c) */
enum { OR_PRECOND_NONE = 0, OR_PRECOND_IP = 1 };
void or_poisson_apply_A(int nx, int ny, int nz, const double *x, double *y);
void or_poisson_apply_Minv(int nx, int ny, int nz, int precond, const double *r, double *u);
int or_cg(int nx, int ny, int nz, int precond, const double *b, double *x, double tol, int maxit,
          double *eps, int *iters);
int or_ppcg(int nx, int ny, int nz, int precond, const double *b, double *x, double tol, int maxit,
            double *eps, int *iters);

#endif
