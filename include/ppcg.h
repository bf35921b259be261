/*
 * ppcg -- C ABI of the GB300 Poisson solver of arXiv 2411.14631 Sec. 2.3: the
 * preconditioned pipelined conjugate gradient (PPCG; Ghysels & Vanroose 2014,
 * Algorithm 4) that replaces RAMSES' conjugate gradient for the cell-level potential,
 * with the 7-point incomplete-Poisson preconditioner (centre 13/12, the six face
 * neighbours 1/6, Sec. 2.3) and the convergence measure of Eq. 3,
 * eps_i = sqrt((r_i . u_i) / (r_0 . u_0)), u_i = M^-1 r_i.
 *
 * Linear system: A x = b on a box of nx*ny*nz cells.  Vectors are FP64 arrays of
 * n = nx*ny*nz entries indexed i + nx (j + ny k).  A = 6 I - N with (N v)_c the sum of v
 * over the face neighbours of cell c inside the box: the 7-point Laplacian times -h^2
 * with homogeneous Dirichlet boundaries.  The caller folds Dirichlet boundary values and
 * h^2 4 pi G rho into b.  The preconditioner stencil is the same in every cell; a
 * neighbour outside the box contributes nothing.  PPCG_PRECOND_NONE makes M^-1 the
 * identity (pipelined CG, the same iterates as the textbook CG in exact arithmetic).
 *
 * Iteration semantics: iteration i (i = 0, 1, ...) makes x_{i+1}.  The solve stops at the
 * first i >= 1 with eps_i <= tol (status AMR_OK), after max_iter iterations without
 * that (AMR_ENOCONV), or when a step length is not positive and finite
 * (AMR_EBREAKDOWN: A or M^-1 is not positive definite in floating point).  When
 * r_0 . u_0 = 0 the initial guess is returned with 0 iterations, eps_0 = 0.
 *
 * Memory: every d_* pointer is device memory owned by the caller; the library allocates
 * nothing.  d_work holds the solver's vectors and scalars (ppcg_workspace_bytes, base
 * aligned to 256 bytes) and must stay untouched between ppcg_start and the last
 * ppcg_iterate of a solve.  d_eps, when not NULL, receives eps_0 .. eps_iters
 * (max_iter + 1 doubles).  Asynchronous calls take a stream and can be captured in a
 * CUDA graph; ppcg_poll and ppcg_solve synchronise the stream.
 */
#ifndef PPCG_H
#define PPCG_H

#include "amrhydro.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { PPCG_PRECOND_NONE = 0, PPCG_PRECOND_IP = 1 };
enum { POISSON_OP_A = 0, POISSON_OP_MINV = 1 };

typedef struct {
    int32_t nx, ny, nz;       /* box size in cells, each >= 1 */
    int32_t precond;          /* PPCG_PRECOND_NONE or PPCG_PRECOND_IP */
    double tol;               /* stop at the first i >= 1 with eps_i <= tol; >= 0 */
    int32_t max_iter;         /* >= 0 */
    int32_t check_every;      /* ppcg_solve: iterations launched between host checks (0: 16) */
    int32_t tile_y;           /* rows of the 32-wide tile of one thread block: 8 or 16 (0: 8) */
    int32_t seg;              /* z planes one thread block marches through (0: chosen; else >= 4) */
} ppcg_params;

typedef struct {
    int32_t iters;            /* iterations made (updates of x) */
    int32_t done;             /* 1 once the solve has stopped */
    int32_t status;           /* AMR_OK, AMR_ENOCONV (also while running) or AMR_EBREAKDOWN */
    int32_t pad;
    double eps;               /* eps_iters (Eq. 3) */
} ppcg_info;

/* Bytes of d_work for a box (8 vectors of n doubles plus scalars and block partials);
   0 if a size is < 1. */
size_t ppcg_workspace_bytes(int32_t nx, int32_t ny, int32_t nz);

/* d_out = A d_in (op = POISSON_OP_A) or M^-1 d_in (POISSON_OP_MINV, the incomplete-Poisson
   stencil); asynchronous.  AMR_EINVAL for a bad size, op or NULL pointer. */
amr_status poisson_apply(int32_t nx, int32_t ny, int32_t nz, int32_t op, const double *d_in, double *d_out,
                         amr_stream stream);

/* Start a solve: r_0 = b - A x_0, u_0 = M^-1 r_0, w_0 = A u_0, the inner products
   r_0 . u_0 and w_0 . u_0 and the first step length; eps_0 to d_eps[0].  Asynchronous.
   AMR_EINVAL / AMR_ECAPACITY for bad arguments or a short workspace. */
amr_status ppcg_start(const ppcg_params *prm, const double *d_b, const double *d_x, void *d_work,
                      size_t work_bytes, double *d_eps, amr_stream stream);

/* Launch `count` PPCG iterations, one fused kernel each (both preconditioner and operator
   applications, the eight vector recurrences and the next iteration's two inner
   products; the last thread block to finish reduces the inner products in a fixed order
   and computes the next step length).  Iterations after the solve has stopped return at
   once, so over-launching is harmless.  d_x is updated in place.  Asynchronous. */
amr_status ppcg_iterate(const ppcg_params *prm, double *d_x, void *d_work, size_t work_bytes, double *d_eps,
                        int32_t count, amr_stream stream);

/* Read the solve's state (synchronises the stream). */
amr_status ppcg_poll(const void *d_work, ppcg_info *h_info, amr_stream stream);

/* ppcg_start, then ppcg_iterate in chunks of check_every with a ppcg_poll after each,
   until the solve stops.  Returns the solve's status (AMR_OK, AMR_ENOCONV,
   AMR_EBREAKDOWN) or an argument / CUDA error; h_info may be NULL. */
amr_status ppcg_solve(const ppcg_params *prm, const double *d_b, double *d_x, void *d_work, size_t work_bytes,
                      double *d_eps, ppcg_info *h_info, amr_stream stream);

#ifdef __cplusplus
}
#endif
#endif
