/*
 * amrhydro -- C ABI of the GB300 (sm_103a) AMR Godunov hydro hot path.
 *
 * The operations are those of RAMSES' level step as named in arXiv 2411.14631:
 * Table 1 lists godunov_fine (the hydro solver), newdt_fine (time stepping) and
 * refine_fine (refinement); Sec. 1 describes the fully threaded octree (cubic cells
 * split recursively into eight octants) and the Peano-Hilbert ordering of space.  The
 * paper prints no hydro scheme; the one computed here is the unsplit MUSCL-Hancock
 * scheme (MinMod slopes, HLLC or exact Riemann solver) on the octree with one global
 * time step for all levels (the "single time step" option discussed with Eq. 1,
 * Sec. 2.3), refluxing at coarse-fine faces and restriction of refined cells.
 *
 * Conventions shared by every entry point:
 *   - Level l has 2^l cells per dimension in the unit box; dx_l = 2^-l.  An oct at
 *     level l holds 2^3 level-l cells and has oct coordinates (ix,iy,iz) in
 *     [0, 2^(l-1)); its father cell is the level-(l-1) cell (ix,iy,iz).
 *   - Octs are numbered by (level, Hilbert key); cell id = oct*8 + c with
 *     c = cx + 2 cy + 4 cz.
 *   - State arrays are FP64 structure-of-arrays u[v*ncell + cell], ncell = 8*noct,
 *     v = rho, rho u, rho v, rho w, E (conserved) or rho, u, v, w, p (primitive).
 *   - Every pointer named d_* is device memory owned by the caller; h_* is host memory.
 *     The library never allocates device memory and never frees caller memory.
 *   - Calls that take a stream are asynchronous on it, make no host synchronisation
 *     and read the time step through a device pointer, so a sequence of them can be
 *     captured in a CUDA graph (hydro_step_static_scratch is not covered by this
 *     statement).  amr_build_octree and amr_get_status synchronise.
 *   - Argument errors are returned at once.  Errors found on the device (a
 *     non-physical state, a failed exact solve) are written to params->d_status
 *     (first error wins) and read with amr_get_status.  Nothing aborts or traps.
 */
#ifndef AMRHYDRO_H
#define AMRHYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *amr_stream;   /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
    AMR_OK = 0,
    AMR_EINVAL = -1,        /* bad argument or malformed oct list */
    AMR_EUNBALANCED = -2,   /* an oct's father lacks a father-level neighbour (2:1 rule) */
    AMR_ECAPACITY = -3,     /* a caller buffer is smaller than the query said */
    AMR_ECUDA = -4,         /* a CUDA runtime call failed */
    AMR_ETIMEOUT = -5,      /* a bounded device-side wait gave up */
    AMR_ENONPHYSICAL = -6,  /* a non-physical state: vacuum in an exact Riemann problem (HLLC flux
                               used instead), or a cell whose updated state is not finite in the
                               working precision (NaN, +-Inf, or beyond FP32's range in the FP32
                               path); the state is written as computed */
    AMR_ENOCONV = -7,       /* an iteration did not converge: the exact Riemann Newton iteration
                               (HLLC used instead), or a Poisson solve within its iteration cap */
    AMR_EBREAKDOWN = -8     /* a Poisson solve met a step length that is not positive and finite */
} amr_status;

enum { AMR_BC_PERIODIC = 0, AMR_BC_OUTFLOW = 1 };
enum { AMR_RIEMANN_HLLC = 0, AMR_RIEMANN_EXACT = 1, AMR_RIEMANN_MLP = 2, AMR_RIEMANN_MLP_SEEDED = 3 };
enum { AMR_PREC_FP64 = 0, AMR_PREC_FP32 = 1 };
enum { AMR_LIMITER_MINMOD = 0, AMR_LIMITER_MC = 1 };

#define AMR_MAXLEV 21
#define AMR_NCOUNTERS 8

/* Mesh description for amr_build_octree. */
typedef struct {
    int32_t levelmin;   /* levels 1..levelmin are complete; 2 <= levelmin (octree mode) */
    int32_t bc[6];      /* box faces -x,+x,-y,+y,-z,+z: AMR_BC_PERIODIC (both faces of an axis) or AMR_BC_OUTFLOW */
    int32_t n_inst;     /* 0: one octree from the oct list.  > 0: batch mode, n_inst independent
                           uniform unit boxes (the oct list is then ignored) */
    const int32_t *h_inst_n;   /* batch mode: host [n_inst], cells per dimension of each box,
                                  a multiple of 4 (cubic cells of size 1/N) */
} amr_geom;

/* Scheme parameters.  gamma: ratio of specific heats; cfl: Courant number of the
   time step; rho_floor, p_floor: floors applied after cons->prim and to face states;
   riemann: AMR_RIEMANN_*; precision: AMR_PREC_FP64 (all arithmetic in FP64) or
   AMR_PREC_FP32 (reconstruction and Riemann solve in FP32, state accumulation in FP64);
   tile: 1 or 2 = depth of the oct tiles a CTA updates (8 or 64 octs), 0 = default;
   tiles_only: 0 = the deepest complete level is updated by the z-column kernel (the
   same arithmetic per cell as the tiles, less ghost work), 1 = tiles for every level;
   mlp_weights: device pointer to the surrogate's weights (AMR_RIEMANN_MLP and
   AMR_RIEMANN_MLP_SEEDED only);
   mlp_resid_tol: acceptance threshold of the surrogate's residual check;
   limiter: slopes of the reconstruction, AMR_LIMITER_MINMOD (MinMod) or AMR_LIMITER_MC
   (monotonized central, van Leer 1977; updated by the tile kernel on every level);
   d_status: device int32 error word (may be NULL); d_counters: device uint64
   counters[AMR_NCOUNTERS] (may be NULL), accumulated over calls: [0] faces solved by the
   surrogate (AMR_RIEMANN_MLP) or whose Newton solve it seeded (AMR_RIEMANN_MLP_SEEDED),
   [1] faces where the surrogate's answer was not used (fallback to a cold Newton start),
   [2] Newton iterations and [3] Newton solves made by the tile kernel's exact solver
   and by both surrogate modes (the z-column kernels do not count);
   col_kernel: the z-column kernel of the deepest complete level (and of box batches whose
   boxes are multiples of 16 cells): 0 = the library's choice (2 where it applies), 1 = 8 x 8-cell footprints
   marched two planes per step, 2 = 16 x 16-cell footprints with one thread per column
   (FP32 path only, levels and boxes that are multiples of 16 cells; otherwise 1 is used);
   col_seg: cells of z a CTA marches (0 = the library's choice; even; kernel 1 needs a
   power of two that divides the level, kernel 2 takes any even length, the last segment
   of the column being shorter).  Neither changes a result bit (tested): both are launch
   shapes for the autotuner;
   defer_restriction: if nonzero, hydro_step leaves out the restriction of the complete
   levels below the deepest complete one minus one (the levels no later step of the
   single-dt path reads); the caller runs it with hydro_restrict_complete, possibly on
   another stream, so that it overlaps the next step. */
typedef struct {
    double gamma, cfl, rho_floor, p_floor;
    int32_t riemann, precision, tile, tiles_only;
    const void *mlp_weights;
    float mlp_resid_tol;
    int32_t limiter;
    int32_t *d_status;
    unsigned long long *d_counters;
    int32_t col_kernel, col_seg;
    int32_t defer_restriction, reserved;
} hydro_params;

/* The octree: host metadata plus non-owning views into the caller's tree memory.
   Filled by amr_build_octree; the caller keeps the tree memory alive while in use. */
typedef struct {
    int64_t noct;
    int32_t levelmin, levelmax;
    int32_t bc[6];
    int64_t lvl_off[AMR_MAXLEV + 2];        /* octs of level l: [lvl_off[l], lvl_off[l+1]) */
    int64_t tile_off[2][AMR_MAXLEV + 2];    /* tiles of depth d+1 updating level l */
    int64_t reg_base;                       /* first oct owning a flux-register row */
    int32_t *lvl, *ix, *iy, *iz;            /* per oct: level, oct coordinates */
    uint64_t *key;                          /* per oct: Hilbert key, 3*(level-1) bits */
    int32_t *son;                           /* per cell: child oct or -1 */
    int32_t *father;                        /* per oct: father cell, -1 at level 1 */
    int32_t *nbor;                          /* per oct x 6: father-level face-neighbour cell, -1 beyond an outflow face */
    int32_t *nb27;                          /* per oct x 27: same-level neighbour oct, -(1+coarse cell), or INT32_MIN beyond an outflow face */
    uint8_t *refmask;                       /* per oct: bit c set iff cell c is refined */
    uint8_t *fused;                         /* per oct: 1 iff its father cell is restricted inside
                                               hydro_godunov_level (all eight cells leaves, none next
                                               to a refined cell), 0 if hydro_reflux_level does it */
    int32_t *tile_root[2];                  /* per tile: root oct (level l-d-1); batch mode: corner oct */
    int32_t *tile_slot[2];                  /* per tile: (2^(d+1)+2)^3 stencil slots: an oct (>= 0), a
                                               ghost father -(1+g), INT32_MIN beyond an outflow face,
                                               or INT32_MIN+1 (not needed: no updated oct reaches it;
                                               always so for the eight corner slots of a tree-mode
                                               tile, whose cells no face reads) */
    /* batch mode (n_inst > 0): octs of box i are [inst_oct_off[i], inst_oct_off[i+1]) in
       lexicographic (ix fastest) order, lvl[oct] holds the box index, no refinement; the
       time step is per box: d_dt and d_dt_next of the hydro calls are arrays [n_inst]. */
    int32_t n_inst;
    int32_t *inst_n;                        /* device [n_inst]: cells per dimension */
    double *inst_dx;                        /* device [n_inst]: 1 / N */
    int64_t *inst_oct_off;                  /* device [n_inst + 1] */
    int32_t *tile_inst[2];                  /* device, per tile: box index (batch mode) */
    /* octree mode: grid[ix + M (iy + M iz)] = oct index of the deepest complete level
       grid_level (levelmin at least; M = 2^(grid_level-1)), used by the z-column kernel */
    int32_t grid_level;
    int32_t *grid;
    /* batch mode, when every box is a multiple of 16 cells: the z-column kernel's work items
       (8x8-cell footprints x 16-cell segments), box i owning [inst_col_off[i], inst_col_off[i+1]);
       col_work = 0 if not available */
    int64_t col_work;
    int64_t *inst_col_off;
    /* octree mode: the coarse leaves that tiles interpolate from (ghost fathers), in cell
       order; a tile slot -(1+g) (g >= 0) stands for the children of cell ghost_cell[g];
       the ghost fathers of level l are [ghost_off[l], ghost_off[l+1]).  Their interpolated
       children are computed once per update call into the flux-register buffer. */
    int64_t n_ghost;
    int64_t ghost_off[AMR_MAXLEV + 2];
    int32_t *ghost_cell;
    /* octree mode: the cells the step's reflux pass has work for, in cell order: at levels
       levelmin .. levelmax-1, a refined cell whose child oct is not flagged in fused (its
       restriction is not done inside hydro_godunov_level) or a leaf with a refined face
       neighbour.  Those of level l are reflux_cell[reflux_off[l] .. reflux_off[l+1]). */
    int32_t *reflux_cell;
    int64_t reflux_off[AMR_MAXLEV + 2];
} amr_tree;

/* Sizes of the caller buffers amr_build_octree needs for this oct list (host list of
   n_oct records (level, ix, iy, iz), int32).  Pure host computation. */
amr_status amr_build_octree_query(const amr_geom *geom, const int32_t *h_oct_lxyz, int64_t n_oct,
                                  size_t *tree_bytes, size_t *workspace_bytes);

/* Build the octree (Sec. 1: fully threaded tree; Peano-Hilbert order): copy the oct
   list to the device, compute Hilbert keys, sort by (level, key), build son / father /
   nbor / nb27 / refmask and the tile stencil tables, check levels 1..levelmin complete,
   no duplicates, and the 2:1 rule.  d_tree_mem (tree_bytes, 256-byte aligned) holds the
   result; d_workspace (workspace_bytes) is scratch.  Synchronises the stream. */
amr_status amr_build_octree(const amr_geom *geom, const int32_t *h_oct_lxyz, int64_t n_oct,
                            void *d_tree_mem, size_t tree_bytes, void *d_workspace, size_t workspace_bytes,
                            amr_tree *out, amr_stream stream);

/* Primitive -> conserved for every cell, then restriction of refined cells (mean of
   their eight children), finest level first.  Sets a consistent initial state. */
amr_status hydro_init_from_prim(const amr_tree *tree, const hydro_params *params, const double *d_w,
                                double *d_u, amr_stream stream);

/* Conserved -> primitive for every cell, with the floors of params. */
amr_status hydro_prim_of_state(const amr_tree *tree, const hydro_params *params, const double *d_u,
                               double *d_w, amr_stream stream);

/* newdt_fine (Table 1): *d_dt = cfl * min over leaf cells of dx_l / sum_d (|u_d| + c)
   (batch mode: d_dt[i] for each box i, over its cells),
   c = sqrt(gamma p / rho).  FP64 for AMR_PREC_FP64; for AMR_PREC_FP32 it is evaluated
   in FP32, rounded to an FP32 value and scaled by (1 - 2^-16) so that it never exceeds
   the FP64 result. */
amr_status hydro_courant(const amr_tree *tree, const hydro_params *params, const double *d_u,
                         double *d_dt, amr_stream stream);

/* godunov_fine (Table 1) for one level (level >= levelmin) or for every level in one
   launch (level = -1): for every oct of the level(s), gather the ghosted stencil
   (interpolating from the coarser level where a neighbour is absent), MUSCL-Hancock
   predictor, Riemann solve at every face, conservative update into d_u_new (every leaf
   cell of the level's octs, plus the father cells of octs flagged in tree->fused: the
   mean of their eight new children; other refined cells are left to the restriction of
   hydro_reflux_level), and flux-register rows (d_flux_reg, hydro_flux_reg_bytes) for
   oct sides that face a coarser leaf.  Faces whose other side is a refined cell carry
   no flux here.  d_dt: device scalar time step (read, not written).  d_dt_next: if not
   NULL, receives atomically min(*d_dt_next, cfl * dx / sum(|u_d|+c)) over the leaf
   cells whose new value is final after this call (the CFL step of the next step, fused);
   hydro_reflux_level adds the cells it corrects.  Initialise it to a large value. */
amr_status hydro_godunov_level(const amr_tree *tree, int level, const hydro_params *params,
                               const double *d_u_old, double *d_u_new, double *d_flux_reg,
                               const double *d_dt, double *d_dt_next, amr_stream stream);

/* Bytes of the caller's flux-register buffer (device, 256-byte aligned): the register
   rows and the interpolated children of the ghost fathers. */
size_t hydro_flux_reg_bytes(const amr_tree *tree);

/* Refluxing and restriction for coarse level `level` (1 <= level < levelmax): the part
   of the level step of Table 1 (godunov_fine and its coarse-fine bookkeeping) that keeps
   the octree scheme conservative; the method is RAMSES' AMR scheme (Teyssier 2002, the
   code Sec. 1 builds on).  Run from the finest level up after every hydro_godunov_level
   of the step: each leaf cell of the level next to a refined cell receives
   -/+ dt/dx * 1/4 * (sum of the four fine fluxes) from the flux register d_flux_reg
   (device, hydro_flux_reg_bytes, written by hydro_godunov_level in the same step; may be
   NULL when level < levelmin); then each refined cell of the level becomes the mean of
   its eight children, in d_u_new (device FP64 SoA, updated in place).  d_dt: the step's
   device scalar time step; d_dt_next as in hydro_godunov_level, for the corrected cells.
   AMR_EINVAL for a level outside 1 .. levelmax-1 or a missing buffer; asynchronous.
   reflux_level is the same entry point under its shorter name; both names are
   exported. */
amr_status hydro_reflux_level(const amr_tree *tree, int level, const hydro_params *params,
                              const double *d_flux_reg, double *d_u_new, const double *d_dt,
                              double *d_dt_next, amr_stream stream);
amr_status reflux_level(const amr_tree *tree, int level, const hydro_params *params,
                        const double *d_flux_reg, double *d_u_new, const double *d_dt,
                        double *d_dt_next, amr_stream stream);

/* One whole step: checks its arguments (AMR_EINVAL as hydro_godunov_level, before
   anything is written), resets *d_dt_next (if not NULL) to a large value, then godunov on
   every level (one launch), then reflux + restriction from the finest level up.
   Equivalent to the calls above in that order (the same bits): below the deepest
   complete level minus one, where every cell is refined and the step is a pure
   restriction, three levels are restricted per launch (one CTA per subtree). */
amr_status hydro_step(const amr_tree *tree, const hydro_params *params, const double *d_u_old,
                      double *d_u_new, double *d_flux_reg, const double *d_dt, double *d_dt_next,
                      amr_stream stream);

/* The part of hydro_step that hydro_params.defer_restriction leaves out: the restriction
   (mean of the eight children, Table 1's level step) of the complete levels g-2 .. 1 from
   level g-1, g the deepest complete level (tree->grid_level), in d_u (device FP64 SoA, in
   place; the d_u_new of the hydro_step it completes).  It reads level g-1 and writes
   levels g-2 .. 1, which the next hydro_step neither reads nor writes: it may run on
   another stream while that step runs, but must finish before the step after it (which
   writes level g-1 of the same buffer) and before anything reads those levels.  No-op
   when g < 3 or in batch mode; AMR_EINVAL for a missing buffer.  Asynchronous. */
amr_status hydro_restrict_complete(const amr_tree *tree, double *d_u, amr_stream stream);

/* hydro_step without any caller-provided scratch.  The paper has no counterpart: this
   is an interface convenience.  Some callers cannot allocate device memory when they
   want to step: real-time loops that forbid allocation after start-up, and hosts whose
   device memory is owned by another framework's memory pool (a second allocator would
   fragment or overcommit it).  For them, the flux register lives in a fixed array inside
   this library, sized for at most AMR_STATIC_REG_MAX_OCTS octs above levelmin (31.5 MB,
   held by every GPU that loads the library until the process exits).  Trees with more
   such octs, or whose register with its ghost-children part (hydro_flux_reg_bytes)
   exceeds the array, get AMR_ECAPACITY and nothing runs.  Inputs and outputs are the
   caller's, as for hydro_step; no call allocates or frees device memory.  The first
   call on each device looks up the array's device address (no allocation) and caches
   it; make that first call before any stream capture.  The set-up is safe when several
   host threads make their first call at once.  cudaDeviceReset unloads the library's
   device code, and the cached address then names memory that no longer exists: after a
   reset this entry point must not be called again in the same process.  Every call
   shares the one array: calls whose work overlaps on the GPU (other streams, other host
   threads) race and give wrong results.  No register row needs a starting value: every
   row read in a call is written earlier in the same call, so nothing is cleared. */
#define AMR_STATIC_REG_MAX_OCTS 131072
amr_status hydro_step_static_scratch(const amr_tree *tree, const hydro_params *params, const double *d_u_old,
                                     double *d_u_new, const double *d_dt, double *d_dt_next, amr_stream stream);

/* ---- learned Riemann surrogate --------------------------------------------------------
   The paper has no learned component.  The project puts a small network in place of the
   iterative exact Riemann solver (Toro 2009, Ch. 4) of godunov_fine (Table 1): 7 -> 64 ->
   64 -> 64 -> 2, SiLU, BF16 weights with FP32 accumulation on the tensor cores.  Inputs
   are the normalised face-normal problem (rho_ref = rho_L, p_ref = max(p_L,p_R),
   c_ref = sqrt(p_ref/rho_ref), ubar = (u_L+u_R)/2):
     x = [log(rho_L/rho_ref), (u_L-ubar)/c_ref, log(p_L/p_ref), log(rho_R/rho_ref),
          (u_R-ubar)/c_ref, log(p_R/p_ref), gamma]  (stored as 8 floats, slot 7 unused),
     y = [log(p_star/p_ref), (u_star-ubar)/c_ref].
   Master parameters theta are FP32 in the order W1[64][7] b1 W2[64][64] b2 W3[64][64] b3
   W4[2][64] b4 (AMR_MLP_NPARAMS values).  With params->riemann = AMR_RIEMANN_MLP
   (AMR_PREC_FP32 only) the Godunov kernel evaluates the network at every face, accepts
   (p_star, u_star) when p_star > 0 and both |f(p_star)| and the velocity relation are
   within mlp_resid_tol * (c_L + c_R), and otherwise solves the face exactly; counters[0]
   and [1] count accepted faces and fallbacks.  With AMR_RIEMANN_MLP_SEEDED the network's
   p_star is instead the initial guess of the exact Newton iteration at every face (the
   linearised guess where the prediction is unusable), so every face gets the exact
   solver's answer to its tolerance and the network only saves iterations. */
#define AMR_MLP_NPARAMS 8962
int mlp_nparams(void);
/* Bytes of the packed BF16 weight block (device, 16-byte aligned) used by every kernel. */
size_t mlp_packed_bytes(void);
/* Scratch bytes mlp_grad / mlp_train_step need for a batch of n samples. */
size_t mlp_scratch_bytes(int64_t n);
/* FP32 master parameters -> packed BF16 block. */
amr_status mlp_pack(const float *d_theta, void *d_packed, amr_stream stream);
/* Dataset from face states d_states[n][6] = (rho_L,u_L,p_L,rho_R,u_R,p_R) (FP64): the
   exact FP64 solution labels each problem; writes d_x[n][8], d_y[n][2].  A problem the
   exact solver rejects (vacuum, no convergence) sets *d_status (if not NULL). */
amr_status mlp_make_dataset(const double *d_states, int64_t n, double gamma, float *d_x, float *d_y,
                            int32_t *d_status, amr_stream stream);
/* Inference: d_y[n][2] = net(d_x[n][8]); n = 0 is a no-op (d_x, d_y may be NULL). */
amr_status mlp_forward(const void *d_packed, const float *d_x, float *d_y, int64_t n, amr_stream stream);
/* Inference on the 5th-generation tensor cores: the same network as mlp_forward, d_y[n][2]
   = net(d_x[n][8]), over tiles of 128 samples (tcgen05.mma with BF16 operands in shared
   memory and FP32 accumulators in tensor memory).  The hidden layers' biases enter the
   accumulation as two BF16 terms (hi + lo, within 2^-17 of the FP32 bias); otherwise
   the activations are the same BF16 values as mlp_forward's up to the order of the FP32
   accumulation.  Slot 7 of each input row is ignored, as in mlp_forward.  d_x must be
   16-byte and d_y 8-byte aligned (else AMR_EINVAL); n = 0 is a no-op (d_x, d_y may be
   NULL).  Waits for the tensor cores are
   bounded; one that runs out writes AMR_ETIMEOUT to *d_status (may be NULL).
   Asynchronous. */
amr_status mlp_forward_tc(const void *d_packed, const float *d_x, float *d_y, int64_t n, int32_t *d_status,
                          amr_stream stream);
/* The roofline of mlp_forward_tc: the throughput of the MUFU tanh (tanh.approx.bf16x2,
   two results per instruction), which bounds it (192 tanh per sample).  Runs four CTAs
   of 512 threads per SM, each thread eight independent chains; writes the longest CTA
   time in SM clocks to *d_cycles and the number of tanh results of the launch to
   *h_results (host).  Results per clock per SM = *h_results / (SMs * *d_cycles).
   Asynchronous (d_cycles is valid after the stream reaches this point). */
amr_status mlp_tanh_rate(unsigned long long *d_cycles, int64_t *h_results, amr_stream stream);
/* d_grad[AMR_MLP_NPARAMS] = gradient of sum_i d_dy[i] . y(x_i) with respect to theta,
   through the BF16 network (for gradient checks). */
amr_status mlp_grad(const void *d_packed, const float *d_x, const float *d_dy, int64_t n, float *d_grad,
                    float *d_scratch, size_t scratch_bytes, amr_stream stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step count t >= 1) on the mean over the
   n samples of |y - d_y|^2; updates theta, the moments and the packed block; writes the
   batch loss before the step to *d_loss (if not NULL). */
amr_status mlp_train_step(float *d_theta, float *d_adam_m, float *d_adam_v, void *d_packed, const float *d_x,
                          const float *d_y, int64_t n, float lr, int64_t t, float *d_loss, float *d_scratch,
                          size_t scratch_bytes, amr_stream stream);

/* Training data for the surrogate, harvested from the method's own runs: the FP64
   Godunov kernel reconstructs every face of every level from d_u (with time step *d_dt)
   and writes a deterministic one-in-`stride` sample of the floored face-normal states
   (rho_L, u_L, p_L, rho_R, u_R, p_R) to d_states[capacity][6]; *d_count (caller zeroes
   it) counts the sampled faces, possibly more than capacity (the rest are dropped).
   d_u is not modified. */
amr_status hydro_harvest_faces(const amr_tree *tree, const hydro_params *params, const double *d_u,
                               const double *d_dt, double *d_states, int64_t capacity, int64_t stride,
                               unsigned long long *d_count, amr_stream stream);

/* ---- sub-cycled step, dt(l+1) = dt(l)/2 -----------------------------------------------
   Sec. 2.3 (the weights next to Eq. 1) sets sub-cycled levels, where level l+1 makes two
   steps per step of level l, against one time step for all levels (hydro_step); the
   paper prints no scheme.  The one computed here:
     - dt_l = dt_base 2^-(l - levelmin); dt_base = C_cfl * min over leaves of
       2^(l - levelmin) dx_l / sum_d (|u_d| + c) (hydro_courant_levels), so every level
       runs at the same Courant number;
     - coarse first: level c is advanced by dt_c, then level c+1 makes two steps of dt_c/2.
       The first reads level-c ghosts at the start time T.  For the second, the leaves of
       level c hold the mean of their states at T and T + dt_c plus the first fine
       step's reflux correction (the coarse update carries no flux at faces next to
       refined cells), and the refined cells of level c the mean of their children;
     - after each fine step, coarse leaves next to refined cells take -/+ dt_{c+1}/dx_c
       * 1/4 * sum of the fine fluxes; refined cells are restricted.
   d_u: state, advanced in place by one step of the coarsest level; d_scratch: a second
   state-sized buffer; d_flux_reg: hydro_flux_reg_bytes; d_dt: receives dt_base;
   d_dt_levels: device double[AMR_MAXLEV + 2], receives dt_l.  Asynchronous, no host
   synchronisation (capturable in a CUDA graph).  Octree mode only.  With one level it is
   hydro_step with the same dt. */
amr_status hydro_courant_levels(const amr_tree *t, const hydro_params *params, const double *d_u, double *d_dt,
                                amr_stream stream);
amr_status hydro_step_subcycled(const amr_tree *t, const hydro_params *params, double *d_u, double *d_scratch,
                                double *d_flux_reg, double *d_dt, double *d_dt_levels, amr_stream stream);

/* ---- refinement between steps (refine_fine, Table 1) ------------------------------
   The paper names the routine, not its rules.  The rules here:
     - a cell at level l, levelmin <= l < params->levelmax, is refined iff its mass
       rho dx_l^3 exceeds params->mass_thr (rho is the cell's own density; a refined cell
       holds the mean of its children); cells above levelmin always are (levels
       1..levelmin stay complete), cells at params->levelmax or deeper never are;
     - 2:1 balance, level by level from the finest up: a refined cell also refines the
       parent-level cells containing its 26 neighbours (2 per axis); nothing is needed
       beyond an outflow face, periodic faces wrap;
     - a cell exists iff its father is refined: the new oct list is the root oct plus the
       child oct of every refined cell (octs whose father is no longer refined are
       dropped, several levels at once if needed; new octs appear one level at a time).
   The three calls: amr_refine (the new oct list, on the device), amr_build_octree_device
   (the new tree from it) and amr_remap_state (the state on the new tree). */
typedef struct {
    double mass_thr;      /* refine a cell iff rho dx^3 > mass_thr (>= 0) */
    int32_t levelmax;     /* deepest level the new tree may have, levelmin .. 20 */
    int32_t pad;
} amr_refine_params;

/* Scratch bytes amr_refine needs for tree t (0 for a batch tree). */
size_t amr_refine_work_bytes(const amr_tree *t);

/* The refined tree's oct list from state d_u (conserved FP64 SoA of t): d_lxyz receives
   (level, ix, iy, iz) for *h_n octs in no particular order (cap >= 8 * t->noct + 1
   entries of 4 int32); h_level_counts[0 .. AMR_MAXLEV] the octs per level.  d_work:
   amr_refine_work_bytes(t) bytes, 256-byte aligned.  Synchronises.  AMR_EINVAL for bad
   arguments, AMR_ECAPACITY for short buffers, AMR_EUNBALANCED if t breaks the 2:1 rule. */
amr_status amr_refine(const amr_tree *t, const amr_refine_params *params, const double *d_u, void *d_work,
                      size_t work_bytes, int32_t *d_lxyz, int64_t cap, int64_t *h_level_counts, int64_t *h_n,
                      amr_stream stream);

/* amr_build_octree for an oct list already on the device, with its octs per level
   h_level_counts[0 .. AMR_MAXLEV] (checked against the list; AMR_EINVAL if they differ).
   Octree mode only (geom->n_inst == 0).  Synchronises. */
amr_status amr_build_octree_device_query(const amr_geom *geom, const int64_t *h_level_counts, size_t *tree_bytes,
                                         size_t *workspace_bytes);
amr_status amr_build_octree_device(const amr_geom *geom, const int32_t *d_oct_lxyz, const int64_t *h_level_counts,
                                   void *d_tree_mem, size_t tree_bytes, void *d_workspace, size_t workspace_bytes,
                                   amr_tree *out, amr_stream stream);

/* The state on t_new from the state on t_old (both FP64 SoA, distinct buffers): an oct
   present in both trees is copied; a new oct's cells are interpolated from their father
   cell in t_old with the ghost-cell formula
     U = U_F + sum_d s_d/4 minmod(U_F - U_{F-e_d}, U_{F+e_d} - U_F),
   which keeps the leaf totals of mass, momentum and energy.  t_new must come from
   amr_refine on t_old.  Asynchronous; a father missing from t_old writes
   AMR_EUNBALANCED to d_status (may be NULL). */
amr_status amr_remap_state(const amr_tree *t_old, const double *d_u_old, const amr_tree *t_new, double *d_u_new,
                           int32_t *d_status, amr_stream stream);

/* Global conservation diagnostics: the totals of the conserved variables over the leaf
   cells, computed on the device in FP64.  The level step of Table 1 (godunov_fine with
   its refluxing at coarse-fine faces; RAMSES' scheme, Teyssier 2002, on which Sec. 1
   builds) conserves them up to rounding in a periodic box; the paper prints no formula,
   the one computed is the plain definition.  d_totals (device double[nbox][2][5], nbox =
   n_inst in batch mode, else 1): [b][0][v] = sum over the leaf cells of box b of
   U_v dV and [b][1][v] = sum of |U_v| dV (v = rho, rho u, rho v, rho w, E; dV = dx_l^3,
   or (1/N)^3 for a box of N^3 cells), the second a scale for the drift of the first.
   The octs are cut into fixed chunks of 256 (per box), each summed in a fixed order (an
   oct's cells in cell order, then a fixed tree over the chunk), and each box's chunk
   sums are added in a fixed order: the result is the same bit for bit for every launch
   shape.  blocks: CTAs of the chunk pass (0 = 4 per SM); it changes the speed, not the
   result.  d_u: device FP64 SoA state (16-byte aligned); d_work: hydro_conservation_
   work_bytes(tree) bytes of device scratch, 256-byte aligned.  AMR_EINVAL for a missing
   or misaligned buffer or blocks < 0, AMR_ECAPACITY for a short d_work.  No atomics, no
   host synchronisation; asynchronous on the stream. */
size_t hydro_conservation_work_bytes(const amr_tree *tree);
amr_status hydro_conservation(const amr_tree *tree, const double *d_u, double *d_totals, void *d_work,
                              size_t work_bytes, int32_t blocks, amr_stream stream);

/* The FP32 path's conversions of state values, exposed so that they can be checked
   against IEEE conversions; the paper has no counterpart (its code is FP64 throughout).
   hydro_state_to_fp32: d_y[i] = the FP32 value the FP32 path reads for the FP64 state
   value d_x[i]: round to nearest, ties away from zero (IEEE rounds ties to even); |x|
   below 2^-126 gives a signed zero; |x| >= 2^128, +-Inf and NaN give a non-finite float
   of the same sign (+-Inf or a NaN).  hydro_state_from_fp32: d_x[i] = the FP64 value of
   the FP32 value d_y[i] (exact; +-Inf and NaN kept; FP32 denormals give a signed zero).
   Device arrays of n >= 0 elements; AMR_EINVAL for n < 0 or a NULL array with n > 0;
   asynchronous on the stream. */
amr_status hydro_state_to_fp32(const double *d_x, float *d_y, int64_t n, amr_stream stream);
amr_status hydro_state_from_fp32(const float *d_y, double *d_x, int64_t n, amr_stream stream);

/* Copy params->d_status and params->d_counters to the host (synchronises the device). */
amr_status amr_get_status(const hydro_params *params, int32_t *h_status, unsigned long long *h_counters);

const char *amr_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
