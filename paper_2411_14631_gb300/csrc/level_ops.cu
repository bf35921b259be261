// Per-level operations around the Godunov update: the CFL time step (newdt_fine,
// Table 1), refluxing + restriction, initial-state set-up, and the C entry points.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cstring>
#include <mutex>
#include "hydro_math.cuh"

namespace amr {
amr_status godunov_dispatch_fp32(const amr_tree *t, int level, const hydro_params *p, const double *u_old,
                                 double *u_new, double *reg, const double *dt, double *dt_next, cudaStream_t st);
amr_status harvest_dispatch(const amr_tree *t, const hydro_params *p, const double *u, const double *dt, double *out,
                            int64_t cap, int64_t stride, unsigned long long *count, cudaStream_t st);
amr_status godunov_dispatch_fp64(const amr_tree *t, int level, const hydro_params *p, const double *u_old,
                                 double *u_new, double *reg, const double *dt, double *dt_next, cudaStream_t st);

// warp minimum of positive doubles (compared as their bit patterns), then one atomic per warp
__device__ __forceinline__ void min_to(double *target, double v)
{
    unsigned long long b = v < DBL_MAX ? (unsigned long long)__double_as_longlong(v) : ~0ull;
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
        b = o < b ? o : b;
    }
    if ((threadIdx.x & 31) == 0 && b != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(target), b);
}

template <typename R>
// lscale >= 0: each leaf's candidate is multiplied by 2^(l - lscale), the coarsest
// level's step that gives this leaf its own step dt 2^-(l - lscale) (sub-cycling)
__global__ void k_courant(TreeView tv, int64_t cell0, const double *__restrict__ u, double gamma, double rf,
                          double pf, double cfl, double *dt, int lscale)
{
    const int64_t cell = cell0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    double cand = DBL_MAX;
    if (cell < tv.ncell && tv.son[cell] < 0) {
        double U[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = u[v * tv.ncell + cell];
        Prm<R> p;
        p.gamma = to_work<R>(gamma); p.rho_floor = to_work<R>(rf); p.p_floor = to_work<R>(pf);
        const int l = tv.lvl[cell >> 3];
        cand = cfl_candidate<R>(U, p, to_work<R>(cfl), to_work<R>(pow2(-l)));
        if (lscale >= 0) cand = scale_pow2(cand, l - lscale);
    }
    min_to(dt, cand);
}

// sub-cycling: the step of every level from the coarsest level's step
__global__ void k_dt_levels(const double *__restrict__ dt_base, int levelmin, double *dtl)
{
    const int l = threadIdx.x;
    if (l < AMR_MAXLEV + 2) dtl[l] = l > levelmin ? scale_pow2(*dt_base, levelmin - l) : *dt_base;
}

// sub-cycling: leaves of one level take the mean of two states (time interpolation)
__global__ void k_lerp_leaves(TreeView tv, int level, double *U, const double *__restrict__ N)
{
    const int64_t cell = tv.lvl_off[level] * 8 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (cell >= tv.lvl_off[level + 1] * 8 || tv.son[cell] >= 0) return;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const int64_t i = v * tv.ncell + cell;
        U[i] = 0.5 * (U[i] + N[i]);
    }
}

// batch mode: per-box CFL step (box cell ranges are multiples of 64, so a warp never
// straddles two boxes)
template <typename R>
__global__ void k_courant_batch(TreeView tv, const double *__restrict__ u, double gamma, double rf, double pf,
                                double cfl, double *dt)
{
    const int64_t cell = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    double cand = DBL_MAX;
    int b = 0;
    if (cell < tv.ncell) {
        b = tv.lvl[cell >> 3];
        double U[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = u[v * tv.ncell + cell];
        Prm<R> p;
        p.gamma = to_work<R>(gamma); p.rho_floor = to_work<R>(rf); p.p_floor = to_work<R>(pf);
        cand = cfl_candidate<R>(U, p, to_work<R>(cfl), to_work<R>(tv.inst_dx[b]));
    }
    b = __shfl_sync(0xffffffffu, b, 0);
    min_to(dt + b, cand);
}

// Coarse level l: leaf cells next to a refined cell take the fine fluxes from the
// register (-/+ dt/dx * 1/4 * sum of the four fine fluxes); refined cells become the
// mean of their eight children.  One cell; returns its CFL candidate (DBL_MAX if none).
template <typename R>
__device__ __forceinline__ double reflux_cell(const TreeView &tv, int level, int64_t cell,
                                              const double *__restrict__ reg, double *u, const double *dtp,
                                              bool want_dt, double gamma, double rf, double pf, double cfl,
                                              int restrict_all)
{
    double cand = DBL_MAX;
    const int64_t o = cell >> 3;
    const int c = int(cell & 7);
    const int32_t s = tv.son[cell];
    if (s >= 0) {
        if (restrict_all || !tv.fused[s]) {               // else restricted by the update kernel
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double sum = 0.0;
#pragma unroll
                for (int q = 0; q < 8; ++q) sum += u[v * tv.ncell + int64_t(s) * 8 + q];
                u[v * tv.ncell + cell] = 0.125 * sum;
            }
        }
    } else if (reg && level >= tv.levelmin) {
        const double lam = scale_pow2(*dtp, level);   // dt / dx, exact
        double U[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = u[v * tv.ncell + cell];
        bool hit = false;
        for (int f = 0; f < 6; ++f) {
            const int d = f >> 1, side = f & 1;
            int64_t nb;
            if (((c >> d) & 1) != side) {
                nb = o * 8 + (c ^ (1 << d));
            } else {
                const int32_t N = tv.nbor[6 * o + f];
                if (N < 0) continue;                      // outflow face of the box
                const int32_t so = tv.son[N];
                if (so < 0) continue;                     // coarser neighbour
                nb = int64_t(so) * 8 + (c ^ (1 << d));
            }
            const int32_t fo = tv.son[nb];
            if (fo < 0) continue;
            const int opp = 2 * d + (1 - side);
            const double *rrow = reg + ((int64_t(fo) - tv.reg_base) * 6 + opp) * NV;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double corr = 0.25 * rrow[v];
                U[v] = side ? U[v] - lam * corr : U[v] + lam * corr;
            }
            hit = true;
        }
        if (hit) {
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v * tv.ncell + cell] = U[v];
            if (want_dt) {
                Prm<R> p;
                p.gamma = to_work<R>(gamma); p.rho_floor = to_work<R>(rf); p.p_floor = to_work<R>(pf);
                cand = cfl_candidate<R>(U, p, to_work<R>(cfl), to_work<R>(pow2(-level)));
            }
        }
    }
    return cand;
}

template <typename R>
__global__ void k_reflux(TreeView tv, int level, const double *__restrict__ reg, double *u, const double *dtp,
                         double *dt_next, double gamma, double rf, double pf, double cfl, int restrict_all)
{
    const int64_t cell = tv.lvl_off[level] * 8 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    double cand = DBL_MAX;
    if (cell < tv.lvl_off[level + 1] * 8)
        cand = reflux_cell<R>(tv, level, cell, reg, u, dtp, dt_next != nullptr, gamma, rf, pf, cfl, restrict_all);
    if (dt_next) min_to(dt_next, cand);
}

// The same pass over the cells of the tree's work list of one level only (the others have
// nothing to do when not everything is restricted).
template <typename R>
__global__ void k_reflux_list(TreeView tv, int level, const int32_t *__restrict__ list, int64_t n,
                              const double *__restrict__ reg, double *u, const double *dtp, double *dt_next,
                              double gamma, double rf, double pf, double cfl)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    double cand = DBL_MAX;
    if (i < n) cand = reflux_cell<R>(tv, level, list[i], reg, u, dtp, dt_next != nullptr, gamma, rf, pf, cfl, 0);
    if (dt_next) min_to(dt_next, cand);
}

// Restriction of complete levels: one CTA per oct O of level L restricts the nlev levels
// L + nlev - 1 .. L of O's subtree (nlev <= 3), the deepest from level L + nlev in global
// memory, the others from the values it has just formed (kept in shared memory).  Every
// cell is the mean of its eight children summed in cell order, as in k_reflux.  Valid
// where levels L .. L + nlev are complete (every cell of levels L .. L + nlev - 1 refined):
// the levels below the deepest complete one.
__global__ void __launch_bounds__(256) k_restrict_complete(TreeView tv, int L, int nlev, double *u)
{
    __shared__ int32_t son1[8], son2[64], son3[512];   // son octs of O's cells, of theirs, ...
    __shared__ double v2[NV][512], v1[NV][64];
    const int t = threadIdx.x;
    const int64_t O = tv.lvl_off[L] + blockIdx.x;
    auto mean8 = [&](const double *c) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += c[q];
        return 0.125 * acc;
    };
    if (nlev >= 2 && t < 8) son1[t] = tv.son[O * 8 + t];
    __syncthreads();
    if (nlev == 3 && t < 64) son2[t] = tv.son[int64_t(son1[t >> 3]) * 8 + (t & 7)];
    __syncthreads();
    if (nlev == 3) {
        for (int j = t; j < 512; j += blockDim.x) son3[j] = tv.son[int64_t(son2[j >> 3]) * 8 + (j & 7)];
        __syncthreads();
        // level L+2: the 512 cells of the 64 octs son2[], from their sons son3[] at level L+3
#pragma unroll 2
        for (int w = t; w < 512 * NV; w += blockDim.x) {
            const int v = w >> 9, j = w & 511;
            const double2 *src = reinterpret_cast<const double2 *>(u + v * tv.ncell + int64_t(son3[j]) * 8);
            double c[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const double2 q2 = src[h];
                c[2 * h] = q2.x;
                c[2 * h + 1] = q2.y;
            }
            const double m = mean8(c);
            u[v * tv.ncell + int64_t(son2[j >> 3]) * 8 + (j & 7)] = m;
            v2[v][j] = m;
        }
        __syncthreads();
    }
    if (nlev >= 2) {
        // level L+1: the 64 cells of the 8 octs son1[]
        for (int w = t; w < 64 * NV; w += blockDim.x) {
            const int v = w >> 6, k = w & 63;
            const int64_t cell = int64_t(son1[k >> 3]) * 8 + (k & 7);
            double c[8];
            if (nlev == 3) {
#pragma unroll
                for (int q = 0; q < 8; ++q) c[q] = v2[v][k * 8 + q];
            } else {
                const int64_t s2 = tv.son[cell];
#pragma unroll
                for (int q = 0; q < 8; ++q) c[q] = u[v * tv.ncell + s2 * 8 + q];
            }
            const double m = mean8(c);
            u[v * tv.ncell + cell] = m;
            v1[v][k] = m;
        }
        __syncthreads();
    }
    // level L: O's eight cells
    if (t < 8 * NV) {
        const int v = t >> 3, c0 = t & 7;
        double c[8];
        if (nlev >= 2) {
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = v1[v][c0 * 8 + q];
        } else {
            const int64_t s1 = tv.son[O * 8 + c0];
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = u[v * tv.ncell + s1 * 8 + q];
        }
        u[v * tv.ncell + O * 8 + c0] = mean8(c);
    }
}

__global__ void k_prim_to_cons(int64_t ncell, const double *__restrict__ w, double *u, double gamma)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= ncell) return;
    const double rho = w[i], vx = w[ncell + i], vy = w[2 * ncell + i], vz = w[3 * ncell + i], p = w[4 * ncell + i];
    u[i] = rho;
    u[ncell + i] = rho * vx;
    u[2 * ncell + i] = rho * vy;
    u[3 * ncell + i] = rho * vz;
    u[4 * ncell + i] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz);
}

__global__ void k_cons_to_prim(int64_t ncell, const double *__restrict__ u, double *w, double gamma, double rf, double pf)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= ncell) return;
    double U[NV], W[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = u[v * ncell + i];
    Prm<double> p;
    p.gamma = gamma; p.rho_floor = rf; p.p_floor = pf;
    cons_to_prim(U, p, W);
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v * ncell + i] = W[v];
}

__global__ void k_to_fp32(int64_t n, const double *__restrict__ x, float *__restrict__ y)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = d2f_bits(x[i]);
}

__global__ void k_from_fp32(int64_t n, const float *__restrict__ y, double *__restrict__ x)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] = f2d_bits(y[i]);
}

static amr_status check(const amr_tree *t, const hydro_params *p)
{
    if (!t || !p || t->noct <= 0) return AMR_EINVAL;
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->rho_floor > 0.0) || !(p->p_floor > 0.0)) return AMR_EINVAL;
    if (p->riemann < AMR_RIEMANN_HLLC || p->riemann > AMR_RIEMANN_MLP_SEEDED) return AMR_EINVAL;
    if (p->precision != AMR_PREC_FP64 && p->precision != AMR_PREC_FP32) return AMR_EINVAL;
    if (p->tile < 0 || p->tile > 2) return AMR_EINVAL;
    if (p->limiter != AMR_LIMITER_MINMOD && p->limiter != AMR_LIMITER_MC) return AMR_EINVAL;
    if (p->col_kernel < 0 || p->col_kernel > 2 || p->col_seg < 0 || (p->col_seg & 1)) return AMR_EINVAL;
    return AMR_OK;
}

static amr_status reflux_launch(const amr_tree *t, int level, const hydro_params *p, const double *reg, double *u,
                                const double *dt, double *dt_next, cudaStream_t st, int restrict_all = 0)
{
    const TreeView tv = make_view(t);
    if (!restrict_all && t->reflux_cell && level >= t->levelmin && level < t->levelmax) {
        // only the level's cells on the work list
        const int64_t a = t->reflux_off[level], n = t->reflux_off[level + 1] - a;
        if (n <= 0) return AMR_OK;
        const unsigned nb = unsigned((n + 255) / 256);
        if (p->precision == AMR_PREC_FP32)
            k_reflux_list<float><<<nb, 256, 0, st>>>(tv, level, t->reflux_cell + a, n, reg, u, dt, dt_next, p->gamma,
                                                     p->rho_floor, p->p_floor, p->cfl);
        else
            k_reflux_list<double><<<nb, 256, 0, st>>>(tv, level, t->reflux_cell + a, n, reg, u, dt, dt_next,
                                                      p->gamma, p->rho_floor, p->p_floor, p->cfl);
        AMR_CUDA_TRY(cudaGetLastError());
        return AMR_OK;
    }
    const int64_t nc = (t->lvl_off[level + 1] - t->lvl_off[level]) * 8;
    if (nc <= 0) return AMR_OK;
    const unsigned nb = unsigned((nc + 255) / 256);
    if (p->precision == AMR_PREC_FP32)
        k_reflux<float><<<nb, 256, 0, st>>>(tv, level, reg, u, dt, dt_next, p->gamma, p->rho_floor, p->p_floor, p->cfl,
                                            restrict_all);
    else
        k_reflux<double><<<nb, 256, 0, st>>>(tv, level, reg, u, dt, dt_next, p->gamma, p->rho_floor, p->p_floor, p->cfl,
                                             restrict_all);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

// Restriction of the complete levels below lo_end (levels lo_end - 1 .. 1), three levels
// per launch from the top down.
static amr_status restrict_complete_launch(const amr_tree *t, int lo_end, double *u, cudaStream_t st)
{
    const TreeView tv = make_view(t);
    for (int top = lo_end - 1; top >= 1;) {
        const int nlev = top >= 3 ? 3 : top;
        const int L = top - nlev + 1;
        const int64_t nb = t->lvl_off[L + 1] - t->lvl_off[L];
        if (nb > 0) {
            k_restrict_complete<<<unsigned(nb), 256, 0, st>>>(tv, L, nlev, u);
            AMR_CUDA_TRY(cudaGetLastError());
        }
        top = L - 1;
    }
    return AMR_OK;
}

}  // namespace amr

using namespace amr;

extern "C" size_t hydro_flux_reg_bytes(const amr_tree *t)
{
    if (!t) return 0;
    return reg_total_bytes(t);
}

extern "C" amr_status hydro_init_from_prim(const amr_tree *t, const hydro_params *p, const double *d_w, double *d_u,
                                           amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_w || !d_u) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t nc = 8 * t->noct;
    k_prim_to_cons<<<unsigned((nc + 255) / 256), 256, 0, st>>>(nc, d_w, d_u, p->gamma);
    AMR_CUDA_TRY(cudaGetLastError());
    for (int l = t->levelmax - 1; l >= 1; --l) {
        amr_status r = reflux_launch(t, l, p, nullptr, d_u, nullptr, nullptr, st, 1);
        if (r != AMR_OK) return r;
    }
    return AMR_OK;
}

extern "C" amr_status hydro_prim_of_state(const amr_tree *t, const hydro_params *p, const double *d_u, double *d_w,
                                          amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_w || !d_u) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t nc = 8 * t->noct;
    k_cons_to_prim<<<unsigned((nc + 255) / 256), 256, 0, st>>>(nc, d_u, d_w, p->gamma, p->rho_floor, p->p_floor);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status hydro_courant(const amr_tree *t, const hydro_params *p, const double *d_u, double *d_dt,
                                    amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_u || !d_dt) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const TreeView tv = make_view(t);
    if (t->n_inst > 0) {
        AMR_CUDA_TRY(cudaMemsetAsync(d_dt, 0x7F, sizeof(double) * size_t(t->n_inst), st));
        const unsigned nb = unsigned((8 * t->noct + 255) / 256);
        if (p->precision == AMR_PREC_FP32)
            k_courant_batch<float><<<nb, 256, 0, st>>>(tv, d_u, p->gamma, p->rho_floor, p->p_floor, p->cfl, d_dt);
        else
            k_courant_batch<double><<<nb, 256, 0, st>>>(tv, d_u, p->gamma, p->rho_floor, p->p_floor, p->cfl, d_dt);
        AMR_CUDA_TRY(cudaGetLastError());
        return AMR_OK;
    }
    AMR_CUDA_TRY(cudaMemsetAsync(d_dt, 0x7F, sizeof(double), st));
    const int64_t c0 = t->lvl_off[t->levelmin] * 8, nc = 8 * t->noct - c0;
    const unsigned nb = unsigned((nc + 255) / 256);
    if (p->precision == AMR_PREC_FP32)
        k_courant<float><<<nb, 256, 0, st>>>(tv, c0, d_u, p->gamma, p->rho_floor, p->p_floor, p->cfl, d_dt, -1);
    else
        k_courant<double><<<nb, 256, 0, st>>>(tv, c0, d_u, p->gamma, p->rho_floor, p->p_floor, p->cfl, d_dt, -1);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

// the argument checks of the update (also made by hydro_step before it writes anything)
static amr_status godunov_args(const amr_tree *t, int level, const hydro_params *p, const double *d_u_old,
                               const double *d_u_new, const double *d_flux_reg, const double *d_dt)
{
    if (check(t, p) != AMR_OK || !d_u_old || !d_u_new || !d_dt) return AMR_EINVAL;
    if ((p->riemann == AMR_RIEMANN_MLP || p->riemann == AMR_RIEMANN_MLP_SEEDED) &&
        (p->precision != AMR_PREC_FP32 || !p->mlp_weights))
        return AMR_EINVAL;
    if (level != -1 && (level < t->levelmin || level > t->levelmax)) return AMR_EINVAL;
    if (t->levelmax > t->levelmin && !d_flux_reg) return AMR_EINVAL;
    return AMR_OK;
}

extern "C" amr_status hydro_godunov_level(const amr_tree *t, int level, const hydro_params *p, const double *d_u_old,
                                          double *d_u_new, double *d_flux_reg, const double *d_dt, double *d_dt_next,
                                          amr_stream stream)
{
    if (godunov_args(t, level, p, d_u_old, d_u_new, d_flux_reg, d_dt) != AMR_OK) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->precision == AMR_PREC_FP32)
        return godunov_dispatch_fp32(t, level, p, d_u_old, d_u_new, d_flux_reg, d_dt, d_dt_next, st);
    return godunov_dispatch_fp64(t, level, p, d_u_old, d_u_new, d_flux_reg, d_dt, d_dt_next, st);
}

extern "C" amr_status hydro_reflux_level(const amr_tree *t, int level, const hydro_params *p, const double *d_flux_reg,
                                         double *d_u_new, const double *d_dt, double *d_dt_next, amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_u_new || !d_dt) return AMR_EINVAL;
    if (level < 1 || level >= t->levelmax) return AMR_EINVAL;
    if (level >= t->levelmin && !d_flux_reg) return AMR_EINVAL;
    return reflux_launch(t, level, p, d_flux_reg, d_u_new, d_dt, d_dt_next, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" amr_status reflux_level(const amr_tree *t, int level, const hydro_params *p, const double *d_flux_reg,
                                   double *d_u_new, const double *d_dt, double *d_dt_next, amr_stream stream)
{
    return hydro_reflux_level(t, level, p, d_flux_reg, d_u_new, d_dt, d_dt_next, stream);
}

// ---- sub-cycled step -----------------------------------------------------------------
static amr_status sc_advance(const amr_tree *t, const hydro_params *p, int c, double *U, double *N, double *reg,
                             double *dtl, cudaStream_t st)
{
    amr_status r = hydro_godunov_level(t, c, p, U, N, reg, dtl + c, nullptr, reinterpret_cast<amr_stream>(st));
    if (r != AMR_OK) return r;
    if (c < t->levelmax) {
        if ((r = sc_advance(t, p, c + 1, U, N, reg, dtl, st)) != AMR_OK) return r;
        // ghosts of the second fine step: coarse leaves interpolated in time plus the first
        // fine step's correction; refined cells restricted from the fine level
        const int64_t nc = (t->lvl_off[c + 1] - t->lvl_off[c]) * 8;
        if (nc > 0) {
            k_lerp_leaves<<<unsigned((nc + 255) / 256), 256, 0, st>>>(make_view(t), c, U, N);
            AMR_CUDA_TRY(cudaGetLastError());
        }
        if ((r = reflux_launch(t, c, p, reg, U, dtl + c + 1, nullptr, st, 1)) != AMR_OK) return r;
        if ((r = reflux_launch(t, c, p, reg, N, dtl + c + 1, nullptr, st, 0)) != AMR_OK) return r;
        if ((r = sc_advance(t, p, c + 1, U, N, reg, dtl, st)) != AMR_OK) return r;
        if ((r = reflux_launch(t, c, p, reg, N, dtl + c + 1, nullptr, st, 0)) != AMR_OK) return r;
    }
    // the level's new state becomes current (its cells are contiguous in each variable)
    const int64_t c0 = t->lvl_off[c] * 8, n = (t->lvl_off[c + 1] - t->lvl_off[c]) * 8, ncell = 8 * t->noct;
    if (n > 0)
        for (int v = 0; v < NV; ++v)
            AMR_CUDA_TRY(cudaMemcpyAsync(U + v * ncell + c0, N + v * ncell + c0, size_t(n) * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
    return AMR_OK;
}

extern "C" amr_status hydro_courant_levels(const amr_tree *t, const hydro_params *p, const double *d_u, double *d_dt,
                                           amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_u || !d_dt || t->n_inst != 0) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const TreeView tv = make_view(t);
    AMR_CUDA_TRY(cudaMemsetAsync(d_dt, 0x7F, sizeof(double), st));
    const int64_t c0 = t->lvl_off[t->levelmin] * 8, nc = 8 * t->noct - c0;
    const unsigned nb = unsigned((nc + 255) / 256);
    if (p->precision == AMR_PREC_FP32)
        k_courant<float><<<nb, 256, 0, st>>>(tv, c0, d_u, p->gamma, p->rho_floor, p->p_floor, p->cfl, d_dt,
                                             t->levelmin);
    else
        k_courant<double><<<nb, 256, 0, st>>>(tv, c0, d_u, p->gamma, p->rho_floor, p->p_floor, p->cfl, d_dt,
                                              t->levelmin);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status hydro_step_subcycled(const amr_tree *t, const hydro_params *p, double *d_u, double *d_scratch,
                                           double *d_flux_reg, double *d_dt, double *d_dt_levels, amr_stream stream)
{
    if (check(t, p) != AMR_OK || t->n_inst != 0 || !d_u || !d_scratch || !d_dt || !d_dt_levels || d_u == d_scratch)
        return AMR_EINVAL;
    if (t->levelmax > t->levelmin && !d_flux_reg) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    amr_status r = hydro_courant_levels(t, p, d_u, d_dt, stream);
    if (r != AMR_OK) return r;
    k_dt_levels<<<1, 32, 0, st>>>(d_dt, t->levelmin, d_dt_levels);
    AMR_CUDA_TRY(cudaGetLastError());
    if ((r = sc_advance(t, p, t->levelmin, d_u, d_scratch, d_flux_reg, d_dt_levels, st)) != AMR_OK) return r;
    for (int l = t->levelmin - 1; l >= 1; --l)
        if ((r = reflux_launch(t, l, p, nullptr, d_u, d_dt_levels, nullptr, st, 1)) != AMR_OK) return r;
    return AMR_OK;
}

extern "C" amr_status hydro_restrict_complete(const amr_tree *t, double *d_u, amr_stream stream)
{
    if (!t || !d_u) return AMR_EINVAL;
    if (t->n_inst > 0) return AMR_OK;
    const int gl = t->grid_level, lstop = gl >= 2 ? gl - 1 : 1;
    if (lstop <= 1) return AMR_OK;
    return restrict_complete_launch(t, lstop, d_u, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" amr_status hydro_step(const amr_tree *t, const hydro_params *p, const double *d_u_old, double *d_u_new,
                                 double *d_flux_reg, const double *d_dt, double *d_dt_next, amr_stream stream)
{
    if (godunov_args(t, -1, p, d_u_old, d_u_new, d_flux_reg, d_dt) != AMR_OK) return AMR_EINVAL;
    if (d_dt_next)
        AMR_CUDA_TRY(cudaMemsetAsync(d_dt_next, 0x7F, sizeof(double) * size_t(t->n_inst > 0 ? t->n_inst : 1),
                                     reinterpret_cast<cudaStream_t>(stream)));
    amr_status r = hydro_godunov_level(t, -1, p, d_u_old, d_u_new, d_flux_reg, d_dt, d_dt_next, stream);
    if (r != AMR_OK) return r;
    // reflux + restriction per level from the finest up to the level above the deepest
    // complete one; the complete levels below that are pure restrictions, three per launch
    const int gl = t->n_inst > 0 ? 0 : t->grid_level;
    const int lstop = gl >= 2 ? gl - 1 : 1;
    // a tree complete up to its finest level: the update kernel restricted every father of
    // the finest level (all its octs are flagged fused) and level gl-1 has no leaf, so that
    // level's pass would find no work
    const int lfirst = (gl >= 2 && gl == t->levelmax) ? gl - 2 : t->levelmax - 1;
    for (int l = lfirst; l >= lstop; --l) {
        r = reflux_launch(t, l, p, d_flux_reg, d_u_new, d_dt, d_dt_next, reinterpret_cast<cudaStream_t>(stream));
        if (r != AMR_OK) return r;
    }
    if (lstop > 1 && !p->defer_restriction)
        return restrict_complete_launch(t, lstop, d_u_new, reinterpret_cast<cudaStream_t>(stream));
    return AMR_OK;
}

// ---- hydro_step with the flux register in library-owned device memory ----------------
// For callers that cannot allocate device memory when they step.  The register is a
// fixed file-scope device array; host code must not pass the symbol itself to a kernel
// (in host code it names a host-side stand-in), so its device address is looked up once
// per device, with that device current, and cached.  The cache is an atomic per device;
// the first look-up on a device runs under a mutex, so concurrent first calls from
// several host threads are safe.
static __device__ __align__(256) double g_static_reg[size_t(AMR_STATIC_REG_MAX_OCTS) * 6 * NV];
static std::atomic<double *> g_static_reg_addr[256];
static std::mutex g_static_reg_mu;

static amr_status static_reg_address(int dev, double **out)
{
    double *a = g_static_reg_addr[dev].load(std::memory_order_acquire);
    if (!a) {
        std::lock_guard<std::mutex> lock(g_static_reg_mu);
        a = g_static_reg_addr[dev].load(std::memory_order_relaxed);
        if (!a) {
            void *addr = nullptr;
            AMR_CUDA_TRY(cudaGetSymbolAddress(&addr, g_static_reg));
            a = static_cast<double *>(addr);
            g_static_reg_addr[dev].store(a, std::memory_order_release);
        }
    }
    *out = a;
    return AMR_OK;
}

extern "C" amr_status hydro_step_static_scratch(const amr_tree *t, const hydro_params *p, const double *d_u_old,
                                                double *d_u_new, const double *d_dt, double *d_dt_next,
                                                amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_u_old || !d_u_new || !d_dt) return AMR_EINVAL;
    if (t->noct - t->reg_base > AMR_STATIC_REG_MAX_OCTS ||
        reg_total_bytes(t) > size_t(AMR_STATIC_REG_MAX_OCTS) * 6 * NV * sizeof(double))
        return AMR_ECAPACITY;
    int dev = 0;
    AMR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return AMR_EINVAL;
    double *reg = nullptr;
    const amr_status r = static_reg_address(dev, &reg);
    if (r != AMR_OK) return r;
    return hydro_step(t, p, d_u_old, d_u_new, reg, d_dt, d_dt_next, stream);
}

extern "C" amr_status hydro_harvest_faces(const amr_tree *t, const hydro_params *p, const double *d_u,
                                          const double *d_dt, double *d_states, int64_t capacity, int64_t stride,
                                          unsigned long long *d_count, amr_stream stream)
{
    if (check(t, p) != AMR_OK || !d_u || !d_dt || !d_states || !d_count || capacity < 0 || stride < 1)
        return AMR_EINVAL;
    if (t->n_inst > 0) return AMR_EINVAL;   // octree runs only
    return harvest_dispatch(t, p, d_u, d_dt, d_states, capacity, stride, d_count,
                            reinterpret_cast<cudaStream_t>(stream));
}

extern "C" amr_status hydro_state_to_fp32(const double *d_x, float *d_y, int64_t n, amr_stream stream)
{
    if (n < 0 || (n > 0 && (!d_x || !d_y))) return AMR_EINVAL;
    if (n == 0) return AMR_OK;
    const int64_t nb = (n + 255) / 256;
    k_to_fp32<<<unsigned(nb < 4096 ? nb : 4096), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n, d_x, d_y);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status hydro_state_from_fp32(const float *d_y, double *d_x, int64_t n, amr_stream stream)
{
    if (n < 0 || (n > 0 && (!d_x || !d_y))) return AMR_EINVAL;
    if (n == 0) return AMR_OK;
    const int64_t nb = (n + 255) / 256;
    k_from_fp32<<<unsigned(nb < 4096 ? nb : 4096), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n, d_y, d_x);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status amr_get_status(const hydro_params *p, int32_t *h_status, unsigned long long *h_counters)
{
    if (!p) return AMR_EINVAL;
    if (h_status) {
        *h_status = 0;
        if (p->d_status) AMR_CUDA_TRY(cudaMemcpy(h_status, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    if (h_counters) {
        std::memset(h_counters, 0, sizeof(unsigned long long) * AMR_NCOUNTERS);
        if (p->d_counters)
            AMR_CUDA_TRY(cudaMemcpy(h_counters, p->d_counters, sizeof(unsigned long long) * AMR_NCOUNTERS,
                                    cudaMemcpyDeviceToHost));
    }
    return AMR_OK;
}

extern "C" const char *amr_status_string(int s)
{
    switch (s) {
    case AMR_OK: return "ok";
    case AMR_EINVAL: return "invalid argument";
    case AMR_EUNBALANCED: return "octree violates the 2:1 rule";
    case AMR_ECAPACITY: return "caller buffer too small";
    case AMR_ECUDA: return "CUDA runtime error";
    case AMR_ETIMEOUT: return "device wait timed out";
    case AMR_ENONPHYSICAL: return "non-physical state (exact-solver vacuum or a non-finite cell)";
    case AMR_ENOCONV: return "iteration did not converge";
    case AMR_EBREAKDOWN: return "Krylov iteration broke down";
    default: return "unknown status";
    }
}
