// godunov_fine (Table 1 of arXiv 2411.14631) on GB300: a CTA updates one tile of sibling
// octs at a time, looping over tiles.  A depth-D tile is the 2^D x 2^D x 2^D block of level-l octs below one
// level-(l-D) oct; its ghosted stencil is (2^D+2)^3 oct slots = (2^(D+1)+4)^3 cells.
// Phases, all through shared memory:
//   1 gather the stencil cells that phase 2 reads from u_old (FP64 loads; a slot is a
//     level-l oct, a coarse leaf cell interpolated to its eight children, a clamped
//     outflow ghost, or unused; no corner slot is read), convert to primitives in the
//     working precision R;
//   2 MinMod slopes and the MUSCL-Hancock half-step predictor for the updated cells and
//     their face neighbours (the cells the faces read);
//   3 one Riemann solve per face touching an updated cell;
//   4 FP64 conservative update of the tile's existing octs, fused CFL candidate for the
//     next step, and flux-register rows for oct sides facing coarser leaves.
#pragma once
#include <cfloat>
#include <type_traits>
#include "hydro_math.cuh"
#include "mlp_warp.cuh"
#include "godunov_col.cuh"
#include "godunov_pen.cuh"

namespace amr {

constexpr int32_t UNNEEDED_SLOT = INT32_MIN + 1;

template <int D> struct Geo {
    static constexpr int NS = (1 << D) + 2;      // slots per axis
    static constexpr int NSLOT = NS * NS * NS;
    static constexpr int C = 2 * NS;             // stencil cells per axis
    static constexpr int NC = C * C * C;
    static constexpr int P = C - 2;              // predicted cells per axis (stencil 1..C-2)
    static constexpr int NP = P * P * P;
    static constexpr int CI = 1 << (D + 1);      // updated cells per axis (stencil 2..C-3)
    static constexpr int NI = CI * CI * CI;
    static constexpr int NF = (CI + 1) * CI * CI;  // faces per direction
    static constexpr int OI = 1 << D;            // interior oct slots per axis
    // What the phases read.  The faces need the predicted states of the updated cells and of
    // their face neighbours (no edge or corner cells of the predicted block): NPN cells.
    // Those read their face neighbours: the stencil cells at most two cells outside the
    // updated block in one axis, or one cell outside in two axes.  By slot: every cell of
    // the interior and face slots (NFULL), the two cells next to the interior of each edge
    // slot (NEDGE), nothing of the corner slots.
    static constexpr int NPN = CI * CI * CI + 6 * CI * CI;
    static constexpr int NFULL = OI * OI * OI + 6 * OI * OI;
    static constexpr int NEDGE = 12 * OI;
    static constexpr int NG = 8 * NFULL + 2 * NEDGE;
};

struct GArgs {
    TreeView tv;
    const int32_t *tile_root, *tile_slot;
    const int32_t *tile_inst;    // batch mode: box of each tile (dt, dt_next are per box)
    int64_t tile_off[AMR_MAXLEV + 2];
    int64_t t_begin, t_end;
    int32_t lfirst, llast;                 // levels covered by [t_begin, t_end)
    const double *u_old;
    double *u_new, *reg;
    const double *dt;
    double *dt_next;
    double gamma, rho_floor, p_floor, cfl;
    int32_t *status;
    unsigned long long *counters;
    const void *mlp;          // packed surrogate weights (RS == AMR_RIEMANN_MLP)
    float mlp_tol;            // residual acceptance threshold
    int32_t mlp_seed;         // 1: the network's p* seeds Newton at every face (no acceptance test)
    int32_t limiter;          // AMR_LIMITER_* of the slopes
    const void *ghost;        // if set: interpolated children of the ghost fathers, R [NV][ghost_stride]
    int64_t ghost_stride;     // 8 * n_ghost
    double *harvest;          // if set: sampled face states [cap][6] are written, u_new is not
    int64_t harvest_cap, harvest_stride;
    unsigned long long *harvest_count;
};

// value of a neighbour of coarse leaf cell F (level lc, coordinates X) along axis d,
// side s = +-1: the level-lc cell there, or the coarser leaf containing it
__device__ __forceinline__ int64_t coarse_neighbour(const TreeView &tv, int64_t oF, const int64_t X[3], int lc,
                                                    int d, int s)
{
    int64_t P[3] = {X[0], X[1], X[2]};
    P[d] += s;
    const int64_t n = int64_t(1) << lc;
    if (P[d] < 0 || P[d] >= n) {
        if (tv.bc[2 * d + (s > 0)] == AMR_BC_PERIODIC) P[d] = (P[d] + n) % n;
        else P[d] = X[d];                       // outflow: clamp at the cell's own level
    }
    const int cc = int(P[0] & 1) + 2 * int(P[1] & 1) + 4 * int(P[2] & 1);
    if ((P[0] >> 1) == tv.ix[oF] && (P[1] >> 1) == tv.iy[oF] && (P[2] >> 1) == tv.iz[oF]) return oF * 8 + cc;
    const int32_t N = tv.nbor[6 * oF + 2 * d + (s > 0)];   // father-level neighbour of oF
    if (N < 0) return oF * 8 + (int(X[0] & 1) + 2 * int(X[1] & 1) + 4 * int(X[2] & 1));              // unreachable for a valid tree; stay in bounds
    const int32_t so = tv.son[N];
    return so >= 0 ? int64_t(so) * 8 + cc : int64_t(N);
}

// The interpolation of coarse leaf cell F to its children, on conserved variables in the
// working precision R (FP64 values read from the state): its value uc and its MinMod
// slopes m[d] = minmod(U_F - U_{F-e_d}, U_{F+e_d} - U_F) ...
template <typename R>
__device__ __forceinline__ void interp_slopes(const TreeView &tv, const double *__restrict__ u, int64_t F,
                                              R uc[NV], R m[3][NV])
{
    const int64_t oF = F >> 3;
    const int cf = int(F & 7);
    const int lc = tv.lvl[oF];
    const int64_t X[3] = {2 * int64_t(tv.ix[oF]) + (cf & 1), 2 * int64_t(tv.iy[oF]) + ((cf >> 1) & 1),
                          2 * int64_t(tv.iz[oF]) + ((cf >> 2) & 1)};
    int64_t nm[3], np[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        nm[d] = coarse_neighbour(tv, oF, X, lc, d, -1);
        np[d] = coarse_neighbour(tv, oF, X, lc, d, +1);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        uc[v] = to_work<R>(u[v * tv.ncell + F]);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            m[d][v] = minmod(uc[v] - to_work<R>(u[v * tv.ncell + nm[d]]), to_work<R>(u[v * tv.ncell + np[d]]) - uc[v]);
    }
}

// ... and child c of it: U_F + sum_d s_d/4 m[d], s_d = +1 on the upper side of axis d
template <typename R>
__device__ __forceinline__ R interp_value(R uc, const R m[3][NV], int v, int c)
{
    R r = uc;
#pragma unroll
    for (int d = 0; d < 3; ++d) r = r + (((c >> d) & 1) ? R(0.25) * m[d][v] : -R(0.25) * m[d][v]);
    return r;
}

template <typename R>
__device__ void interp_child(const TreeView &tv, const double *__restrict__ u, int64_t F, int c, R out[NV])
{
    R uc[NV], m[3][NV];
    interp_slopes<R>(tv, u, F, uc, m);
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = interp_value<R>(uc[v], m, v, c);
}

// The children of ghost fathers [g0, g1), all eight per father, into out[v][8 g + c]: the
// values the tiles of the next finer level read in place of absent octs.  One thread per
// father: the slopes are found once for its eight children.
template <typename R>
__global__ void __launch_bounds__(256) k_ghost(TreeView tv, const double *__restrict__ u, int64_t g0, int64_t g1,
                                               int64_t stride, R *__restrict__ out)
{
    const int64_t g = g0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (g >= g1) return;
    R uc[NV], m[3][NV];
    interp_slopes<R>(tv, u, tv.ghost_cell[g], uc, m);
    // a father's eight children are 8 consecutive values (32 or 64 bytes from a multiple
    // of that offset): 16-byte stores when the buffer is 16-byte aligned
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        R ch[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) ch[c] = interp_value<R>(uc[v], m, v, c);
        R *o = out + v * stride + 8 * g;
        if (vec) {
            if constexpr (sizeof(R) == 4) {
                reinterpret_cast<float4 *>(o)[0] = make_float4(ch[0], ch[1], ch[2], ch[3]);
                reinterpret_cast<float4 *>(o)[1] = make_float4(ch[4], ch[5], ch[6], ch[7]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) reinterpret_cast<double2 *>(o)[k] = make_double2(ch[2 * k], ch[2 * k + 1]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) o[c] = ch[c];
        }
    }
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

// threads per CTA: depth-1 tiles (512 stencil cells) 128, depth-2 tiles (1728) 512.  A
// depth-2 CTA's shared memory admits one per SM, so it may take every register (no
// spills); the FP32 depth-1 update (HLLC or exact) fits 64 registers, eight CTAs per SM;
// the FP64 and surrogate variants keep the compiler's own budget.
template <int D> __host__ __device__ constexpr int threads_for() { return D == 1 ? 128 : 512; }
template <typename R, int D, int RS> constexpr int min_ctas_for()
{
    return (D == 1 && sizeof(R) == 4 && RS != AMR_RIEMANN_MLP) ? 8 : 1;
}

template <typename R, int D, int RS>
struct Smem {
    using G = Geo<D>;
    R W[NV][G::NC];                 // stencil primitives; later reused for fluxes
    R Q[4 * NV][G::NP];             // predicted state (5) + slopes (3 x 5)
    int32_t slot[G::NSLOT];
    uint8_t ref[G::NSLOT];
    // surrogate staging, per warp: 32 faces x 8 features, then 32 x 2 outputs
    float mlpx[RS == AMR_RIEMANN_MLP ? threads_for<D>() / 32 : 1][RS == AMR_RIEMANN_MLP ? 32 * 10 : 1];
    // the cells the phases read (built once per CTA): interior and face slots, edge-slot
    // cells (slot << 3 | child), predicted cells
    uint8_t gfull[G::NFULL];
    uint16_t gedge[2 * G::NEDGE];
    std::conditional_t<(G::NP < 256), uint8_t, uint16_t> plist[G::NPN];
};
static_assert(Geo<2>::NSLOT <= 256, "slot indices fit a byte");

// left and right states of face r0 of direction DIR (face-normal frame), floored
template <typename R, int D, int RS, int DIR>
__device__ __forceinline__ void face_states(const Smem<R, D, RS> &sm, int r0, const Prm<R> &pr, R WL[NV], R WR[NV])
{
    using G = Geo<D>;
    const int fa = r0 % (G::CI + 1), t1 = (r0 / (G::CI + 1)) % G::CI, t2 = r0 / ((G::CI + 1) * G::CI);
    const int Lx = DIR == 0 ? fa : 1 + t1;
    const int Ly = DIR == 0 ? 1 + t1 : DIR == 1 ? fa : 1 + t2;
    const int Lz = DIR == 2 ? fa : 1 + t2;
    const int pl = Lx + G::P * (Ly + G::P * Lz);
    const int pR = pl + (DIR == 0 ? 1 : DIR == 1 ? G::P : G::P * G::P);
    constexpr int S = NV + NV * DIR;
    R tL[NV], dL[NV], tR[NV], dR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        tL[v] = sm.Q[v][pl]; dL[v] = sm.Q[S + v][pl];
        tR[v] = sm.Q[v][pR]; dR[v] = sm.Q[S + v][pR];
    }
    face_state<DIR>(tL, dL, R(0.5), pr, WL);
    face_state<DIR>(tR, dR, R(-0.5), pr, WR);
}

template <typename R, int D, int RS, int DIR>
__device__ __forceinline__ void face_flux(Smem<R, D, RS> &sm, R (*sF)[NV][Geo<D>::NF], int r0, const Prm<R> &pr,
                                          int32_t *status, const GArgs &a, int64_t tile, unsigned &n_it,
                                          unsigned &n_solve)
{
    using G = Geo<D>;
    const int fa = r0 % (G::CI + 1), t1 = (r0 / (G::CI + 1)) % G::CI, t2 = r0 / ((G::CI + 1) * G::CI);
    // predicted-cell coordinates (stencil - 1) of the left cell
    const int Lx = DIR == 0 ? fa : 1 + t1;
    const int Ly = DIR == 0 ? 1 + t1 : DIR == 1 ? fa : 1 + t2;
    const int Lz = DIR == 2 ? fa : 1 + t2;
    const int pl = Lx + G::P * (Ly + G::P * Lz);
    const int pR = pl + (DIR == 0 ? 1 : DIR == 1 ? G::P : G::P * G::P);
    constexpr int N0 = DIR + 1, T1 = DIR == 0 ? 2 : 1, T2 = DIR == 2 ? 2 : 3;   // normal, transverse
    constexpr int S = NV + NV * DIR;                                             // slopes along DIR
    R WL[NV], WR[NV];
    {
        R tL[NV], dL[NV], tR[NV], dR[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            tL[v] = sm.Q[v][pl]; dL[v] = sm.Q[S + v][pl];
            tR[v] = sm.Q[v][pR]; dR[v] = sm.Q[S + v][pR];
        }
        face_state<DIR>(tL, dL, R(0.5), pr, WL);
        face_state<DIR>(tR, dR, R(-0.5), pr, WR);
    }
    if (a.harvest) {
        // deterministic sample of the faces (hash of tile, direction and face)
        uint64_t h = (uint64_t(tile) * 3 + DIR) * 0x9E3779B97F4A7C15ull + uint64_t(r0) * 0xBF58476D1CE4E5B9ull;
        h ^= h >> 31;
        if (h % uint64_t(a.harvest_stride) == 0) {
            const unsigned long long k = atomicAdd(a.harvest_count, 1ull);
            if (int64_t(k) < a.harvest_cap) {
                double *o = a.harvest + 6 * int64_t(k);
                o[0] = double(WL[0]); o[1] = double(WL[1]); o[2] = double(WL[4]);
                o[3] = double(WR[0]); o[4] = double(WR[1]); o[5] = double(WR[4]);
            }
        }
        return;
    }
    R Fn[NV];
    if (RS == AMR_RIEMANN_EXACT) {
        R ps, us;
        const R tol = sizeof(R) == 8 ? R(1e-14) : R(1e-6);
        int its;
        const int e = exact_star(WL, WR, pr.gamma, tol, 50, ps, us, R(-1), &its);
        n_it += its;
        ++n_solve;
        if (e == 0) {
            R W0[NV], U0[NV];
            exact_sample0(WL, WR, pr.gamma, ps, us, W0);
            flux_normal(W0, pr.gamma, Fn, U0);
        } else {
            set_error(status, e);
            hllc(WL, WR, pr.gamma, Fn);
        }
    } else {
        hllc(WL, WR, pr.gamma, Fn);
    }
    sF[DIR][0][r0] = Fn[0];
    sF[DIR][N0][r0] = Fn[1];
    sF[DIR][T1][r0] = Fn[2];
    sF[DIR][T2][r0] = Fn[3];
    sF[DIR][4][r0] = Fn[4];
}


// Riemann solve of the warp's 32 faces with the learned surrogate: features of each
// face-normal problem, the network on the tensor cores (two groups of 16), then the
// acceptance test -- p* > 0 and finite, |f(p*)| = |f_L + f_R + u_R - u_L| and
// |u* - (u_L+u_R)/2 - (f_R - f_L)/2| both within tol * (c_L + c_R) (Toro Eq. 4.5, 4.9) --
// sampling of the accepted (p*, u*) at x/t = 0, and the exact Newton solver for the rest.
// All 32 lanes of the warp take part; lanes past the last face carry a dummy problem.
template <typename R, int D, int RS>
__device__ __forceinline__ void mlp_faces(Smem<R, D, RS> &sm, R (*sF)[NV][Geo<D>::NF], const Prm<R> &pr,
                                          const GArgs &a, unsigned &n_acc, unsigned &n_fb, unsigned &n_it,
                                          unsigned &n_solve)
{
    using G = Geo<D>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *stg = sm.mlpx[warp];
    const mlp::Packed P = mlp::view(a.mlp);
    for (int base = warp * 32; base < 3 * G::NF; base += nw * 32) {
        const int f = base + lane;
        const bool valid = f < 3 * G::NF;
        const int d = valid ? f / G::NF : 0, r0 = valid ? f - d * G::NF : 0;
        R WL[NV], WR[NV];
        if (d == 0) face_states<R, D, RS, 0>(sm, r0, pr, WL, WR);
        else if (d == 1) face_states<R, D, RS, 1>(sm, r0, pr, WL, WR);
        else face_states<R, D, RS, 2>(sm, r0, pr, WL, WR);
        R x[7], pref, ubar, cref;
        mlp::features(WL[0], WL[1], WL[4], WR[0], WR[1], WR[4], pr.gamma, x, pref, ubar, cref);
#pragma unroll
        for (int k = 0; k < 7; ++k) stg[lane * 8 + k] = float(x[k]);
        stg[lane * 8 + 7] = 0.0f;
        __syncwarp();
        float o0[4], o1[4];
        mlp::forward16(P, stg, lane, o0);
        mlp::forward16(P, stg + 16 * 8, lane, o1);
        if ((lane & 3) == 0) {
            const int g = lane >> 2;
            stg[256 + 2 * g] = o0[0]; stg[256 + 2 * g + 1] = o0[1];
            stg[256 + 2 * (g + 8)] = o0[2]; stg[256 + 2 * (g + 8) + 1] = o0[3];
            stg[256 + 2 * (g + 16)] = o1[0]; stg[256 + 2 * (g + 16) + 1] = o1[1];
            stg[256 + 2 * (g + 24)] = o1[2]; stg[256 + 2 * (g + 24) + 1] = o1[3];
        }
        __syncwarp();
        const R y0 = R(stg[256 + 2 * lane]), y1 = R(stg[256 + 2 * lane + 1]);
        __syncwarp();
        const R g = pr.gamma;
        const R rL = WL[0], uL = WL[1], pL = WL[4], rR = WR[0], uR = WR[1], pR = WR[4];
        const R cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
        const bool vac = R(2) * (cL + cR) / (g - R(1)) <= uR - uL;
        const R ps = pref * exp(y0), us = ubar + cref * y1;
        bool ok = !vac && isfinite(ps) && ps > R(0) && isfinite(us);
        if (ok && !a.mlp_seed) {
            R fL, dfL, fR, dfR;
            side_f(ps, rL, pL, cL, g, fL, dfL);
            side_f(ps, rR, pR, cR, g, fR, dfR);
            const R tolc = R(a.mlp_tol) * (cL + cR);
            ok = fabs(fL + fR + (uR - uL)) <= tolc && fabs(us - (R(0.5) * (uL + uR) + R(0.5) * (fR - fL))) <= tolc;
        }
        R Fn[NV], W0[NV], U0[NV];
        if (ok && !a.mlp_seed) {
            exact_sample0(WL, WR, g, ps, us, W0);
            flux_normal(W0, g, Fn, U0);
        } else {
            // exact Newton solve: seeded by the network's p* when it is usable (seeded
            // mode), from the linearised guess otherwise
            R ps2, us2;
            const R tol = sizeof(R) == 8 ? R(1e-14) : R(1e-6);
            int its;
            const int e = exact_star(WL, WR, g, tol, 50, ps2, us2, ok ? ps : R(-1), &its);
            if (valid) {
                n_it += its;
                ++n_solve;
            }
            if (e == 0) {
                exact_sample0(WL, WR, g, ps2, us2, W0);
                flux_normal(W0, g, Fn, U0);
            } else {
                if (valid) set_error(a.status, e);
                hllc(WL, WR, g, Fn);
            }
        }
        // accepted (seeded) faces and fallbacks (cold starts)
        const unsigned acc = __ballot_sync(0xffffffffu, ok && valid), fb = __ballot_sync(0xffffffffu, !ok && valid);
        n_acc += __popc(acc);
        n_fb += __popc(fb);
        if (valid) {
            const int N0 = d + 1, T1 = d == 0 ? 2 : 1, T2 = d == 2 ? 2 : 3;
            sF[d][0][r0] = Fn[0];
            sF[d][N0][r0] = Fn[1];
            sF[d][T1][r0] = Fn[2];
            sF[d][T2][r0] = Fn[3];
            sF[d][4][r0] = Fn[4];
        }
    }
}

// Riemann problem at face r0 of direction DIR: left state = predicted cell + half its
// slope, right state = next cell - half its slope (floored), in the face-normal frame.
template <typename R, int D, int RS>
__global__ void __launch_bounds__(threads_for<D>(), (min_ctas_for<R, D, RS>())) k_godunov(GArgs a)
{
    using G = Geo<D>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R, D, RS> &sm = *reinterpret_cast<Smem<R, D, RS> *>(smem_raw);
    R(*sF)[NV][G::NF] = reinterpret_cast<R(*)[NV][G::NF]>(&sm.W[0][0]);   // aliases W after phase 2
    static_assert(3 * NV * G::NF <= NV * G::NC, "flux buffer must fit in the stencil buffer");
    const TreeView &tv = a.tv;
    const int tid = threadIdx.x;
    Prm<R> pr;
    pr.gamma = to_work<R>(a.gamma); pr.rho_floor = to_work<R>(a.rho_floor); pr.p_floor = to_work<R>(a.p_floor);
    pr.limiter = a.limiter;
    const R cflR = to_work<R>(a.cfl);

    unsigned n_acc = 0, n_fb = 0;   // surrogate: accepted faces, fallbacks (counted by lane 0)
    unsigned n_it = 0, n_solve = 0; // Newton iterations and Newton solves of this thread
    // The launch has as many CTAs as fit on the GPU at once, each looping over tiles: the
    // next tile's slot entries and refinement masks are loaded into registers while the
    // current tile runs (one slot per thread: NSLOT <= threads).
    static_assert(G::NSLOT <= threads_for<D>(), "one slot per thread");
    int32_t e_nx = 0;
    uint8_t rf_nx = 0;
    bool have_nx = false;
    {
        // the lists of the cells the phases read, compacted in index order by warps 0-2
        // (visible to all after the first tile's slot barrier)
        const int lane = tid & 31, w = tid >> 5;
        const unsigned below = (1u << lane) - 1u;
        auto bnd = [](int i, int n) { return int(i == 0 || i == n - 1); };
        int n = 0;
        if (w == 0) {
            for (int b = 0; b < G::NSLOT; b += 32) {
                const int s = b + lane;
                const bool want = s < G::NSLOT &&
                                  bnd(s % G::NS, G::NS) + bnd((s / G::NS) % G::NS, G::NS) + bnd(s / (G::NS * G::NS), G::NS) <= 1;
                const unsigned m = __ballot_sync(0xffffffffu, want);
                const int k = n + __popc(m & below);
                if (want && k < G::NFULL) sm.gfull[k] = uint8_t(s);
                n += __popc(m);
            }
        } else if (w == 1) {
            auto out = [](int i) { return i < 2 ? 2 - i : (i > G::C - 3 ? i - (G::C - 3) : 0); };
            for (int b = 0; b < 8 * G::NSLOT; b += 32) {
                const int q = b + lane, sl = q >> 3, c = q & 7;
                const int sx = sl % G::NS, sy = (sl / G::NS) % G::NS, sz = sl / (G::NS * G::NS);
                const bool want = q < 8 * G::NSLOT && bnd(sx, G::NS) + bnd(sy, G::NS) + bnd(sz, G::NS) == 2 &&
                                  out(2 * sx + (c & 1)) + out(2 * sy + ((c >> 1) & 1)) + out(2 * sz + (c >> 2)) == 2;
                const unsigned m = __ballot_sync(0xffffffffu, want);
                const int k = n + __popc(m & below);
                if (want && k < 2 * G::NEDGE) sm.gedge[k] = uint16_t(q);
                n += __popc(m);
            }
        } else if (w == 2) {
            for (int b = 0; b < G::NP; b += 32) {
                const int p = b + lane;
                const bool want = p < G::NP &&
                                  bnd(p % G::P, G::P) + bnd((p / G::P) % G::P, G::P) + bnd(p / (G::P * G::P), G::P) <= 1;
                const unsigned m = __ballot_sync(0xffffffffu, want);
                const int k = n + __popc(m & below);
                if (want && k < G::NPN) sm.plist[k] = p;
                n += __popc(m);
            }
        }
    }
    for (int64_t t = a.t_begin + blockIdx.x; t < a.t_end; t += gridDim.x) {
        // ---- level of this tile and its geometry
        const int32_t root = a.tile_root[t];
        int l = a.lfirst;
        int64_t n;                   // cells per dimension of the tile's level (or box)
        double dx, lam;              // cell size, dt / dx
        double *dtn;                 // where the next step's CFL candidates go
        int64_t X0[3];               // global cell coordinates of stencil index 0
        if (a.tile_inst) {
            // batch mode: a box of N^3 cells of size 1/N, its own time step; the root is
            // the tile's corner oct
            const int b = a.tile_inst[t];
            n = tv.inst_n[b];
            dx = tv.inst_dx[b];
            lam = a.dt[b] * double(n);
            dtn = a.dt_next ? a.dt_next + b : nullptr;
            X0[0] = 2 * int64_t(tv.ix[root]) - 2; X0[1] = 2 * int64_t(tv.iy[root]) - 2; X0[2] = 2 * int64_t(tv.iz[root]) - 2;
        } else {
            while (l < a.llast && t >= a.tile_off[l + 1]) ++l;
            n = int64_t(1) << l;
            // a depth-D root covers 2^(D+1) level-l cells per axis; stencil index 0 is two cells before
            X0[0] = int64_t(tv.ix[root]) * (2 << D) - 2;
            X0[1] = int64_t(tv.iy[root]) * (2 << D) - 2;
            X0[2] = int64_t(tv.iz[root]) * (2 << D) - 2;
            dx = pow2(-l);
            lam = scale_pow2(*a.dt, l);    // dt / dx, exact
            dtn = a.dt_next;
        }
        int mine_out = 0;
        const bool finer = !a.tile_inst && l < tv.levelmax;   // only then can a stencil cell be refined
        if (tid < G::NSLOT) {
            int32_t e;
            uint8_t rf;
            if (have_nx) {
                e = e_nx;
                rf = rf_nx;
            } else {
                e = a.tile_slot[t * G::NSLOT + tid];
                rf = e >= 0 ? tv.refmask[e] : 0;
            }
            sm.slot[tid] = e;
            sm.ref[tid] = (e >= 0 && finer) ? rf : 0;
            mine_out = (e == OUTSIDE);
        }
        const int any_outside = __syncthreads_or(mine_out);   // barrier: slots visible to all
        // the next tile's slot entries (their refinement masks after the predictor)
        const int64_t t_nx = t + gridDim.x;
        have_nx = t_nx < a.t_end;
        if (have_nx && tid < G::NSLOT) e_nx = a.tile_slot[t_nx * G::NSLOT + tid];

        // ---- phase 1: gather + primitives of the listed cells (c fastest so a warp reads
        // whole octs)
        for (int kg = tid; kg < G::NG; kg += blockDim.x) {
            int s, c;
            if (kg < 8 * G::NFULL) {
                s = sm.gfull[kg >> 3];
                c = kg & 7;
            } else {
                const int q = sm.gedge[kg - 8 * G::NFULL];
                s = q >> 3;
                c = q & 7;
            }
            const int sx = s % G::NS, sy = (s / G::NS) % G::NS, sz = s / (G::NS * G::NS);
            const int i = 2 * sx + (c & 1), j = 2 * sy + ((c >> 1) & 1), k = 2 * sz + ((c >> 2) & 1);
            const int si = i + G::C * (j + G::C * k);
            const int32_t e = sm.slot[s];
            if (e == OUTSIDE) continue;
            R Uw[NV];
            if (e >= 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) Uw[v] = to_work<R>(a.u_old[v * tv.ncell + int64_t(e) * 8 + c]);
            } else if (e == UNNEEDED_SLOT) {
                Uw[0] = R(1); Uw[1] = R(0); Uw[2] = R(0); Uw[3] = R(0); Uw[4] = R(1);
            } else if (a.ghost) {
                const R *gh = static_cast<const R *>(a.ghost) + (int64_t(-1) - e) * 8 + c;
#pragma unroll
                for (int v = 0; v < NV; ++v) Uw[v] = gh[v * a.ghost_stride];
            } else {
                interp_child<R>(tv, a.u_old, tv.ghost_cell[int64_t(-1) - e], c, Uw);
            }
            R Wc[NV];
            cons_to_prim_w(Uw, pr, Wc);
#pragma unroll
            for (int v = 0; v < NV; ++v) sm.W[v][si] = Wc[v];
        }
        __syncthreads();
        if (any_outside) {
            // outflow ghosts: copy the cell at the clamped coordinates (zero gradient)
            for (int q = tid; q < G::NC; q += blockDim.x) {
                const int i = q % G::C, j = (q / G::C) % G::C, k = q / (G::C * G::C);
                int64_t g[3] = {X0[0] + i, X0[1] + j, X0[2] + k};
                bool out = false;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (g[d] < 0) { g[d] = 0; out = true; }
                    else if (g[d] >= n) { g[d] = n - 1; out = true; }
                }
                if (!out) continue;
                const int src = int(g[0] - X0[0]) + G::C * (int(g[1] - X0[1]) + G::C * int(g[2] - X0[2]));
#pragma unroll
                for (int v = 0; v < NV; ++v) sm.W[v][q] = sm.W[v][src];
            }
            __syncthreads();
        }

        // ---- phase 2: slopes + predictor on the listed cells of stencil 1..C-2
        const R lamR = to_work<R>(lam);
        const R hl = R(0.5) * lamR;
        for (int kp = tid; kp < G::NPN; kp += blockDim.x) {
            const int p = sm.plist[kp];
            const int i = 1 + p % G::P, j = 1 + (p / G::P) % G::P, k = 1 + p / (G::P * G::P);
            const int si = i + G::C * (j + G::C * k);
            const int st[3] = {1, G::C, G::C * G::C};
            R Wc[NV], Dl[3][NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Wc[v] = sm.W[v][si];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    Dl[d][v] = slope(pr, Wc[v] - sm.W[v][si - st[d]], sm.W[v][si + st[d]] - Wc[v]);
            R Wt[NV];
            muscl_predict(Wc, Dl, hl, pr.gamma, Wt);
#pragma unroll
            for (int v = 0; v < NV; ++v) sm.Q[v][p] = Wt[v];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < NV; ++v) sm.Q[NV + NV * d + v][p] = Dl[d][v];
        }
        __syncthreads();

        if (have_nx && tid < G::NSLOT) rf_nx = e_nx >= 0 ? tv.refmask[e_nx] : 0;

        // ---- phase 3: Riemann problem at every face touching an updated cell
        if constexpr (RS == AMR_RIEMANN_MLP) {
            mlp_faces<R, D, RS>(sm, sF, pr, a, n_acc, n_fb, n_it, n_solve);
        } else {
            for (int f = tid; f < 3 * G::NF; f += blockDim.x) {
                const int d = f / G::NF, r0 = f - d * G::NF;
                if (d == 0) face_flux<R, D, RS, 0>(sm, sF, r0, pr, a.status, a, t, n_it, n_solve);
                else if (d == 1) face_flux<R, D, RS, 1>(sm, sF, r0, pr, a.status, a, t, n_it, n_solve);
                else face_flux<R, D, RS, 2>(sm, sF, r0, pr, a.status, a, t, n_it, n_solve);
            }
        }
        __syncthreads();
        if (a.harvest) continue;   // harvesting only: no update (the loop ends with no barrier due)

        // ---- flux register: oct sides whose neighbour slot is a coarse leaf (face fluxes
        // only, so it may run beside the update)
        constexpr int NREG = G::OI * G::OI * G::OI * 6;
        auto reg_task = [&](int w) {
            const int o = w / 6, f = w % 6, d = f >> 1, side = f & 1;
            const int ox = 1 + o % G::OI, oy = 1 + (o / G::OI) % G::OI, oz = 1 + o / (G::OI * G::OI);
            const int32_t e = sm.slot[ox + G::NS * (oy + G::NS * oz)];
            if (e < 0 || e < tv.reg_base) return;   // base-level octs never face a coarser leaf
            int nsl[3] = {ox, oy, oz};
            nsl[d] += side ? 1 : -1;
            const int32_t en = sm.slot[nsl[0] + G::NS * (nsl[1] + G::NS * nsl[2])];
            if (en >= 0 || en == OUTSIDE || en == UNNEEDED_SLOT) return;
            double sum[NV] = {0, 0, 0, 0, 0};
            for (int c = 0; c < 8; ++c) {
                const int pc[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                if (pc[d] != side) continue;
                const int ii[3] = {2 * ox + pc[0] - 2, 2 * oy + pc[1] - 2, 2 * oz + pc[2] - 2};
                const int t1 = ii[d == 0 ? 1 : 0], t2 = ii[d == 2 ? 1 : 2];
                const int r0 = (ii[d] + side) + (G::CI + 1) * (t1 + G::CI * t2);
#pragma unroll
                for (int v = 0; v < NV; ++v) sum[v] += to_state(sF[d][v][r0]);
            }
            const int64_t row = (int64_t(e) - tv.reg_base) * 6 + f;
#pragma unroll
            for (int v = 0; v < NV; ++v) a.reg[row * NV + v] = sum[v];
        };
        // with depth-1 tiles the update has one cell for half the threads: the other half
        // writes the register rows meanwhile
        constexpr bool EARLY_REG = threads_for<D>() >= G::NI + NREG;
        if (EARLY_REG && a.reg && tid >= G::NI && tid < G::NI + NREG) reg_task(tid - G::NI);

        // ---- phase 4: FP64 update of existing cells + fused CFL candidate
        // new states of octs whose father is restricted here, in the (now free) predictor buffer
        double(*sU)[G::NI] = reinterpret_cast<double(*)[G::NI]>(&sm.Q[0][0]);
        static_assert(sizeof(double) * NV * G::NI <= sizeof(R) * 4 * NV * G::NP, "restriction buffer");
        unsigned long long my_dt = ~0ull;   // bit pattern of the smallest positive candidate
        for (int q = tid; q < G::NI; q += blockDim.x) {
            const int c = q & 7, o = q >> 3;
            const int ox = 1 + o % G::OI, oy = 1 + (o / G::OI) % G::OI, oz = 1 + o / (G::OI * G::OI);
            const int s = ox + G::NS * (oy + G::NS * oz);
            const int32_t e = sm.slot[s];
            if (e < 0) continue;                                    // no oct here: nothing to update
            if ((sm.ref[s] >> c) & 1) continue;   // refined: its value comes from the restriction
            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
            const int ii[3] = {2 * ox + cx - 2, 2 * oy + cy - 2, 2 * oz + cz - 2};   // interior coords 0..CI-1
            R dU[NV] = {0, 0, 0, 0, 0};     // flux sums in the working precision
            bool nbref = false;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int t1 = ii[d == 0 ? 1 : 0], t2 = ii[d == 2 ? 1 : 2];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    // neighbour cell across the face: stencil coords of this cell +- e_d
                    int nc[3] = {ii[0] + 2, ii[1] + 2, ii[2] + 2};
                    nc[d] += side ? 1 : -1;
                    const int ns = (nc[0] >> 1) + G::NS * ((nc[1] >> 1) + G::NS * (nc[2] >> 1));
                    const int ncc = (nc[0] & 1) + 2 * (nc[1] & 1) + 4 * (nc[2] & 1);
                    if (finer && sm.slot[ns] >= 0 && ((sm.ref[ns] >> ncc) & 1)) { nbref = true; continue; }
                    const int fa = ii[d] + side;
                    const int r0 = fa + (G::CI + 1) * (t1 + G::CI * t2);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const R F = sF[d][v][r0];
                        dU[v] = side ? dU[v] - F : dU[v] + F;
                    }
                }
            }
            const int64_t cell = int64_t(e) * 8 + c;
            double Un[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                // FP64 accumulation: U_new = U_old + dt/dx * (sum of face fluxes); in the FP32 path
                // the increment is formed in FP32 (dt/dx is exact there: dt is an FP32 value and
                // dx a power of two) and added in FP64
                if (sizeof(R) == 8) Un[v] = a.u_old[v * tv.ncell + cell] + lam * to_state(dU[v]);
                else Un[v] = a.u_old[v * tv.ncell + cell] + to_state(lamR * dU[v]);
                a.u_new[v * tv.ncell + cell] = Un[v];
            }
            if (!state_finite<R>(Un)) set_error(a.status, AMR_ENONPHYSICAL);
            if (tv.fused[e]) {
#pragma unroll
                for (int v = 0; v < NV; ++v) sU[v][q] = Un[v];   // kept for the restriction pass
            }
            if (dtn && !nbref) {
                // CFL candidate (newdt_fine) from the final new state of this leaf cell
                const double cand = cfl_candidate<R>(Un, pr, cflR, to_work<R>(dx));
                my_dt = umin64(my_dt, dbits(cand));
            }
        }
        if (dtn) {
            for (int off = 16; off > 0; off >>= 1) my_dt = umin64(my_dt, __shfl_xor_sync(0xffffffffu, my_dt, off));
            if ((tid & 31) == 0 && my_dt != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(dtn), my_dt);
        }

        // ---- restriction of father cells whose eight children are final here: one thread per
        // (oct, variable), children summed in cell order, so every FP64 lane does useful work
        __syncthreads();
        for (int w = tid; w < G::OI * G::OI * G::OI * NV; w += blockDim.x) {
            const int o = w / NV, v = w % NV;
            const int ox = 1 + o % G::OI, oy = 1 + (o / G::OI) % G::OI, oz = 1 + o / (G::OI * G::OI);
            const int32_t e = sm.slot[ox + G::NS * (oy + G::NS * oz)];
            if (e < 0 || !tv.fused[e]) continue;
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < 8; ++c) acc += sU[v][o * 8 + c];
            a.u_new[v * tv.ncell + tv.father[e]] = 0.125 * acc;
        }

        // ---- flux register rows (with depth-1 tiles written above, during the update)
        if (a.reg && !EARLY_REG)
            for (int w = tid; w < NREG; w += blockDim.x) reg_task(w);
        __syncthreads();
    }
    if (RS == AMR_RIEMANN_MLP && a.counters && (tid & 31) == 0 && (n_acc | n_fb)) {
        atomicAdd(a.counters + 0, (unsigned long long)n_acc);
        atomicAdd(a.counters + 1, (unsigned long long)n_fb);
    }
    if (RS != AMR_RIEMANN_HLLC && a.counters) {
        const unsigned it_w = __reduce_add_sync(0xffffffffu, n_it), so_w = __reduce_add_sync(0xffffffffu, n_solve);
        if ((tid & 31) == 0 && so_w) {
            atomicAdd(a.counters + 2, (unsigned long long)it_w);
            atomicAdd(a.counters + 3, (unsigned long long)so_w);
        }
    }
}

template <typename R, int D, int RS>
static amr_status launch(const GArgs &a, int64_t ntile, cudaStream_t st)
{
    if (ntile <= 0) return AMR_OK;
    // 227 KB per CTA at most; the FP32 depth-1 update keeps eight CTAs in an SM's 228 KB
    // (each with its 1 KB reserved by the system)
    static_assert(sizeof(Smem<R, D, RS>) <= 227 * 1024, "tile shared memory");
    static_assert(min_ctas_for<R, D, RS>() == 1 || (sizeof(Smem<R, D, RS>) + 1024) * 8 <= 228 * 1024,
                  "eight depth-1 CTAs per SM");
    const size_t bytes = sizeof(Smem<R, D, RS>);
    auto kern = k_godunov<R, D, RS>;
    AMR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    // as many CTAs as are resident at once (each loops over tiles and prefetches the next
    // tile's slot table)
    int dev = 0, nsm = 152, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads_for<D>(), bytes) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t resident = int64_t(per_sm) * nsm;
    const int64_t grid = ntile < resident ? ntile : resident;
    kern<<<unsigned(grid), threads_for<D>(), bytes, st>>>(a);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

// The z-column kernel for the deepest complete level (or the box batch): the pencil
// kernel (16 x 16 footprints, FP32) where it applies and is not declined, else the slab
// kernel (8 x 8 footprints).
template <typename R>
amr_status launch_column(const amr_tree *t, const hydro_params *p, const double *u_old, double *u_new,
                         const double *dt, double *dt_next, cudaStream_t st)
{
    const bool exact = p->riemann == AMR_RIEMANN_EXACT;
    if constexpr (sizeof(R) == 4) {
        const bool fits = t->n_inst > 0 ? (t->col_work > 0 && t->col_work % 4 == 0) : (t->grid_level >= 4);
        if (p->col_kernel != 1 && fits)
            return exact ? launch_pen<AMR_RIEMANN_EXACT>(t, p, u_old, u_new, dt, dt_next, p->col_seg, st)
                         : launch_pen<AMR_RIEMANN_HLLC>(t, p, u_old, u_new, dt, dt_next, p->col_seg, st);
    }
    return exact ? launch_col<R, AMR_RIEMANN_EXACT>(t, p, u_old, u_new, dt, dt_next, st)
                 : launch_col<R, AMR_RIEMANN_HLLC>(t, p, u_old, u_new, dt, dt_next, st);
}

// Launch the kernel(s) of precision R for one level or for all levels (level = -1).
// Levels whose tiles of the requested depth would be rooted above level 1 use depth 1.
template <typename R>
amr_status dispatch_impl(const amr_tree *t, int level, const hydro_params *p, const double *u_old, double *u_new,
                         double *reg, const double *dt, double *dt_next, cudaStream_t st)
{
    int depth = p->tile == 0 ? 1 : p->tile;
    if (depth != 1 && depth != 2) return AMR_EINVAL;
    const bool mlp_like = p->riemann == AMR_RIEMANN_MLP || p->riemann == AMR_RIEMANN_MLP_SEEDED;
    // the z-column kernel implements MinMod slopes; the MC limiter runs in the tile kernel
    const bool col_ok = !p->tiles_only && !mlp_like && p->limiter == AMR_LIMITER_MINMOD;
    if (depth == 2 && sizeof(R) == 8) return AMR_EINVAL;   // an FP64 12^3-cell stencil does not fit in smem
    if (t->n_inst > 0) {
        // batch mode: every box in one launch (z-column kernel when every box is a multiple of
        // 16 cells, else tiles)
        if (level != -1) return AMR_EINVAL;
        if (col_ok && t->col_work > 0) return launch_column<R>(t, p, u_old, u_new, dt, dt_next, st);
        if (depth == 2 && t->tile_off[1][1] == 0) depth = 1;            // some box is not a multiple of 8
        if (mlp_like) depth = 1;
        const int d = depth;
        GArgs a;
        a.tv = make_view(t);
        a.tile_root = t->tile_root[d - 1];
        a.tile_slot = t->tile_slot[d - 1];
        a.tile_inst = t->tile_inst[d - 1];
        for (int i = 0; i < AMR_MAXLEV + 2; ++i) a.tile_off[i] = t->tile_off[d - 1][i];
        a.lfirst = a.llast = 0;
        a.t_begin = 0;
        a.t_end = t->tile_off[d - 1][1];
        a.u_old = u_old; a.u_new = u_new; a.reg = nullptr; a.dt = dt; a.dt_next = dt_next;
        a.gamma = p->gamma; a.rho_floor = p->rho_floor; a.p_floor = p->p_floor; a.cfl = p->cfl;
        a.status = p->d_status; a.counters = p->d_counters;
        a.mlp = p->mlp_weights; a.mlp_tol = p->mlp_resid_tol; a.mlp_seed = p->riemann == AMR_RIEMANN_MLP_SEEDED;
        a.limiter = p->limiter;
        a.harvest = nullptr; a.harvest_cap = 0; a.harvest_stride = 1; a.harvest_count = nullptr;
        a.ghost = nullptr; a.ghost_stride = 0;
        const int64_t nt = a.t_end;
        constexpr int D2 = 2 - (sizeof(R) == 8);
        if (mlp_like) {
            if (sizeof(R) == 8 || !p->mlp_weights) return AMR_EINVAL;
            return launch<R, 1, AMR_RIEMANN_MLP>(a, nt, st);
        }
        if (p->riemann == AMR_RIEMANN_EXACT)
            return d == 1 ? launch<R, 1, AMR_RIEMANN_EXACT>(a, nt, st) : launch<R, D2, AMR_RIEMANN_EXACT>(a, nt, st);
        return d == 1 ? launch<R, 1, AMR_RIEMANN_HLLC>(a, nt, st) : launch<R, D2, AMR_RIEMANN_HLLC>(a, nt, st);
    }
    // level: >= 0 one level, -1 all levels, <= -2 the range encoded as -2 - (hi << 8 | lo)
    int l0 = level < 0 ? t->levelmin : level, l1 = level < 0 ? t->levelmax : level;
    if (level <= -2) { l0 = (-2 - level) & 255; l1 = (-2 - level) >> 8; }
    if (l0 < t->levelmin || l1 > t->levelmax) return AMR_EINVAL;
    // levels below the deepest complete level have no leaf cells and no octs whose father
    // this kernel restricts: nothing to update there
    const int gl = t->grid_level;
    if (t->grid && gl > l0) l0 = gl;
    if (l0 > l1) return AMR_OK;
    // the deepest complete level goes to the z-column kernel (bitwise the same per cell);
    // the levels above it to the tile kernel
    if (col_ok && t->grid && gl >= 3 && gl >= l0 && gl <= l1) {
        const amr_status r = launch_column<R>(t, p, u_old, u_new, dt, dt_next, st);
        if (r != AMR_OK) return r;
        // levels below a complete level have no leaf cells: nothing of theirs survives the
        // restriction, so they are not updated
        hydro_params q = *p;
        q.tiles_only = 1;
        if (gl < l1) return dispatch_impl<R>(t, -2 - (l1 << 8 | (gl + 1)), &q, u_old, u_new, reg, dt, dt_next, st);
        return AMR_OK;
    }
    // the children of every coarse leaf these tiles interpolate from, once, into the part
    // of the flux-register buffer after its rows
    const void *ghost = nullptr;
    if (reg && t->n_ghost > 0 && t->ghost_cell) {
        const int64_t g0 = t->ghost_off[l0 - 1], g1 = t->ghost_off[l1];
        R *gb = reinterpret_cast<R *>(reinterpret_cast<char *>(reg) + reg_rows_bytes(t));
        if (g1 > g0) {
            const int64_t nthr = g1 - g0;
            k_ghost<R><<<unsigned((nthr + 255) / 256), 256, 0, st>>>(make_view(t), u_old, g0, g1, 8 * t->n_ghost, gb);
            AMR_CUDA_TRY(cudaGetLastError());
        }
        ghost = gb;
    }
    int lsplit = l0;
    while (lsplit <= l1 && lsplit - depth < 1) ++lsplit;
    for (int pass = 0; pass < 2; ++pass) {
        const int d = pass == 0 ? 1 : depth;
        const int la = pass == 0 ? l0 : lsplit, lb = pass == 0 ? lsplit - 1 : l1;
        if ((pass == 0 && depth == 1) || la > lb) continue;
        GArgs a;
        a.tv = make_view(t);
        a.tile_root = t->tile_root[d - 1];
        a.tile_slot = t->tile_slot[d - 1];
        a.tile_inst = nullptr;
        for (int i = 0; i < AMR_MAXLEV + 2; ++i) a.tile_off[i] = t->tile_off[d - 1][i];
        a.lfirst = la;
        a.llast = lb;
        a.t_begin = t->tile_off[d - 1][la];
        a.t_end = t->tile_off[d - 1][lb + 1];
        a.u_old = u_old; a.u_new = u_new; a.reg = reg; a.dt = dt; a.dt_next = dt_next;
        a.gamma = p->gamma; a.rho_floor = p->rho_floor; a.p_floor = p->p_floor; a.cfl = p->cfl;
        a.status = p->d_status; a.counters = p->d_counters;
        const int64_t nt = a.t_end - a.t_begin;
        a.mlp = p->mlp_weights;
        a.mlp_tol = p->mlp_resid_tol;
        a.mlp_seed = p->riemann == AMR_RIEMANN_MLP_SEEDED;
        a.limiter = p->limiter;
        a.harvest = nullptr;
        a.harvest_cap = 0;
        a.harvest_stride = 1;
        a.harvest_count = nullptr;
        a.ghost = ghost;
        a.ghost_stride = 8 * t->n_ghost;
        constexpr int D2 = 2 - (sizeof(R) == 8);
        amr_status r;
        if (mlp_like) {
            if (sizeof(R) == 8 || !p->mlp_weights) return AMR_EINVAL;   // the surrogate runs in the FP32 path
            // the network's fragments need the register budget of 128-thread CTAs: depth-1 tiles
            if (d != 1) {
                a.tile_root = t->tile_root[0];
                a.tile_slot = t->tile_slot[0];
                for (int i = 0; i < AMR_MAXLEV + 2; ++i) a.tile_off[i] = t->tile_off[0][i];
                a.t_begin = t->tile_off[0][la];
                a.t_end = t->tile_off[0][lb + 1];
            }
            r = launch<R, 1, AMR_RIEMANN_MLP>(a, a.t_end - a.t_begin, st);
        } else if (p->riemann == AMR_RIEMANN_EXACT) {
            r = d == 1 ? launch<R, 1, AMR_RIEMANN_EXACT>(a, nt, st) : launch<R, D2, AMR_RIEMANN_EXACT>(a, nt, st);
        } else {
            r = d == 1 ? launch<R, 1, AMR_RIEMANN_HLLC>(a, nt, st) : launch<R, D2, AMR_RIEMANN_HLLC>(a, nt, st);
        }
        if (r != AMR_OK) return r;
    }
    return AMR_OK;
}

// Face-state harvest: the FP64 depth-1 kernel through phase 2, writing a deterministic
// sample (one face in `stride`) of the floored face-normal states, no update.
inline amr_status harvest_impl(const amr_tree *t, const hydro_params *p, const double *u, const double *dt,
                               double *out, int64_t cap, int64_t stride, unsigned long long *count, cudaStream_t st)
{
    GArgs a;
    a.tv = make_view(t);
    a.tile_root = t->tile_root[0];
    a.tile_slot = t->tile_slot[0];
    a.tile_inst = nullptr;
    for (int i = 0; i < AMR_MAXLEV + 2; ++i) a.tile_off[i] = t->tile_off[0][i];
    a.lfirst = t->levelmin;
    a.llast = t->levelmax;
    a.t_begin = t->tile_off[0][t->levelmin];
    a.t_end = t->tile_off[0][t->levelmax + 1];
    a.u_old = u; a.u_new = nullptr; a.reg = nullptr; a.dt = dt; a.dt_next = nullptr;
    a.gamma = p->gamma; a.rho_floor = p->rho_floor; a.p_floor = p->p_floor; a.cfl = p->cfl;
    a.status = p->d_status; a.counters = nullptr;
    a.mlp = nullptr; a.mlp_tol = 0.0f; a.mlp_seed = 0; a.limiter = p->limiter;
    a.harvest = out; a.harvest_cap = cap; a.harvest_stride = stride; a.harvest_count = count;
    a.ghost = nullptr; a.ghost_stride = 0;
    return launch<double, 1, AMR_RIEMANN_HLLC>(a, a.t_end - a.t_begin, st);
}

}  // namespace amr
