// godunov_fine on a complete finest level: the z-column ("2.5D") form of the update.
//
// When the finest level l is complete (2^(l-1) octs per axis, nothing refined) the level
// is a uniform grid; a CTA owns an FX x FY-cell footprint and marches a ZC-cell segment
// of its column in z, two cell planes (one oct layer) per slab k, k+1, keeping rings of
//   W  -- primitive stencil planes k .. k+3,
//   Q  -- predicted planes k .. k+2 (W~ and the three MinMod slopes),
//   Fz -- z-face fluxes below planes k .. k+2,
// so every stencil plane is gathered, predicted and every z face solved once per
// segment; only the x-y halo is repeated.  Per cell the arithmetic is the tile kernel's,
// in the same order (gather conversion, predictor, face states, Riemann solve, flux sum
// x-left, x-right, y-left, y-right, z-below, z-above, FP64 update, CFL candidate,
// restriction), so the two kernels give bitwise equal states.
#pragma once
#include "hydro_math.cuh"

namespace amr {

template <typename R, int FX, int FY, bool FINER> struct ColSmem {
    static constexpr int SX = FX + 4, SY = FY + 4;   // stencil footprint (cells)
    R W[4][NV][SY * SX];                             // ring, slot = plane & 3 (live: k .. k+3)
    // Q ring, slot = (plane + 6) % 3 (live: k .. k+2).  A plane keeps the predicted cells the
    // faces read: the FX x FY interior and four strips outside it, top (j = FY+2), left
    // (i = 1), bottom (j = 1), right (i = FX+2); the corners are never read and not kept.
    // The interior is row-major (stride FX) with the two halves of rows 4..7 swapped (qx in
    // the kernel); the slot stride is padded by 16 floats (faces whose two sides lie in
    // adjacent slots, and warps that straddle two planes, then meet fewer bank conflicts).
    static constexpr int QC = FX * FY + 2 * (FX + FY);
    static constexpr int QT = FX * FY, QL = QT + FX, QB = QL + FY, QR = QB + FX;
    static constexpr int QS = 4 * NV * QC + 16;
    R Q[3][QS];
    R Fx[2][NV][FY * (FX + 1)];                      // x faces of the slab's two planes
    R Fy[2][NV][(FY + 1) * FX];
    R Fz[3][NV][FY * FX];                            // face below plane j, slot (j + 6) % 3
    // new states of the last two slabs, [child c][oct o of the slab][variable]; the row
    // length is padded so that the update's stores (16 lanes: 4 octs x 4 children) and the
    // restriction's loads (16 lanes: consecutive (oct, variable)) each take one wavefront
    static constexpr int NOS = (FX / 2) * (FY / 2), UC = NOS * NV + 4;
    double U[2][8][UC];
    int32_t cell0[2][NOS];                           // cell id of each oct's child 0 (-1: refined)
    int32_t oct[4][(SX / 2) * (SY / 2)];             // oct id per footprint oct column, slot = oct layer & 3
    // refined flag of each stencil cell, slot = plane & 7 (live: k-1 .. k+5, longer than the
    // W ring); only when the level has finer levels
    uint8_t ref[FINER ? 8 : 1][FINER ? SY * SX : 1];
};

struct ColArgs {
    TreeView tv;
    const int32_t *grid;
    // batch mode (n_inst > 0): per-box work offsets, octs lexicographic per box
    int32_t n_inst;
    const int64_t *inst_col_off, *inst_oct_off;
    int64_t work;
    int32_t finer;          // the level has refined cells (finer levels exist)
    int level;
    int64_t n;              // cells per dimension
    int zc;                 // segment length in cells (power of two, divides n)
    const double *u_old;
    double *u_new;
    const double *dt;
    double *dt_next;
    double gamma, rho_floor, p_floor, cfl;
    int32_t *status;
};

// Riemann flux in the face-normal frame (HLLC, or the exact solver with HLLC fallback)
template <typename R, int RS>
__device__ __forceinline__ void col_solve(const R WL[NV], const R WR[NV], const Prm<R> &pr, int32_t *status,
                                          R Fn[NV])
{
    if (RS == AMR_RIEMANN_EXACT) {
        R ps, us;
        const R tol = sizeof(R) == 8 ? R(1e-14) : R(1e-6);
        const int e = exact_star(WL, WR, pr.gamma, tol, 50, ps, us);
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
}

// face between predicted cells pl (left) and pr_ (right) of rings QL, QR along DIR
template <typename R, int DIR, int PXY>
__device__ __forceinline__ void col_face(const R (*QL)[PXY], const R (*QR)[PXY], int pl, int pr_, const Prm<R> &pr,
                                         R WL[NV], R WR[NV])
{
    constexpr int S = NV + NV * DIR;
    R tL[NV], dL[NV], tR[NV], dR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        tL[v] = QL[v][pl]; dL[v] = QL[S + v][pl];
        tR[v] = QR[v][pr_]; dR[v] = QR[S + v][pr_];
    }
    face_state<DIR>(tL, dL, R(0.5), pr, WL);
    face_state<DIR>(tR, dR, R(-0.5), pr, WR);
}

template <int DIR, typename R, int N>
__device__ __forceinline__ void col_store(R (*F)[N], int r, const R Fn[NV])
{
    constexpr int N0 = DIR + 1, T1 = DIR == 0 ? 2 : 1, T2 = DIR == 2 ? 2 : 3;
    F[0][r] = Fn[0];
    F[N0][r] = Fn[1];
    F[T1][r] = Fn[2];
    F[T2][r] = Fn[3];
    F[4][r] = Fn[4];
}

template <typename R, int RS, int FX, int FY, bool FINER>
__global__ void __launch_bounds__(256) k_godunov_col(ColArgs a)
{
    using S = ColSmem<R, FX, FY, FINER>;
    constexpr int SX = S::SX, SY = S::SY;
    constexpr int QC = S::QC, QT = S::QT, QL = S::QL, QB = S::QB, QR = S::QR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    auto Qp = [&](int slot) { return reinterpret_cast<R (*)[QC]>(sm.Q[slot]); };
    // Q index of interior cell (ix, iy): row-major, the two 4-cell halves of a row swapped
    // in rows 4..7, so that a 4 x 8 block (the predictor's stores) and 8 x 4 blocks (the
    // faces' loads) each fall on 32 distinct banks
    static_assert(FX == 8, "the interior swizzle assumes rows of two 4-cell halves");
    auto qx = [](int ix, int iy) { return (ix ^ (((iy >> 2) & 1) << 2)) + FX * iy; };
    const TreeView &tv = a.tv;
    const int tid = threadIdx.x, nt = blockDim.x;
    Prm<R> pr;
    pr.gamma = to_work<R>(a.gamma); pr.rho_floor = to_work<R>(a.rho_floor); pr.p_floor = to_work<R>(a.p_floor);
    const R cflR = to_work<R>(a.cfl);
    const bool batch = a.n_inst > 0;
    const bool per[3] = {tv.bc[0] == AMR_BC_PERIODIC, tv.bc[2] == AMR_BC_PERIODIC, tv.bc[4] == AMR_BC_PERIODIC};
    unsigned long long my_dt = ~0ull;

    const double *uo[NV];
    double *un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        uo[v] = a.u_old + v * tv.ncell;
        un[v] = a.u_new + v * tv.ncell;
    }

    for (int64_t b = blockIdx.x; b < a.work; b += gridDim.x) {
        // geometry of this work item: the level (or the box), its column footprint and segment
        int l = a.level;
        int64_t n = a.n, wb = b;
        int32_t obase = 0;                        // batch: first oct of the box
        double dx, lam;
        double *dtn = a.dt_next;
        if (batch) {
            int lo = 0, hi = a.n_inst - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.inst_col_off[mid] <= b) lo = mid; else hi = mid - 1;
            }
            n = tv.inst_n[lo];
            wb = b - a.inst_col_off[lo];
            obase = int32_t(a.inst_oct_off[lo]);
            dx = tv.inst_dx[lo];
            lam = a.dt[lo] * double(n);
            dtn = a.dt_next ? a.dt_next + lo : nullptr;
        } else {
            dx = pow2(-l);
            lam = scale_pow2(*a.dt, l);           // dt / dx, exact
        }
        const int64_t M = n / 2;
        const R lamR = to_work<R>(lam);
        const R hl = R(0.5) * lamR;
        const R dxR = to_work<R>(dx);
        // cell coordinates, oct and cell ids fit in 32 bits (at most 2^12 cells per axis and
        // fewer than 2^27 octs)
        const int ni = int(n);
        const int64_t nfx = n / FX, nfy = n / FY;
        const int64_t fxy = wb % (nfx * nfy), seg = wb / (nfx * nfy);
        const int X0 = int(fxy % nfx) * FX - 2, Y0 = int(fxy / nfx) * FY - 2;   // stencil index 0
        const int z0 = int(seg) * a.zc;
        auto wrap = [&](int c, int axis) -> int {
            if (c >= 0 && c < ni) return c;
            if (per[axis]) return c < 0 ? c + ni : c - ni;   // within one period of the box
            return c < 0 ? 0 : ni - 1;             // outflow: clamp at this level
        };
        const int32_t Mi = int32_t(M);

        // the oct ids of the footprint's oct columns at oct layer L, wrapped or clamped like
        // the cells (X0, Y0 are even, so both cells of a footprint oct slot, and both planes
        // of a layer, land in one oct)
        constexpr int NO = (SX / 2) * (SY / 2);
        auto oct_fill = [&](int L, int o) {
            const int wx = wrap(X0 + 2 * (o % (SX / 2)), 0), wy = wrap(Y0 + 2 * (o / (SX / 2)), 1);
            const int32_t oi = (wx >> 1) + Mi * ((wy >> 1) + Mi * (wrap(2 * L, 2) >> 1));
            sm.oct[L & 3][o] = batch ? obase + oi : a.grid[oi];
        };
        // item q of the gather of oct layer L (cell planes 2L, 2L+1) of the stencil footprint
        // into the W ring
        auto gather_item = [&](int L, int q) {
            const int o = q >> 3, c = q & 7;
            const int i = 2 * (o % (SX / 2)) + (c & 1), j = 2 * (o / (SX / 2)) + ((c >> 1) & 1);
            const int zp = 2 * L + ((c >> 2) & 1);
            const int32_t cid = sm.oct[L & 3][o] * 8 + (wrap(X0 + i, 0) & 1) + 2 * (wrap(Y0 + j, 1) & 1) +
                                4 * (wrap(zp, 2) & 1);
            R Uw[NV], Wc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Uw[v] = to_work<R>(uo[v][cid]);
            cons_to_prim_w(Uw, pr, Wc);
#pragma unroll
            for (int v = 0; v < NV; ++v) sm.W[zp & 3][v][i + SX * j] = Wc[v];
            if constexpr (FINER) sm.ref[zp & 7][i + SX * j] = (tv.refmask[cid >> 3] >> (cid & 7)) & 1;
        };
        auto gather = [&](int L) {
            for (int q = tid; q < NO * 8; q += nt) gather_item(L, q);
        };
        // L2 prefetch of the oct rows (two 32-byte halves per variable) of oct layer L
        auto prefetch_item = [&](int L, int w) {
            const int o = w / (2 * NV), v = (w / 2) % NV, h = w & 1;
            const double *ptr = a.u_old + int64_t(v) * tv.ncell + int64_t(sm.oct[L & 3][o]) * 8 + 4 * h;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
        };
        auto q3 = [](int p) { return (p + 6) % 3; };   // planes start at z0 - 2 >= -2
        // MinMod slopes + MUSCL-Hancock predictor of planes p0 and p0+1 (of each, the QC
        // cells the faces read), one loop so that every warp of the CTA takes a share
        auto predict2 = [&](int p0, bool fill, int fillL) {
            // threads past the predictions fill the oct table of layer fillL
            if (fill)
                for (int w = tid - 2 * QC; w >= 0 && w < NO; w += nt) oct_fill(fillL, w);
            for (int r2 = tid; r2 < 2 * QC; r2 += nt) {
                const int dp = r2 >= QC, r = r2 - dp * QC, p = p0 + dp;
                const int s0 = p & 3, sm1 = (p - 1) & 3, sp1 = (p + 1) & 3, qs = q3(p);
                // item r: interior cells in blocks 4 wide and FY tall (an 8 x 4 block with
                // the W row stride of 12 would meet 2-way bank conflicts on every load),
                // then the strips, each cell at Q index qi
                int i, j, qi = r;
                static_assert(FX % 4 == 0, "interior blocks are 4 cells wide");
                if (r < QT) {
                    const int ix = 4 * (r / (4 * FY)) + r % 4, iy = (r / 4) % FY;
                    i = 2 + ix; j = 2 + iy; qi = qx(ix, iy);
                }
                else if (r < QL) { i = 2 + (r - QT); j = FY + 2; }
                else if (r < QB) { i = 1; j = 2 + (r - QL); }
                else if (r < QR) { i = 2 + (r - QB); j = 1; }
                else { i = FX + 2; j = 2 + (r - QR); }
                const int si = i + SX * j;
                R Wc[NV], Dl[3][NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) Wc[v] = sm.W[s0][v][si];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    Dl[0][v] = minmod(Wc[v] - sm.W[s0][v][si - 1], sm.W[s0][v][si + 1] - Wc[v]);
                    Dl[1][v] = minmod(Wc[v] - sm.W[s0][v][si - SX], sm.W[s0][v][si + SX] - Wc[v]);
                    Dl[2][v] = minmod(Wc[v] - sm.W[sm1][v][si], sm.W[sp1][v][si] - Wc[v]);
                }
                R Wt[NV];
                muscl_predict(Wc, Dl, hl, pr.gamma, Wt);
                R (*Qs)[QC] = Qp(qs);
#pragma unroll
                for (int v = 0; v < NV; ++v) Qs[v][qi] = Wt[v];
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int v = 0; v < NV; ++v) Qs[NV + NV * d + v][qi] = Dl[d][v];
            }
        };
        // z faces below planes j (face j-1 | j), for the listed planes
        auto zfaces = [&](int j0, int count) {
            const int qa = q3(j0 - 1), qb = q3(j0), qc = q3(j0 + 1);
            for (int r = tid; r < count * FX * FY; r += nt) {
                const int dj = r / (FX * FY);          // FX * FY is a power of two
                const int rr = r % (FX * FY), qz = qx(rr % FX, rr / FX);
                R WL[NV], WR[NV], Fn[NV];
                col_face<R, 2, QC>(Qp(dj ? qb : qa), Qp(dj ? qc : qb), qz, qz, pr, WL, WR);
                col_solve<R, RS>(WL, WR, pr, a.status, Fn);
                col_store<2>(sm.Fz[dj ? qc : qb], rr, Fn);
            }
        };

        constexpr int NXF = FY * (FX + 1), NYF = (FY + 1) * FX;
        constexpr int NG = (SX / 2) * (SY / 2) * 8, NU = 2 * FX * FY, NR = (FX / 2) * (FY / 2) * NV;
        // x and y faces of planes k, k+1 and z faces below planes k+1, k+2 (those of slab k),
        // one loop over all three kinds: the face states are formed per kind, the Riemann
        // solve is shared (a warp that straddles two kinds solves once), the flux is stored
        // per kind
        constexpr int NF = 2 * (NXF + NYF + FX * FY), NP = NO * NV * 2;
        auto slab_faces = [&](int k, bool pf, int pfL) {
            const int qk0 = q3(k), qk1 = q3(k + 1), qk2 = q3(k + 2);
            // the prefetches of oct layer pfL go out first; nothing waits on them
            if (pf)
                for (int w = tid; w < NP; w += nt) prefetch_item(pfL, w);
            for (int r = tid; r < NF; r += nt) {
                R WL[NV], WR[NV], Fn[NV];
                int kind, dz, rr;
                if (r < 2 * NXF) {
                    // x faces, stored at rr: for rr < FX*FY the face on the right of interior
                    // cell rr, else the face on the left of interior column 0 in row rr - FX*FY
                    kind = 0; dz = r / NXF; rr = r % NXF;
                    int pl, pq;
                    if (rr < QT) {
                        const int ix = rr % FX, iy = rr / FX;
                        pl = qx(ix, iy);
                        pq = ix == FX - 1 ? QR + iy : qx(ix + 1, iy);
                    } else {
                        pl = QL + (rr - QT);
                        pq = qx(0, rr - QT);
                    }
                    const int qs = dz ? qk1 : qk0;
                    col_face<R, 0, QC>(Qp(qs), Qp(qs), pl, pq, pr, WL, WR);
                } else if (r < 2 * (NXF + NYF)) {
                    // y faces, stored at rr = col + FX * fa (fa = 0: below row 0, strip B)
                    const int r2 = r - 2 * NXF;
                    kind = 1; dz = r2 / NYF; rr = r2 % NYF;
                    const int col = rr % FX, fa = rr / FX;
                    const int pl = fa == 0 ? QB + col : qx(col, fa - 1), pq = fa == FY ? QT + col : qx(col, fa);
                    const int qs = dz ? qk1 : qk0;
                    col_face<R, 1, QC>(Qp(qs), Qp(qs), pl, pq, pr, WL, WR);
                } else {
                    // the face below plane k+1+dz: between planes k+dz and k+1+dz
                    const int r2 = r - 2 * (NXF + NYF);
                    kind = 2; dz = r2 / (FX * FY); rr = r2 % (FX * FY);
                    const int qz = qx(rr % FX, rr / FX);
                    col_face<R, 2, QC>(Qp(dz ? qk1 : qk0), Qp(dz ? qk2 : qk1), qz, qz, pr, WL, WR);
                }
                col_solve<R, RS>(WL, WR, pr, a.status, Fn);
                if (kind == 0) col_store<0>(sm.Fx[dz], rr, Fn);
                else if (kind == 1) col_store<1>(sm.Fy[dz], rr, Fn);
                else col_store<2>(sm.Fz[dz ? qk2 : qk1], rr, Fn);
            }
        };
        // FP64 update of cell q of slab k (fused CFL candidate); keeps the new state
        // the old state of cell q of slab k, loaded ahead of the update
        auto update_load = [&](int k, int q, double Uo[NV]) -> int32_t {
            const int dz = q / (FX * FY), r = q % (FX * FY), x = r % FX, y = r / FX;
            const int o = ((x + 2) >> 1) + (SX / 2) * ((y + 2) >> 1);
            const int32_t cid = sm.oct[(k >> 1) & 3][o] * 8 + (x & 1) + 2 * (y & 1) + 4 * dz;
#pragma unroll
            for (int v = 0; v < NV; ++v) Uo[v] = uo[v][cid];
            return cid;
        };
        auto update = [&](int k, int q, const double Uo[NV], int32_t cid) {
            const int dz = q / (FX * FY), r = q % (FX * FY), x = r % FX, y = r / FX;
            const int p = k + dz;
            const int ub = (k >> 1) & 1;
            // with finer levels: a refined cell is left to the restriction, and a face whose
            // other side is refined carries no flux here (the finer level supplies it)
            bool sk[6] = {false, false, false, false, false, false};
            const int uo8 = (x >> 1) + (FX / 2) * (y >> 1), uc = (x & 1) + 2 * (y & 1) + 4 * dz;
            if constexpr (FINER) {
                const int si = (x + 2) + SX * (y + 2);
                const uint8_t *rp = sm.ref[p & 7];
                if (rp[si]) {
                    if (uc == 0) sm.cell0[ub][uo8] = -1;
                    return;
                }
                sk[0] = rp[si - 1]; sk[1] = rp[si + 1]; sk[2] = rp[si - SX]; sk[3] = rp[si + SX];
                sk[4] = sm.ref[(p - 1) & 7][si]; sk[5] = sm.ref[(p + 1) & 7][si];
            }
            R dU[NV] = {0, 0, 0, 0, 0};
            const int fzl = q3(p), fzu = fzl == 2 ? 0 : fzl + 1;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (!sk[0]) dU[v] = dU[v] + sm.Fx[dz][v][x ? x - 1 + FX * y : FX * FY + y];
                if (!sk[1]) dU[v] = dU[v] - sm.Fx[dz][v][x + FX * y];
                if (!sk[2]) dU[v] = dU[v] + sm.Fy[dz][v][x + FX * y];
                if (!sk[3]) dU[v] = dU[v] - sm.Fy[dz][v][x + FX * (y + 1)];
                if (!sk[4]) dU[v] = dU[v] + sm.Fz[fzl][v][r];
                if (!sk[5]) dU[v] = dU[v] - sm.Fz[fzu][v][r];
            }
            const bool nbref = sk[0] || sk[1] || sk[2] || sk[3] || sk[4] || sk[5];
            double Un[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (sizeof(R) == 8) Un[v] = Uo[v] + lam * to_state(dU[v]);
                else Un[v] = Uo[v] + to_state(lamR * dU[v]);
                un[v][cid] = Un[v];
                sm.U[ub][uc][uo8 * NV + v] = Un[v];
            }
            if (!state_finite<R>(Un)) set_error(a.status, AMR_ENONPHYSICAL);
            if (uc == 0) sm.cell0[ub][uo8] = cid;
            if (dtn && !nbref) my_dt = min(my_dt, (unsigned long long)__double_as_longlong(cfl_candidate<R>(Un, pr, cflR, dxR)));
        };
        // restriction of the father of one oct of slab k (its eight cells in order), variable v
        auto restrict_one = [&](int k, int w) {
            const int o = w / NV, v = w % NV;
            const int ub = (k >> 1) & 1;
            const int32_t c0 = sm.cell0[ub][o];
            if (c0 < 0) return;                       // a refined cell: the oct is not restricted here
            const int32_t oct = c0 >> 3;
            if (!tv.fused[oct]) return;
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < 8; ++c) acc += sm.U[ub][c][w];     // w = o * NV + v
            a.u_new[v * tv.ncell + tv.father[oct]] = 0.125 * acc;    // v is not a constant here
        };

        // prologue, keeping to the ring sizes (W: 4 planes, Q and Fz: 3): planes z0-2 .. z0+1,
        // predictions z0-1, z0, the z face below z0 together with planes z0+2, z0+3 (which
        // replace the dead z0-2, z0-1), predictions z0+1, z0+2 (replacing z0-1), the faces
        // of slab z0; first the oct tables of layers z0/2-1 .. z0/2+2
        for (int w = tid; w < 4 * NO; w += nt) oct_fill(z0 / 2 - 1 + w / NO, w % NO);
        __syncthreads();
        gather(z0 / 2 - 1);
        gather(z0 / 2);
        __syncthreads();
        predict2(z0 - 1, false, 0);
        __syncthreads();
        zfaces(z0, 1);
        gather(z0 / 2 + 1);
        __syncthreads();
        predict2(z0 + 1, false, 0);
        __syncthreads();
        slab_faces(z0, false, 0);
        __syncthreads();
        // per slab k: {update of slab k, gather of the layer slab k+2 needs, restriction of
        // slab k-2} share one phase, then the predictions and faces of slab k+2
        static_assert(NU <= 256, "one update item per thread of a 256-thread CTA");
        for (int k = z0; k < z0 + a.zc; k += 2) {
            const bool more = k + 2 < z0 + a.zc;
            const int nwork = NU + (more ? NG : 0) + (k > z0 ? NR : 0);
            // a thread with an update item loads its old state first, so that the load
            // latency overlaps its gather or restriction item; the update follows them
            const bool upd = tid < NU;
            double Uo[NV];
            int32_t ucid = 0;
            if (upd) ucid = update_load(k, tid, Uo);
            for (int w = upd ? tid + nt : tid; w < nwork; w += nt) {
                if (w < NU) {
                    // not reached: update items are the threads' first items
                } else if (more && w < NU + NG) {
                    gather_item(k / 2 + 2, w - NU);
                } else {
                    if (!batch) restrict_one(k - 2, w - NU - (more ? NG : 0));
                }
            }
            if (upd) update(k, tid, Uo, ucid);
            __syncthreads();
            if (!more) break;
            // the oct table of layer k/2+3 (slot of the dead layer k/2-1), which the gather of
            // slab k+2 and the update of slab k+6 read, is filled beside the predictions; the
            // layer's state rows are prefetched into L2 beside the faces
            const bool ahead = k + 4 < z0 + a.zc;
            predict2(k + 3, ahead, k / 2 + 3);
            __syncthreads();
            slab_faces(k + 2, ahead, k / 2 + 3);
            __syncthreads();
        }
        // the last slab's restriction
        if (!batch)
            for (int w = tid; w < NR; w += nt) restrict_one(z0 + a.zc - 2, w);
        if (batch && dtn) {
            // boxes have their own time steps: reduce this work item's candidates now
            for (int off = 16; off > 0; off >>= 1) my_dt = min(my_dt, __shfl_xor_sync(0xffffffffu, my_dt, off));
            if ((tid & 31) == 0 && my_dt != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(dtn), my_dt);
            my_dt = ~0ull;
        }
        __syncthreads();
    }
    if (a.dt_next) {
        for (int off = 16; off > 0; off >>= 1) my_dt = min(my_dt, __shfl_xor_sync(0xffffffffu, my_dt, off));
        if ((tid & 31) == 0 && my_dt != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(a.dt_next), my_dt);
    }
}

template <typename R, int RS>
amr_status launch_col(const amr_tree *t, const hydro_params *p, const double *u_old, double *u_new, const double *dt,
                      double *dt_next, cudaStream_t st)
{
    constexpr int FX = 8, FY = 8;
    ColArgs a;
    a.tv = make_view(t);
    a.grid = t->grid;
    a.n_inst = t->n_inst;
    a.inst_col_off = t->inst_col_off;
    a.inst_oct_off = t->inst_oct_off;
    a.finer = t->n_inst == 0 && t->grid_level < t->levelmax;
    if (t->n_inst > 0) {
        a.level = 0;
        a.n = 0;
        a.zc = 16;
        a.work = t->col_work;
    } else {
        a.level = t->grid_level;
        a.n = int64_t(1) << t->grid_level;
        // longest segment (at most 64 cells, fewer prologue planes per cell) that still
        // gives two waves of four CTAs per SM
        int dev = 0, nsm = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        a.zc = a.n < 64 ? int(a.n) : 64;
        while (a.zc > 16 && (a.n / FX) * (a.n / FY) * (a.n / a.zc) < int64_t(8) * nsm) a.zc /= 2;
        const int want = p->col_seg;
        if (want >= 2 && want <= a.n && (want & (want - 1)) == 0) a.zc = want;
        a.work = (a.n / FX) * (a.n / FY) * (a.n / a.zc);
    }
    a.u_old = u_old; a.u_new = u_new; a.dt = dt; a.dt_next = dt_next;
    a.gamma = p->gamma; a.rho_floor = p->rho_floor; a.p_floor = p->p_floor; a.cfl = p->cfl;
    a.status = p->d_status;
    const bool finer = a.finer != 0;
    const size_t bytes = finer ? sizeof(ColSmem<R, FX, FY, true>) : sizeof(ColSmem<R, FX, FY, false>);
    auto kern = finer ? k_godunov_col<R, RS, FX, FY, true> : k_godunov_col<R, RS, FX, FY, false>;
    AMR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    kern<<<unsigned(a.work < 1048576 ? a.work : 1048576), 256, bytes, st>>>(a);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

}  // namespace amr
