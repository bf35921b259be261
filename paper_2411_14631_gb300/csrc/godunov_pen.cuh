// godunov_fine on a complete level, FP32 path: the column-per-thread ("pencil") form of
// the z-column update.
//
// A CTA owns a 16 x 16-cell footprint of the level and marches a segment of its column
// in z one cell plane at a time.  Each of its 256 threads owns one (x, y) column; on top
// of that, warps 0 and 1 predict the four one-cell strips around the footprint (the
// left / right and bottom / top neighbours of the edge cells), warp 2 solves the faces on
// the footprint's right and top edges, and warps 3-7 gather the stencil cells beyond the
// first 256 (each role warp-uniform).  Per plane p:
//   A  gather of stencil plane p+2 (20 x 20 cells, FP64 -> FP32 primitives) into a ring
//      of four planes in shared memory (loads issued first, stores last);
//   B  slopes and MUSCL-Hancock predictor of plane p: the interior thread keeps its
//      cell's -x, -y, +z and -z face states in registers and publishes +x and +y in
//      shared memory; warps 0 and 1 publish the strips' inward face states;
//   C  the z face below plane p from two states the thread holds (no shared memory);
//   -- one barrier --
//   E  FP64 update of plane p-1: its own x-left and y-left fluxes and both z fluxes come
//      from registers, the x-right and y-right fluxes from the neighbours' shared slots;
//   D  the x and y faces on the left and bottom of the thread's cell of plane p (left
//      states from shared memory, right states from registers), published for the
//      neighbours' updates in the next plane;
//   R  restriction of the oct layer finished two planes earlier (one thread per
//      (oct, variable), children in cell order).
// Shared buffers alternate with the plane's parity, so one barrier per plane orders
// every producer before its consumers.  Per cell the arithmetic is the tile kernel's, in
// the same order (gather conversion, predictor, face states, Riemann solve, flux sum
// x-left, x-right, y-left, y-right, z-below, z-above, FP64 update, CFL candidate,
// restriction), so the states are bitwise those of the other kernels.
#pragma once
#include "godunov_col.cuh"

namespace amr {

struct PenGeo {
    static constexpr int FX = 16, FY = 16;            // footprint (cells)
    static constexpr int SX = FX + 4, SY = FY + 4;    // stencil plane (cells)
    static constexpr int NS = SX * SY;                // 400
    static constexpr int NI = FX * FY;                // 256 interior columns = interior threads
    static constexpr int OX = SX / 2, NO = OX * (SY / 2);   // footprint oct columns (10 x 10)
    static constexpr int NT = NI;                     // one thread per column
    static constexpr int NXG = NS - NI;               // gather items beyond the first 256 (144)
    static constexpr int XG0 = 96;                    // first thread with one of them (warp 3)
};

template <bool FINER> struct PenSmem {
    using G = PenGeo;
    // primitive stencil planes, ring slot = plane & 3: (rho, u, v, w) and p
    float4 Wv[4][G::NS];
    float Wp[4][G::NS];
    // face states in the face-normal frame, by plane parity:
    //   Sx: +x states of interior cell x + 16 y, the left strip's at NI + y;
    //   Sy: +y states of interior cells, the bottom strip's at NI + x;
    //   Sr: -x states of the right strip (row y at y), -y of the top strip (column x at 16 + x)
    float4 Sx4[2][G::NI + 16];
    float Sx1[2][G::NI + 16];
    float4 Sy4[2][G::NI + 16];
    float Sy1[2][G::NI + 16];
    float4 Sr4[2][32];
    float Sr1[2][32];
    // fluxes (face-normal frame) by plane parity: the face on the left of interior x = 1..15
    // and the right edge face at (x - 1) + 16 y; the face below y = 1..15 and the top edge
    // face at x + 16 (y - 1)
    float4 Gx4[2][G::NI];
    float Gx1[2][G::NI];
    float4 Gy4[2][G::NI];
    float Gy1[2][G::NI];
    // new states of the last three planes (slot = plane % 3), [variable][x + 16 y]
    double Ur[3][NV][G::NI];
    int32_t oct[8][G::NO];                            // oct id per footprint oct column, slot = layer & 7
    uint8_t ref[FINER ? 8 : 1][FINER ? G::NS : 1];    // refined flag per stencil cell, slot = plane & 7
};

__device__ __forceinline__ void pen_ld(const float4 *a4, const float *a1, int i, float W[NV])
{
    const float4 q = a4[i];
    W[0] = q.x; W[1] = q.y; W[2] = q.z; W[3] = q.w; W[4] = a1[i];
}

__device__ __forceinline__ void pen_st(float4 *a4, float *a1, int i, const float W[NV])
{
    a4[i] = make_float4(W[0], W[1], W[2], W[3]);
    a1[i] = W[4];
}

// dU += s F for the face-normal flux Fn of a face of direction D
template <int D> __device__ __forceinline__ void pen_acc(float dU[NV], const float Fn[NV], bool plus)
{
    constexpr int N0 = D + 1, T1 = D == 0 ? 2 : 1, T2 = D == 2 ? 2 : 3;
    float F[NV];
    F[0] = Fn[0]; F[N0] = Fn[1]; F[T1] = Fn[2]; F[T2] = Fn[3]; F[4] = Fn[4];
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[v] = plus ? dU[v] + F[v] : dU[v] - F[v];
}

template <int RS, bool FINER>
__global__ void __launch_bounds__(PenGeo::NT, 2) k_godunov_pen(ColArgs a)
{
    using G = PenGeo;
    using S = PenSmem<FINER>;
    constexpr int SX = G::SX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const TreeView &tv = a.tv;
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const bool xg = tid >= G::XG0 && tid < G::XG0 + G::NXG;      // has a second gather item
    const int x = lane & 15, y = 2 * (tid >> 5) + (lane >> 4);   // interior column (interior threads)
    const int ci = x + G::FX * y;                                  // its interior index
    const int sio = (x + 2) + SX * (y + 2);                        // its stencil index
    const int oo = ((x + 2) >> 1) + G::OX * ((y + 2) >> 1);        // its footprint oct column
    const int cxy = (x & 1) + 2 * (y & 1);                         // its cell bits in x and y
    Prm<float> pr;
    pr.gamma = d2f_bits(a.gamma); pr.rho_floor = d2f_bits(a.rho_floor); pr.p_floor = d2f_bits(a.p_floor);
    const float cflR = d2f_bits(a.cfl);
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
        // ---- geometry of this work item: the level (or box), footprint and z segment
        int64_t n = a.n, wb = b;
        int32_t obase = 0;
        double dx, lam;
        double *dtn = a.dt_next;
        int zc = a.zc;
        if (batch) {
            // box offsets in 16 x 16 x 16 items: the 8 x 8 x 16 offsets of the tree / 4
            int lo = 0, hi = a.n_inst - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.inst_col_off[mid] / 4 <= b) lo = mid; else hi = mid - 1;
            }
            n = tv.inst_n[lo];
            wb = b - a.inst_col_off[lo] / 4;
            obase = int32_t(a.inst_oct_off[lo]);
            dx = tv.inst_dx[lo];
            lam = a.dt[lo] * double(n);
            dtn = a.dt_next ? a.dt_next + lo : nullptr;
            zc = 16;
        } else {
            dx = pow2(-a.level);
            lam = scale_pow2(*a.dt, a.level);   // dt / dx, exact
        }
        const float lamR = d2f_bits(lam), hl = 0.5f * lamR, dxR = d2f_bits(dx);
        const int ni = int(n), nf = ni / G::FX;
        const int fxy = int(wb % (nf * nf)), seg = int(wb / (nf * nf));
        const int X0 = (fxy % nf) * G::FX - 2, Y0 = (fxy / nf) * G::FY - 2;   // stencil index 0
        const int z0 = seg * zc, z1 = min(z0 + zc, ni);                        // planes [z0, z1)
        const int32_t Mi = int32_t(n / 2);
        auto wrap = [&](int c, int axis) -> int {
            if (c >= 0 && c < ni) return c;
            if (per[axis]) return c < 0 ? c + ni : c - ni;
            return c < 0 ? 0 : ni - 1;
        };
        // oct ids of the footprint's oct columns at oct layer L (wrapped or clamped like the cells)
        auto oct_fill = [&](int L, int o) {
            const int wx = wrap(X0 + 2 * (o % G::OX), 0), wy = wrap(Y0 + 2 * (o / G::OX), 1);
            const int32_t oi = (wx >> 1) + Mi * ((wy >> 1) + Mi * (wrap(2 * L, 2) >> 1));
            sm.oct[L & 7][o] = batch ? obase + oi : a.grid[oi];
        };
        // gather items: stencil cell q (quads of the 2 x 2 cells of one oct column, so four
        // lanes read 32 contiguous bytes of a variable): packed stencil index | oct column
        // << 9 | x-y cell bits << 16.  Thread t: item t, and item 256 + t - 96 for t in [96, 240).
        auto gitem = [&](int q) -> int {
            const int o = q >> 2, sub = q & 3;
            const int i = 2 * (o % G::OX) + (sub & 1), j = 2 * (o / G::OX) + (sub >> 1);
            const int cb = (wrap(X0 + i, 0) & 1) + 2 * (wrap(Y0 + j, 1) & 1);
            return (i + SX * j) | (o << 9) | (cb << 16);
        };
        const int gpk0 = gitem(tid);
        const int gpk1 = xg ? gitem(G::NI + tid - G::XG0) : 0;
        // load of gather item pk of stencil plane z (FP64 state), then conversion and store
        auto gload = [&](int pk, int z, double U[NV]) -> int32_t {
            const int o = (pk >> 9) & 127, cb = pk >> 16;
            const int32_t cid = sm.oct[(z >> 1) & 7][o] * 8 + cb + 4 * (wrap(z, 2) & 1);
#pragma unroll
            for (int v = 0; v < NV; ++v) U[v] = uo[v][cid];
            return cid;
        };
        auto gstore = [&](int pk, int z, const double U[NV], int32_t cid) {
            const int si = pk & 511;
            float Uw[NV], Wc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Uw[v] = d2f_bits(U[v]);
            cons_to_prim_w(Uw, pr, Wc);
            pen_st(sm.Wv[z & 3], sm.Wp[z & 3], si, Wc);
            if constexpr (FINER) sm.ref[z & 7][si] = (tv.refmask[cid >> 3] >> (cid & 7)) & 1;
        };
        auto gather_all = [&](int z) {   // this thread's items, one after the other
            double U[NV];
            int32_t cid = gload(gpk0, z, U);
            gstore(gpk0, z, U, cid);
            if (xg) {
                cid = gload(gpk1, z, U);
                gstore(gpk1, z, U, cid);
            }
        };
        // slopes + predictor of stencil cell si of plane p
        auto predict = [&](int p, int si, float Wt[NV], float Dl[3][NV]) {
            const int s0 = p & 3, sm1 = (p - 1) & 3, sp1 = (p + 1) & 3;
            float Wc[NV], Wa[NV], Wb[NV];
            pen_ld(sm.Wv[s0], sm.Wp[s0], si, Wc);
            pen_ld(sm.Wv[s0], sm.Wp[s0], si - 1, Wa);
            pen_ld(sm.Wv[s0], sm.Wp[s0], si + 1, Wb);
#pragma unroll
            for (int v = 0; v < NV; ++v) Dl[0][v] = minmod(Wc[v] - Wa[v], Wb[v] - Wc[v]);
            pen_ld(sm.Wv[s0], sm.Wp[s0], si - SX, Wa);
            pen_ld(sm.Wv[s0], sm.Wp[s0], si + SX, Wb);
#pragma unroll
            for (int v = 0; v < NV; ++v) Dl[1][v] = minmod(Wc[v] - Wa[v], Wb[v] - Wc[v]);
            pen_ld(sm.Wv[sm1], sm.Wp[sm1], si, Wa);
            pen_ld(sm.Wv[sp1], sm.Wp[sp1], si, Wb);
#pragma unroll
            for (int v = 0; v < NV; ++v) Dl[2][v] = minmod(Wc[v] - Wa[v], Wb[v] - Wc[v]);
            muscl_predict(Wc, Dl, hl, pr.gamma, Wt);
        };
        // restriction of the father of footprint oct (w & 63) of layer k, variable w >> 6
        auto restrict_item = [&](int k, int w) {
            const int v = w >> 6, o = w & 63, ox = o & 7, oy = o >> 3;
            const int32_t oct = sm.oct[k & 7][(ox + 1) + G::OX * (oy + 1)];
            if (!tv.fused[oct]) return;
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                acc += sm.Ur[(2 * k + (c >> 2)) % 3][v][(2 * ox + (c & 1)) + G::FX * (2 * oy + ((c >> 1) & 1))];
            a.u_new[v * tv.ncell + tv.father[oct]] = 0.125 * acc;
        };
        auto restrict_layer = [&](int k) {
            if (batch) return;
            restrict_item(k, tid);
            if (wid == 2) {                               // the 64 items beyond the first 256
                restrict_item(k, G::NI + lane);
                restrict_item(k, G::NI + 32 + lane);
            }
        };

        // ---- prologue: oct tables of layers z0/2-1 .. z0/2+2, stencil planes z0-2 .. z0
        for (int w = tid; w < 4 * G::NO; w += G::NT) oct_fill(z0 / 2 - 1 + w / G::NO, w % G::NO);
        __syncthreads();
        for (int z = z0 - 2; z <= z0; ++z) gather_all(z);
        __syncthreads();

        float pz[NV], fz[NV], fzp[NV], fxo[NV], fyo[NV];   // interior thread state between planes
#pragma unroll
        for (int v = 0; v < NV; ++v) { pz[v] = 0.f; fz[v] = 0.f; fzp[v] = 0.f; fxo[v] = 0.f; fyo[v] = 0.f; }
        for (int p = z0 - 1; p <= z1; ++p) {
            const bool first = p == z0 - 1, last = p == z1, mid = !first && !last;
            const int q = p - 1;                          // plane updated in this iteration
            const bool upd = q >= z0;
            const bool gat = p + 2 <= z1 + 1;
            // old state of the cell to update, and this thread's first gather item: loads first
            double Uo[NV], Ug[NV], Ug1[NV];
            int32_t ucid = 0, gcid = 0, gcid1 = 0;
            if (upd) {
                ucid = sm.oct[(q >> 1) & 7][oo] * 8 + cxy + 4 * (q & 1);
#pragma unroll
                for (int v = 0; v < NV; ++v) Uo[v] = uo[v][ucid];
            }
            if (gat) gcid = gload(gpk0, p + 2, Ug);
            if (gat && xg) gcid1 = gload(gpk1, p + 2, Ug1);
            // oct table of layer (p+5)/2, read by the L2 prefetch of the next plane and by the
            // gather four planes on
            if ((p & 1) && tid < G::NO) {
                const int L = (p + 5) >> 1;
                if (L > z0 / 2 + 2 && 2 * L <= z1 + 1) oct_fill(L, tid);
            }
            // L2 prefetch of oct layer (p+4)/2 (stencil planes p+4 and p+5, gathered two and
            // three planes on): the two 32-byte sectors of each oct's 64-byte row per variable
            // (a bulk prefetch per row was slower than the two sector prefetches)
            if (!(p & 1) && p + 4 <= z1 + 1) {
                const int L = (p + 4) >> 1;
                for (int w = tid; w < G::NO * NV; w += G::NT) {
                    const int o = w / NV, v = w - (w / NV) * NV;
                    const double *src = a.u_old + int64_t(v) * tv.ncell + int64_t(sm.oct[L & 7][o]) * 8;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(src));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(src + 4));
                }
            }
            float mx[NV], my[NV];
            {
                // ---- B: predictor of the thread's cell of plane p
                float Wt[NV], Dl[3][NV];
                predict(p, sio, Wt, Dl);
                if (!first) {
                    // ---- C: the z face below plane p
                    float mz[NV], Fn[NV];
                    face_state<2>(Wt, Dl[2], -0.5f, pr, mz);
                    col_solve<float, RS>(pz, mz, pr, a.status, Fn);
#pragma unroll
                    for (int v = 0; v < NV; ++v) { fzp[v] = fz[v]; fz[v] = Fn[v]; }
                }
                if (!last) face_state<2>(Wt, Dl[2], 0.5f, pr, pz);
                if (mid) {
                    float st[NV];
                    face_state<0>(Wt, Dl[0], 0.5f, pr, st);
                    pen_st(sm.Sx4[p & 1], sm.Sx1[p & 1], ci, st);
                    face_state<1>(Wt, Dl[1], 0.5f, pr, st);
                    pen_st(sm.Sy4[p & 1], sm.Sy1[p & 1], ci, st);
                    face_state<0>(Wt, Dl[0], -0.5f, pr, mx);
                    face_state<1>(Wt, Dl[1], -0.5f, pr, my);
                }
            }
            if (mid && wid < 2) {
                // ---- B: the strips.  Warp 0: the left (lanes 0-15, +x state) and right (-x)
                // neighbour of row lane & 15; warp 1: the bottom (+y) and top (-y) neighbour of
                // column lane & 15
                const bool lo = lane < 16;
                const float half = lo ? 0.5f : -0.5f;
                const int r = lane & 15;
                float Wt[NV], Dl[3][NV], st[NV];
                if (wid == 0) {
                    predict(p, (lo ? 1 : G::FX + 2) + SX * (2 + r), Wt, Dl);
                    face_state<0>(Wt, Dl[0], half, pr, st);
                    if (lo) pen_st(sm.Sx4[p & 1], sm.Sx1[p & 1], G::NI + r, st);
                    else pen_st(sm.Sr4[p & 1], sm.Sr1[p & 1], r, st);
                } else {
                    predict(p, (2 + r) + SX * (lo ? 1 : G::FY + 2), Wt, Dl);
                    face_state<1>(Wt, Dl[1], half, pr, st);
                    if (lo) pen_st(sm.Sy4[p & 1], sm.Sy1[p & 1], G::NI + r, st);
                    else pen_st(sm.Sr4[p & 1], sm.Sr1[p & 1], 16 + r, st);
                }
            }
            if (gat) gstore(gpk0, p + 2, Ug, gcid);
            if (gat && xg) gstore(gpk1, p + 2, Ug1, gcid1);
            __syncthreads();

            // ---- E: FP64 update of plane q = p - 1
            if (upd) {
                const int qb = q & 1;
                bool sk[6] = {false, false, false, false, false, false};
                bool skip = false;
                if constexpr (FINER) {
                    const uint8_t *rp = sm.ref[q & 7];
                    skip = rp[sio] != 0;
                    sk[0] = rp[sio - 1]; sk[1] = rp[sio + 1]; sk[2] = rp[sio - SX]; sk[3] = rp[sio + SX];
                    sk[4] = sm.ref[(q - 1) & 7][sio]; sk[5] = sm.ref[(q + 1) & 7][sio];
                }
                if (!skip) {
                    float fxh[NV], fyh[NV];
                    pen_ld(sm.Gx4[qb], sm.Gx1[qb], ci, fxh);      // the face on the right of x
                    pen_ld(sm.Gy4[qb], sm.Gy1[qb], ci, fyh);      // the face above y
                    float dU[NV] = {0.f, 0.f, 0.f, 0.f, 0.f};
                    // the order of the other kernels: x-left, x-right, y-left, y-right, z-below, z-above
                    if (!sk[0]) pen_acc<0>(dU, fxo, true);
                    if (!sk[1]) pen_acc<0>(dU, fxh, false);
                    if (!sk[2]) pen_acc<1>(dU, fyo, true);
                    if (!sk[3]) pen_acc<1>(dU, fyh, false);
                    if (!sk[4]) pen_acc<2>(dU, fzp, true);
                    if (!sk[5]) pen_acc<2>(dU, fz, false);
                    double Un[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        Un[v] = Uo[v] + f2d_bits(lamR * dU[v]);
                        un[v][ucid] = Un[v];
                        sm.Ur[q % 3][v][ci] = Un[v];
                    }
                    if (!state_finite<float>(Un)) set_error(a.status, AMR_ENONPHYSICAL);
                    const bool nbref = sk[0] || sk[1] || sk[2] || sk[3] || sk[4] || sk[5];
                    if (dtn && !nbref)
                        my_dt = min(my_dt, (unsigned long long)__double_as_longlong(
                                               cfl_candidate<float>(Un, pr, cflR, dxR)));
                }
            }
            // ---- D: x and y faces of plane p
            if (mid) {
                const int pb = p & 1;
                {
                    float WL[NV], Fn[NV];
                    pen_ld(sm.Sx4[pb], sm.Sx1[pb], x ? ci - 1 : G::NI + y, WL);
                    col_solve<float, RS>(WL, mx, pr, a.status, Fn);
#pragma unroll
                    for (int v = 0; v < NV; ++v) fxo[v] = Fn[v];
                    if (x) pen_st(sm.Gx4[pb], sm.Gx1[pb], ci - 1, Fn);
                    pen_ld(sm.Sy4[pb], sm.Sy1[pb], y ? ci - G::FX : G::NI + x, WL);
                    col_solve<float, RS>(WL, my, pr, a.status, Fn);
#pragma unroll
                    for (int v = 0; v < NV; ++v) fyo[v] = Fn[v];
                    if (y) pen_st(sm.Gy4[pb], sm.Gy1[pb], ci - G::FX, Fn);
                }
                if (wid == 2) {
                    // edge faces: lane l < 16 the right face of row l, else the top face of column l - 16
                    const int r = lane & 15;
                    const int li = lane < 16 ? (G::FX - 1) + G::FX * r : r + G::FX * (G::FY - 1);
                    float WL[NV], WR[NV], Fn[NV];
                    if (lane < 16) pen_ld(sm.Sx4[pb], sm.Sx1[pb], li, WL);
                    else pen_ld(sm.Sy4[pb], sm.Sy1[pb], li, WL);
                    pen_ld(sm.Sr4[pb], sm.Sr1[pb], lane, WR);
                    col_solve<float, RS>(WL, WR, pr, a.status, Fn);
                    if (lane < 16) pen_st(sm.Gx4[pb], sm.Gx1[pb], li, Fn);
                    else pen_st(sm.Gy4[pb], sm.Gy1[pb], li, Fn);
                }
            }
            // ---- R: restriction of oct layer k = (p - 3) / 2 (planes 2k, 2k+1 updated and
            // visible since this plane's barrier)
            if ((p & 1) && p >= z0 + 3) restrict_layer((p - 3) >> 1);
        }
        __syncthreads();
        restrict_layer((z1 - 2) >> 1);                    // the segment's last oct layer
        if (batch && dtn) {
            for (int off = 16; off > 0; off >>= 1) my_dt = min(my_dt, __shfl_xor_sync(0xffffffffu, my_dt, off));
            if (lane == 0 && my_dt != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(dtn), my_dt);
            my_dt = ~0ull;
        }
        __syncthreads();
    }
    if (a.dt_next) {
        for (int off = 16; off > 0; off >>= 1) my_dt = min(my_dt, __shfl_xor_sync(0xffffffffu, my_dt, off));
        if (lane == 0 && my_dt != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(a.dt_next), my_dt);
    }
}

// Launch of the pencil kernel for the deepest complete level (or the box batch): zc is
// the z segment of a CTA (0: the default), ragged at the top when it does not divide the
// level.  Requires 16 | n (every box, in batch mode).
template <int RS>
amr_status launch_pen(const amr_tree *t, const hydro_params *p, const double *u_old, double *u_new, const double *dt,
                      double *dt_next, int zc, cudaStream_t st)
{
    using G = PenGeo;
    ColArgs a;
    a.tv = make_view(t);
    a.grid = t->grid;
    a.n_inst = t->n_inst;
    a.inst_col_off = t->inst_col_off;
    a.inst_oct_off = t->inst_oct_off;
    a.finer = t->n_inst == 0 && t->grid_level < t->levelmax;
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (t->n_inst > 0) {
        if (t->col_work <= 0 || t->col_work % 4) return AMR_EINVAL;
        a.level = 0;
        a.n = 0;
        a.zc = 16;
        a.work = t->col_work / 4;
    } else {
        a.level = t->grid_level;
        a.n = int64_t(1) << t->grid_level;
        if (a.n % G::FX) return AMR_EINVAL;
        if (zc <= 0) {
            // default: the even segment length in [8, 64] with the shortest estimated makespan,
            // waves of two CTAs per SM x (segment + 4 planes of prologue); ties go to the
            // longer segment
            const int64_t slots = int64_t(2) * nsm, cols = (a.n / G::FX) * (a.n / G::FY);
            int64_t best = -1;
            for (int s = 8; s <= 64 && s <= a.n; s += 2) {
                const int64_t items = cols * ((a.n + s - 1) / s);
                const int64_t cost = ((items + slots - 1) / slots) * (s + 4);
                if (best < 0 || cost <= best) { best = cost; zc = s; }
            }
        }
        zc = (zc + 1) & ~1;                              // whole oct layers
        if (zc < 2) zc = 2;
        if (zc > a.n) zc = int(a.n);
        a.zc = zc;
        a.work = (a.n / G::FX) * (a.n / G::FY) * ((a.n + zc - 1) / zc);
    }
    a.u_old = u_old; a.u_new = u_new; a.dt = dt; a.dt_next = dt_next;
    a.gamma = p->gamma; a.rho_floor = p->rho_floor; a.p_floor = p->p_floor; a.cfl = p->cfl;
    a.status = p->d_status;
    const bool finer = a.finer != 0;
    const size_t bytes = finer ? sizeof(PenSmem<true>) : sizeof(PenSmem<false>);
    auto kern = finer ? k_godunov_pen<RS, true> : k_godunov_pen<RS, false>;
    AMR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    AMR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    kern<<<unsigned(a.work < 1048576 ? a.work : 1048576), G::NT, bytes, st>>>(a);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

}  // namespace amr
