// Per-state arithmetic of the MUSCL-Hancock / Godunov scheme (device side), templated
// on the working precision R (double for the FP64 path, float for the FP32 path).
// The scheme: Toro 2009 -- MinMod slopes (Sec. 13.7), MUSCL-Hancock predictor in
// primitive variables (Sec. 14.4), HLLC (Sec. 10.4, Davis wave speeds), exact Riemann
// solver (Ch. 4: pressure function, Newton from the PVRS guess, sampling at x/t = 0).
#pragma once
#include "common.cuh"

namespace amr {

// FP64 <-> FP32 by integer bit manipulation.  On sm_103a the hardware conversions run on
// the FP64 pipe (about 2 per clock per SM), as slow as FP64 arithmetic; these run on the
// integer ALUs.
// d2f: round to nearest on the dropped bits, ties away from zero (the hardware rounds
// ties to even; the two differ only when the 29 dropped bits are exactly 1 followed by
// zeros); |x| below the FP32 normal range (2^-126) gives a signed zero; |x| >= 2^128,
// +-Inf and NaN give a non-finite float of the same sign (+-Inf or a NaN: the magnitude's
// high word is clamped to that of 2^128, so only the low word's bits decide which).
// Finite x below 2^128 that round past FLT_MAX give +-Inf, as in the hardware.
// f2d: exact for normal floats and for +-Inf; NaN stays NaN (payload kept); zero and
// FP32 denormals give a signed zero.
__device__ __forceinline__ float d2f_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
    const unsigned ahi = min(hi & 0x7FFFFFFFu, 0x47F00000u);
    const unsigned long long ab = (static_cast<unsigned long long>(ahi) << 32) | lo;
    // one 64-bit add rebiases the exponent (1023 -> 127) and rounds on the highest dropped
    // bit; bits 29..60 are then the FP32 exponent and mantissa
    unsigned m = unsigned((ab + ((1ull << 28) - (896ull << 52))) >> 29);
    m = ahi < (897u << 20) ? 0u : m;
    return __uint_as_float(m | (hi & 0x80000000u));
}

__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = __float_as_uint(f), ab = b & 0x7FFFFFFFu;
    const bool z = ab < 0x00800000u;
    // exponent 255 (Inf, NaN) moves to 2047: one more rebias of 896
    const unsigned bias = ab >= 0x7F800000u ? (1792u << 20) : (896u << 20);
    const unsigned hi = z ? 0u : (ab >> 3) + bias;
    const unsigned lo = z ? 0u : ab << 29;
    return __hiloint2double(int(hi | (b & 0x80000000u)), int(lo));
}

// whether the five values of an FP64 state are finite in the working precision R: for
// FP64 by the exponent fields of the high words (integer operations, off the FP64 pipe);
// for FP32 by the sum of the converted values (non-finite when any of them is, or when
// the state lies beyond FP32's range)
template <typename R> __device__ __forceinline__ bool state_finite(const double U[5]);
template <> __device__ __forceinline__ bool state_finite<double>(const double U[5])
{
    unsigned e = 0;
#pragma unroll
    for (int v = 0; v < 5; ++v) e = max(e, unsigned(__double2hiint(U[v])) & 0x7FF00000u);
    return e < 0x7FF00000u;
}
template <> __device__ __forceinline__ bool state_finite<float>(const double U[5])
{
    const float s = (d2f_bits(U[0]) + d2f_bits(U[1])) + (d2f_bits(U[2]) + d2f_bits(U[3])) + d2f_bits(U[4]);
    return fabsf(s) <= 3.402823466e38f;
}

// working-precision view of an FP64 state value, and back
template <typename R> __device__ __forceinline__ R to_work(double x);
template <> __device__ __forceinline__ double to_work<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_work<float>(double x) { return d2f_bits(x); }
__device__ __forceinline__ double to_state(double x) { return x; }
__device__ __forceinline__ double to_state(float x) { return f2d_bits(x); }

// Products and multiply-adds written out.  Left to itself the compiler fuses a*b + c*d
// into either fma(a, b, c*d) or fma(c, d, a*b), and the choice can differ between kernels
// that inline the same code; these pin one rounding sequence, so that every kernel that
// uses the functions below computes the same bits.  mulr is a multiplication the compiler
// never fuses; fmar a fused multiply-add.
__device__ __forceinline__ float mulr(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulr(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

// u^2 + v^2 + w^2, accumulated left to right
template <typename R> __device__ __forceinline__ R sq3(R u, R v, R w) { return fmar(w, w, fmar(v, v, mulr(u, u))); }

template <typename R> struct Prm {
    R gamma, rho_floor, p_floor;
    int limiter = AMR_LIMITER_MINMOD;   // slopes of the reconstruction
};

// MinMod: zero when the differences disagree in sign (or one is zero), else the one of
// smaller magnitude.  Written as the median of (0, a, b), four min/max operations: for
// finite a, b the same value as the textbook branch (a zero result may carry either sign)
template <typename R> __device__ __forceinline__ R minmod(R a, R b)
{
    return fmax(fmin(a, b), fmin(fmax(a, b), R(0)));
}

template <typename R> __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }

// Monotonized central limiter (van Leer 1977): zero when the differences disagree in
// sign, else the central difference (a+b)/2 limited to twice either difference
template <typename R> __device__ __forceinline__ R mc_limit(R a, R b)
{
    const R m = fmin(fmin(R(2) * fabs(a), R(2) * fabs(b)), R(0.5) * fabs(a + b));
    return a * b > R(0) ? copysign(m, a) : R(0);
}

// slope of the reconstruction from the two one-sided differences
template <typename R> __device__ __forceinline__ R slope(const Prm<R> &p, R a, R b)
{
    return p.limiter == AMR_LIMITER_MC ? mc_limit(a, b) : minmod(a, b);
}

// cons -> prim from conserved values already in the working precision
template <typename R>
__device__ __forceinline__ void cons_to_prim_w(const R U[NV], const Prm<R> &p, R W[NV])
{
    const R rho = rmax(U[0], p.rho_floor), irho = R(1) / rho;
    const R u = mulr(U[1], irho), v = mulr(U[2], irho), w = mulr(U[3], irho);
    const R ek = mulr(mulr(R(0.5), rho), sq3(u, v, w));
    const R pr = mulr(p.gamma - R(1), U[4] - ek);
    W[0] = rho; W[1] = u; W[2] = v; W[3] = w;
    W[4] = rmax(pr, p.p_floor);
}

// conserved (FP64 storage) -> primitive in precision R, floors applied
template <typename R>
__device__ __forceinline__ void cons_to_prim(const double U[NV], const Prm<R> &p, R W[NV])
{
    R Uw[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Uw[v] = to_work<R>(U[v]);
    cons_to_prim_w(Uw, p, W);
}

// physical flux through a face whose normal is the first velocity component
template <typename R>
__device__ __forceinline__ void flux_normal(const R W[NV], R g, R F[NV], R U[NV])
{
    const R rho = W[0], u = W[1], v = W[2], w = W[3], pr = W[4];
    const R E = fmar(mulr(R(0.5), rho), sq3(u, v, w), pr / (g - R(1)));
    const R ru = mulr(rho, u);
    F[0] = ru;
    F[1] = fmar(ru, u, pr);
    F[2] = mulr(ru, v);
    F[3] = mulr(ru, w);
    F[4] = mulr(u, E + pr);
    U[0] = rho; U[1] = ru; U[2] = mulr(rho, v); U[3] = mulr(rho, w); U[4] = E;
}

// HLLC flux (Toro, Spruce & Speares 1994); the side used is chosen before computing,
// so every face does one star state (no divergent branches, no register-array pointers).
template <typename R>
__device__ __forceinline__ void hllc(const R WL[NV], const R WR[NV], R g, R F[NV])
{
    const R rL = WL[0], uL = WL[1], pL = WL[4];
    const R rR = WR[0], uR = WR[1], pR = WR[4];
    const R cL = sqrt(mulr(g, pL) / rL), cR = sqrt(mulr(g, pR) / rR);
    const R SL = fmin(uL - cL, uR - cR);
    const R SR = fmax(uL + cL, uR + cR);
    const R mL = mulr(rL, SL - uL), mR = mulr(rR, SR - uR);   // mass fluxes through the outer waves
    const R Ss = fmar(-uR, mR, fmar(uL, mL, pR - pL)) / (mL - mR);
    const bool left = (SL >= R(0)) || (Ss >= R(0));
    const bool star = !(SL >= R(0)) && (Ss >= R(0) || SR > R(0));
    R WK[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) WK[v] = left ? WL[v] : WR[v];
    const R SK = left ? SL : SR;
    R FK[NV], UK[NV];
    flux_normal(WK, g, FK, UK);
    if (star) {
        // U*_K = f [1, S*, v_K, w_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))],
        // f = rho_K (S_K - u_K) / (S_K - S*); with d = 1/(S_K - S*) the energy component is
        // d ((S_K - u_K) E_K + (S* - u_K) p_K) + f (S* - u_K) S*, one division in all
        const R rK = WK[0], uK = WK[1], pK = WK[4];
        const R d = R(1) / (SK - Ss);
        const R f = mulr(mulr(rK, SK - uK), d);
        const R Us[NV] = {f, mulr(f, Ss), mulr(f, WK[2]), mulr(f, WK[3]),
                          fmar(mulr(f, Ss - uK), Ss, mulr(d, fmar(Ss - uK, pK, mulr(SK - uK, UK[4]))))};
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = fmar(SK, Us[v] - UK[v], FK[v]);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FK[v];
    }
}

// Toro Eq. 4.6-4.7: one side's contribution to the pressure function and derivative
template <typename R>
__device__ __forceinline__ void side_f(R p, R rK, R pK, R cK, R g, R &f, R &df)
{
    if (p > pK) {
        const R A = R(2) / ((g + R(1)) * rK);
        const R B = (g - R(1)) / (g + R(1)) * pK;
        const R q = sqrt(A / (p + B));
        f = (p - pK) * q;
        df = q * (R(1) - R(0.5) * (p - pK) / (B + p));
    } else {
        const R z = (g - R(1)) / (R(2) * g);
        f = R(2) * cK / (g - R(1)) * (pow(p / pK, z) - R(1));
        df = R(1) / (rK * cK) * pow(p / pK, -(g + R(1)) / (R(2) * g));
    }
}

// Exact Riemann problem (Toro Ch. 4).  Returns 0, AMR_ENONPHYSICAL (vacuum) or
// AMR_ENOCONV; on failure the caller uses HLLC.  Newton starts from p0 when p0 > 0 (a
// learned prediction), else from the linearised (PVRS) guess; *iters receives the
// iterations made.
template <typename R>
__device__ int exact_star(const R WL[NV], const R WR[NV], R g, R tol, int maxit, R &ps, R &us, R p0 = R(-1),
                          int *iters = nullptr)
{
    if (iters) *iters = 0;
    const R rL = WL[0], uL = WL[1], pL = WL[4];
    const R rR = WR[0], uR = WR[1], pR = WR[4];
    const R cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    const R du = uR - uL;
    if (R(2) * (cL + cR) / (g - R(1)) <= du) return AMR_ENONPHYSICAL;
    const R eps = sizeof(R) == 8 ? R(1e-300) : R(1e-37);
    R p = p0 > R(0) ? p0 : mulr(R(0.5), pL + pR) - mulr(mulr(mulr(R(0.125), du), rL + rR), cL + cR);
    if (p < eps) p = eps;
    int it;
    for (it = 1; it <= maxit; ++it) {
        R fL, dfL, fR, dfR;
        side_f(p, rL, pL, cL, g, fL, dfL);
        side_f(p, rR, pR, cR, g, fR, dfR);
        R pn = p - (fL + fR + du) / (dfL + dfR);
        if (pn < eps) pn = eps;
        const R change = R(2) * fabs(pn - p) / (pn + p);
        p = pn;
        if (change < tol) break;
    }
    R fL, dfL, fR, dfR;
    side_f(p, rL, pL, cL, g, fL, dfL);
    side_f(p, rR, pR, cR, g, fR, dfR);
    ps = p;
    us = mulr(R(0.5), uL + uR) + mulr(R(0.5), fR - fL);
    if (iters) *iters = it > maxit ? maxit : it;
    return it > maxit ? AMR_ENOCONV : 0;
}

// Sampling at x/t = 0 (Toro Sec. 4.5); transverse velocities from the side of the
// contact the face lies on (left when u* >= 0).
template <typename R>
__device__ void exact_sample0(const R WL[NV], const R WR[NV], R g, R ps, R us, R W[NV])
{
    const R g1 = (g - R(1)) / (R(2) * g), g2 = (g + R(1)) / (R(2) * g);
    const R g3 = R(2) * g / (g - R(1)), g4 = R(2) / (g - R(1));
    const R g5 = R(2) / (g + R(1)), g6 = (g - R(1)) / (g + R(1)), g7 = (g - R(1)) / R(2);
    const R S = R(0);
    R rho, u, p;
    const bool lside = S <= us;
    if (lside) {
        const R rL = WL[0], uL = WL[1], pL = WL[4], cL = sqrt(g * pL / rL);
        if (ps > pL) {
            const R SL = uL - cL * sqrt(g2 * ps / pL + g1);
            if (S <= SL) { rho = rL; u = uL; p = pL; }
            else { rho = rL * (ps / pL + g6) / (ps / pL * g6 + R(1)); u = us; p = ps; }
        } else {
            const R SHL = uL - cL;
            if (S <= SHL) { rho = rL; u = uL; p = pL; }
            else {
                const R cmL = cL * pow(ps / pL, g1);
                const R STL = us - cmL;
                if (S > STL) { rho = rL * pow(ps / pL, R(1) / g); u = us; p = ps; }
                else {
                    const R c = g5 * (cL + g7 * (uL - S));
                    rho = rL * pow(c / cL, g4);
                    u = g5 * (cL + g7 * uL + S);
                    p = pL * pow(c / cL, g3);
                }
            }
        }
    } else {
        const R rR = WR[0], uR = WR[1], pR = WR[4], cR = sqrt(g * pR / rR);
        if (ps > pR) {
            const R SR = uR + cR * sqrt(g2 * ps / pR + g1);
            if (S >= SR) { rho = rR; u = uR; p = pR; }
            else { rho = rR * (ps / pR + g6) / (ps / pR * g6 + R(1)); u = us; p = ps; }
        } else {
            const R SHR = uR + cR;
            if (S >= SHR) { rho = rR; u = uR; p = pR; }
            else {
                const R cmR = cR * pow(ps / pR, g1);
                const R STR = us + cmR;
                if (S <= STR) { rho = rR * pow(ps / pR, R(1) / g); u = us; p = ps; }
                else {
                    const R c = g5 * (cR - g7 * (uR - S));
                    rho = rR * pow(c / cR, g4);
                    u = g5 * (-cR + g7 * uR + S);
                    p = pR * pow(c / cR, g3);
                }
            }
        }
    }
    W[0] = rho; W[1] = u; W[2] = lside ? WL[2] : WR[2]; W[3] = lside ? WL[3] : WR[3]; W[4] = p;
}

// MUSCL-Hancock half step in primitive variables (Toro Sec. 14.4) of a cell from its
// primitives Wc and undivided slopes Dl[d] (hl = dt / (2 dx)); every term's products
// accumulated left to right
template <typename R>
__device__ __forceinline__ void muscl_predict(const R Wc[NV], const R Dl[3][NV], R hl, R gamma, R Wt[NV])
{
    const R rr = Wc[0], u = Wc[1], vv = Wc[2], w = Wc[3], pp = Wc[4];
    R s = fmar(rr, Dl[2][3], fmar(w, Dl[2][0], fmar(rr, Dl[1][2], fmar(vv, Dl[1][0], fmar(rr, Dl[0][1],
                                                                                        mulr(u, Dl[0][0]))))));
    Wt[0] = fmar(-hl, s, rr);
    const R ir = R(1) / rr;
    s = fmar(Dl[0][4], ir, fmar(w, Dl[2][1], fmar(vv, Dl[1][1], mulr(u, Dl[0][1]))));
    Wt[1] = fmar(-hl, s, u);
    s = fmar(Dl[1][4], ir, fmar(w, Dl[2][2], fmar(vv, Dl[1][2], mulr(u, Dl[0][2]))));
    Wt[2] = fmar(-hl, s, vv);
    s = fmar(Dl[2][4], ir, fmar(w, Dl[2][3], fmar(vv, Dl[1][3], mulr(u, Dl[0][3]))));
    Wt[3] = fmar(-hl, s, w);
    s = fmar(mulr(gamma, pp), (Dl[0][1] + Dl[1][2]) + Dl[2][3], fmar(w, Dl[2][4], fmar(vv, Dl[1][4],
                                                                                      mulr(u, Dl[0][4]))));
    Wt[4] = fmar(-hl, s, pp);
}

// face state of a predicted cell, W~ + half Delta_D (half = +1/2: the cell is the face's
// left state; -1/2: its right state), in the face-normal frame of direction D (density,
// normal velocity, the two transverse velocities in axis order, pressure), density and
// pressure floored
template <int D, typename R>
__device__ __forceinline__ void face_state(const R Wt[NV], const R DlD[NV], R half, const Prm<R> &pr, R S[NV])
{
    constexpr int N0 = D + 1, T1 = D == 0 ? 2 : 1, T2 = D == 2 ? 2 : 3;
    S[0] = rmax(fmar(half, DlD[0], Wt[0]), pr.rho_floor);
    S[1] = fmar(half, DlD[N0], Wt[N0]);
    S[2] = fmar(half, DlD[T1], Wt[T1]);
    S[3] = fmar(half, DlD[T2], Wt[T2]);
    S[4] = rmax(fmar(half, DlD[4], Wt[4]), pr.p_floor);
}

// dt candidate of one cell: cfl * dx / sum_d (|u_d| + c), from the FP64 state; p, cfl and
// dx already in the working precision
template <typename R>
__device__ __forceinline__ double cfl_candidate(const double U[NV], const Prm<R> &p, R cfl, R dx)
{
    R W[NV];
    cons_to_prim(U, p, W);
    const R cs = sqrt(p.gamma * W[4] / W[0]);
    const R sig = (fabs(W[1]) + cs) + (fabs(W[2]) + cs) + (fabs(W[3]) + cs);
    if (sizeof(R) == 8) return double(cfl) * (double(dx) / double(sig));
    // FP32: scaled down by (1 - 2^-16) so that it never exceeds the FP64 value
    return to_state(float(cfl) * (float(dx) / float(sig)) * 0.9999847412109375f);
}

}  // namespace amr
