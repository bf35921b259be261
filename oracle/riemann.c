/*
 * Oracle: single-state pieces of the Godunov scheme (TEST INFRASTRUCTURE ONLY).
 *
 * The paper gives the hydro solver only as the Table 1 row godunov_fine; the formulas
 * below are the published methods that solver rests on:
 *   conversions and the physical flux: Euler equations, ideal gas, E = p/(g-1) + rho|u|^2/2;
 *   MinMod: Toro 2009, Sec. 13.7 (undivided differences);
 *   HLLC: Toro 2009, Sec. 10.4 (Davis wave-speed estimates, Eq. 10.48);
 *   exact solver: Toro 2009, Ch. 4 (pressure function Eq. 4.5-4.8, Newton iteration
 *   Sec. 4.3.2 from the PVRS guess, sampling Sec. 4.5).
 * State vectors: W = (rho, u, v, w, p) primitive, U = (rho, rho u, rho v, rho w, E);
 * inside a Riemann problem u is the face-normal velocity and v, w the transverse ones.
 */
#include <math.h>
#include "oracle.h"

double or_minmod(double a, double b)
{
    /* zero at an extremum, otherwise the argument of smaller magnitude */
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

double or_mc(double a, double b)
{
    /* monotonized central (van Leer 1977): zero at an extremum, otherwise the central
       difference (a+b)/2 limited to twice either one-sided difference */
    if (a * b <= 0.0) return 0.0;
    double m = fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
    return a > 0.0 ? m : -m;
}

double or_slope(int limiter, double a, double b)
{
    return limiter == OR_LIMITER_MC ? or_mc(a, b) : or_minmod(a, b);
}

void or_cons_to_prim(const double *U, double gamma, double rho_floor, double p_floor, double *W)
{
    double rho = U[0] > rho_floor ? U[0] : rho_floor;
    double u = U[1] / rho, v = U[2] / rho, w = U[3] / rho;
    double ekin = 0.5 * rho * (u * u + v * v + w * w);
    double p = (gamma - 1.0) * (U[4] - ekin);
    W[0] = rho; W[1] = u; W[2] = v; W[3] = w;
    W[4] = p > p_floor ? p : p_floor;
}

void or_prim_to_cons(const double *W, double gamma, double *U)
{
    double rho = W[0];
    U[0] = rho;
    U[1] = rho * W[1];
    U[2] = rho * W[2];
    U[3] = rho * W[3];
    U[4] = W[4] / (gamma - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

void or_flux_normal(const double *W, double gamma, double *F)
{
    /* physical flux through a face whose normal is the u direction */
    double rho = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
    double E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
    F[0] = rho * u;
    F[1] = rho * u * u + p;
    F[2] = rho * u * v;
    F[3] = rho * u * w;
    F[4] = u * (E + p);
}

void or_hllc(const double *WL, const double *WR, double gamma, double *F)
{
    double rL = WL[0], uL = WL[1], pL = WL[4];
    double rR = WR[0], uR = WR[1], pR = WR[4];
    double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
    double SL = fmin(uL - cL, uR - cR);
    double SR = fmax(uL + cL, uR + cR);
    double Sstar = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
                   (rL * (SL - uL) - rR * (SR - uR));
    double FL[5], FR[5], UL[5], UR[5];
    or_flux_normal(WL, gamma, FL);
    or_flux_normal(WR, gamma, FR);
    or_prim_to_cons(WL, gamma, UL);
    or_prim_to_cons(WR, gamma, UR);
    if (SL >= 0.0) {
        for (int v = 0; v < 5; v++) F[v] = FL[v];
    } else if (Sstar >= 0.0) {
        double f = rL * (SL - uL) / (SL - Sstar);
        double Us[5] = { f, f * Sstar, f * WL[2], f * WL[3],
                         f * (UL[4] / rL + (Sstar - uL) * (Sstar + pL / (rL * (SL - uL)))) };
        for (int v = 0; v < 5; v++) F[v] = FL[v] + SL * (Us[v] - UL[v]);
    } else if (SR > 0.0) {
        double f = rR * (SR - uR) / (SR - Sstar);
        double Us[5] = { f, f * Sstar, f * WR[2], f * WR[3],
                         f * (UR[4] / rR + (Sstar - uR) * (Sstar + pR / (rR * (SR - uR)))) };
        for (int v = 0; v < 5; v++) F[v] = FR[v] + SR * (Us[v] - UR[v]);
    } else {
        for (int v = 0; v < 5; v++) F[v] = FR[v];
    }
}

/* Toro Eq. 4.6-4.7: one side's contribution f_K(p) to the pressure function and its
   derivative; shock branch for p > p_K, rarefaction branch otherwise. */
static void side_f(double p, double rK, double pK, double cK, double gamma, double *f, double *df)
{
    if (p > pK) {
        double A = 2.0 / ((gamma + 1.0) * rK);
        double B = (gamma - 1.0) / (gamma + 1.0) * pK;
        double q = sqrt(A / (p + B));
        *f = (p - pK) * q;
        *df = q * (1.0 - 0.5 * (p - pK) / (B + p));
    } else {
        double z = (gamma - 1.0) / (2.0 * gamma);
        *f = 2.0 * cK / (gamma - 1.0) * (pow(p / pK, z) - 1.0);
        *df = 1.0 / (rK * cK) * pow(p / pK, -(gamma + 1.0) / (2.0 * gamma));
    }
}

int or_exact_star(const double *WL, const double *WR, double gamma, double tol, int maxit,
                  double *pstar, double *ustar, int *iters)
{
    double rL = WL[0], uL = WL[1], pL = WL[4];
    double rR = WR[0], uR = WR[1], pR = WR[4];
    double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
    double du = uR - uL;
    if (iters) *iters = 0;
    /* pressure positivity condition, Toro Eq. 4.40: otherwise vacuum is generated */
    if (2.0 * (cL + cR) / (gamma - 1.0) <= du) return OR_ENONPHYSICAL;
    const double eps = 1e-300;
    double p = 0.5 * (pL + pR) - 0.125 * du * (rL + rR) * (cL + cR);   /* PVRS guess */
    if (p < eps) p = eps;
    int it;
    for (it = 1; it <= maxit; it++) {
        double fL, dfL, fR, dfR;
        side_f(p, rL, pL, cL, gamma, &fL, &dfL);
        side_f(p, rR, pR, cR, gamma, &fR, &dfR);
        double pn = p - (fL + fR + du) / (dfL + dfR);
        if (pn < eps) pn = eps;
        double change = 2.0 * fabs(pn - p) / (pn + p);
        p = pn;
        if (change < tol) break;
    }
    if (iters) *iters = it;
    double fL, dfL, fR, dfR;
    side_f(p, rL, pL, cL, gamma, &fL, &dfL);
    side_f(p, rR, pR, cR, gamma, &fR, &dfR);
    *pstar = p;
    *ustar = 0.5 * (uL + uR) + 0.5 * (fR - fL);
    return it > maxit ? OR_ENOCONV : OR_OK;
}

/* Toro Sec. 4.5: the self-similar solution W(x/t = S) given p*, u*.  Transverse
   velocities are carried by the contact: left values if S <= u*, right otherwise. */
int or_exact_sample(const double *WL, const double *WR, double gamma, double ps, double us,
                    double S, double *W)
{
    double g1 = (gamma - 1.0) / (2.0 * gamma), g2 = (gamma + 1.0) / (2.0 * gamma);
    double g3 = 2.0 * gamma / (gamma - 1.0), g4 = 2.0 / (gamma - 1.0);
    double g5 = 2.0 / (gamma + 1.0), g6 = (gamma - 1.0) / (gamma + 1.0);
    double g7 = (gamma - 1.0) / 2.0;
    double rho, u, p;
    const double *T;
    if (S <= us) {
        double rL = WL[0], uL = WL[1], pL = WL[4], cL = sqrt(gamma * pL / rL);
        T = WL;
        if (ps > pL) {                                   /* left shock */
            double SL = uL - cL * sqrt(g2 * ps / pL + g1);
            if (S <= SL) { rho = rL; u = uL; p = pL; }
            else { rho = rL * (ps / pL + g6) / (ps / pL * g6 + 1.0); u = us; p = ps; }
        } else {                                         /* left rarefaction */
            double SHL = uL - cL;
            if (S <= SHL) { rho = rL; u = uL; p = pL; }
            else {
                double cmL = cL * pow(ps / pL, g1);
                double STL = us - cmL;
                if (S > STL) { rho = rL * pow(ps / pL, 1.0 / gamma); u = us; p = ps; }
                else {
                    double c = g5 * (cL + g7 * (uL - S));
                    rho = rL * pow(c / cL, g4);
                    u = g5 * (cL + g7 * uL + S);
                    p = pL * pow(c / cL, g3);
                }
            }
        }
    } else {
        double rR = WR[0], uR = WR[1], pR = WR[4], cR = sqrt(gamma * pR / rR);
        T = WR;
        if (ps > pR) {                                   /* right shock */
            double SR = uR + cR * sqrt(g2 * ps / pR + g1);
            if (S >= SR) { rho = rR; u = uR; p = pR; }
            else { rho = rR * (ps / pR + g6) / (ps / pR * g6 + 1.0); u = us; p = ps; }
        } else {                                         /* right rarefaction */
            double SHR = uR + cR;
            if (S >= SHR) { rho = rR; u = uR; p = pR; }
            else {
                double cmR = cR * pow(ps / pR, g1);
                double STR = us + cmR;
                if (S <= STR) { rho = rR * pow(ps / pR, 1.0 / gamma); u = us; p = ps; }
                else {
                    double c = g5 * (cR - g7 * (uR - S));
                    rho = rR * pow(c / cR, g4);
                    u = g5 * (-cR + g7 * uR + S);
                    p = pR * pow(c / cR, g3);
                }
            }
        }
    }
    W[0] = rho; W[1] = u; W[2] = T[2]; W[3] = T[3]; W[4] = p;
    return OR_OK;
}

/* Godunov flux at a face: the chosen Riemann solver evaluated at x/t = 0.  A vacuum-
   generating or non-converging exact problem falls back to HLLC and reports it. */
int or_riemann_flux(const double *WL, const double *WR, const or_params *p, double *F)
{
    if (p->riemann == OR_EXACT) {
        double ps, us, W0[5];
        int it;
        int st = or_exact_star(WL, WR, p->gamma, 1e-14, 50, &ps, &us, &it);
        if (st == OR_OK) {
            or_exact_sample(WL, WR, p->gamma, ps, us, 0.0, W0);
            or_flux_normal(W0, p->gamma, F);
            return OR_OK;
        }
        or_hllc(WL, WR, p->gamma, F);
        return st;
    }
    or_hllc(WL, WR, p->gamma, F);
    return OR_OK;
}
