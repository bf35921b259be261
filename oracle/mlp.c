/*
 * Oracle: the learned Riemann surrogate in FP64 (TEST INFRASTRUCTURE ONLY).
 *
 * The paper has no learned component; this is the small network the project puts in
 * place of the iterative exact solver (Toro 2009, Ch. 4).  Architecture:
 * 7 -> 64 -> 64 -> 64 -> 2, SiLU after each hidden layer, linear output.
 * Parameter vector theta (row-major, output index slowest):
 *   W1[64][7] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[2][64] b4[2].
 * Features of a face-normal Riemann problem (L, R, gamma), using the Galilean and
 * scaling invariance of the Euler equations: rho_ref = rho_L, p_ref = max(p_L, p_R),
 * c_ref = sqrt(p_ref / rho_ref), ubar = (u_L + u_R)/2,
 *   x = [ log(rho_L/rho_ref), (u_L-ubar)/c_ref, log(p_L/p_ref),
 *         log(rho_R/rho_ref), (u_R-ubar)/c_ref, log(p_R/p_ref), gamma ];
 * targets y = [ log(pstar / p_ref), (ustar - ubar) / c_ref ].
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define H 64
#define NIN 7
#define NOUT 2
enum { OW1 = 0, OB1 = OW1 + H * NIN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
       OB3 = OW3 + H * H, OW4 = OB3 + H, OB4 = OW4 + NOUT * H, NPAR = OB4 + NOUT };

int64_t or_mlp_nparams(void) { return NPAR; }

void or_mlp_features(const double *WL, const double *WR, double gamma, double *x, double *ref)
{
    double rref = WL[0];
    double pref = WL[4] > WR[4] ? WL[4] : WR[4];
    double cref = sqrt(pref / rref);
    double ubar = 0.5 * (WL[1] + WR[1]);
    x[0] = log(WL[0] / rref);
    x[1] = (WL[1] - ubar) / cref;
    x[2] = log(WL[4] / pref);
    x[3] = log(WR[0] / rref);
    x[4] = (WR[1] - ubar) / cref;
    x[5] = log(WR[4] / pref);
    x[6] = gamma;
    if (ref) { ref[0] = pref; ref[1] = ubar; ref[2] = cref; }
}

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }

/* act (if given) keeps per sample z1,a1,z2,a2,z3,a3 (6*64 values) for the backward pass */
void or_mlp_forward(const double *th, const double *x, int64_t n, double *y, double *act)
{
    for (int64_t s = 0; s < n; s++) {
        double z[3][H], a[3][H];
        const double *in = x + s * NIN;
        for (int j = 0; j < H; j++) {
            double acc = th[OB1 + j];
            for (int i = 0; i < NIN; i++) acc += th[OW1 + j * NIN + i] * in[i];
            z[0][j] = acc; a[0][j] = acc * sigm(acc);
        }
        for (int L = 1; L < 3; L++) {
            int ow = L == 1 ? OW2 : OW3, ob = L == 1 ? OB2 : OB3;
            for (int j = 0; j < H; j++) {
                double acc = th[ob + j];
                for (int i = 0; i < H; i++) acc += th[ow + j * H + i] * a[L - 1][i];
                z[L][j] = acc; a[L][j] = acc * sigm(acc);
            }
        }
        for (int k = 0; k < NOUT; k++) {
            double acc = th[OB4 + k];
            for (int i = 0; i < H; i++) acc += th[OW4 + k * H + i] * a[2][i];
            y[s * NOUT + k] = acc;
        }
        if (act)
            for (int L = 0; L < 3; L++) {
                memcpy(act + s * 6 * H + (2 * L) * H, z[L], sizeof(double) * H);
                memcpy(act + s * 6 * H + (2 * L + 1) * H, a[L], sizeof(double) * H);
            }
    }
}

/* Gradient of sum_s dy[s] . y[s] with respect to theta, accumulated into grad (which the
   caller zeroes).  act must come from or_mlp_forward on the same x. */
void or_mlp_backward(const double *th, const double *x, const double *dy, int64_t n, double *act, double *grad)
{
    for (int64_t s = 0; s < n; s++) {
        const double *in = x + s * NIN;
        const double *z[3], *a[3];
        for (int L = 0; L < 3; L++) { z[L] = act + s * 6 * H + 2 * L * H; a[L] = z[L] + H; }
        double g[H], gz[H];
        for (int k = 0; k < NOUT; k++) {
            grad[OB4 + k] += dy[s * NOUT + k];
            for (int i = 0; i < H; i++) grad[OW4 + k * H + i] += dy[s * NOUT + k] * a[2][i];
        }
        for (int i = 0; i < H; i++) {
            double acc = 0.0;
            for (int k = 0; k < NOUT; k++) acc += th[OW4 + k * H + i] * dy[s * NOUT + k];
            g[i] = acc;
        }
        for (int L = 2; L >= 0; L--) {
            for (int j = 0; j < H; j++) {
                double sg = sigm(z[L][j]);
                gz[j] = g[j] * sg * (1.0 + z[L][j] * (1.0 - sg));     /* SiLU' */
            }
            if (L == 0) {
                for (int j = 0; j < H; j++) {
                    grad[OB1 + j] += gz[j];
                    for (int i = 0; i < NIN; i++) grad[OW1 + j * NIN + i] += gz[j] * in[i];
                }
            } else {
                int ow = L == 1 ? OW2 : OW3, ob = L == 1 ? OB2 : OB3;
                for (int j = 0; j < H; j++) {
                    grad[ob + j] += gz[j];
                    for (int i = 0; i < H; i++) grad[ow + j * H + i] += gz[j] * a[L - 1][i];
                }
                for (int i = 0; i < H; i++) {
                    double acc = 0.0;
                    for (int j = 0; j < H; j++) acc += th[ow + j * H + i] * gz[j];
                    g[i] = acc;
                }
            }
        }
    }
}

/* Adam (Kingma & Ba 2015, Algorithm 1) on a flat parameter vector; t counts from 1 */
void or_adam_step(double *th, double *m, double *v, const double *grad, int64_t n, double lr,
                  double beta1, double beta2, double eps, int64_t t)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        th[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
