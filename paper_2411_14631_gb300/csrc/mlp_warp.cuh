// Warp-level evaluation of the learned Riemann surrogate on the tensor cores.
//
// Network (7 -> 64 -> 64 -> 64 -> 2, SiLU on the hidden layers, linear output), the
// replacement the project makes for the iterative exact Riemann solver (Toro 2009,
// Ch. 4).  BF16 weights and activations, FP32 accumulation: mma.sync m16n8k16, 16
// samples per warp per pass; each layer's FP32 accumulator fragments become the next
// layer's A fragments in registers (the accumulator of an m16n8 tile pair has the
// element layout of an m16k16 A tile).
//
// Packed parameter block (device memory, see mlp_pack):
//   W1 [64][S1] bf16 (in 7 padded to 16), W2, W3 [64][S] bf16, W4 [8][S] bf16 (out 2
//   padded to 8), and the transposes W2T, W3T [64][S], W4T [64][S4T] used by the
//   backward pass; biases b1, b2, b3 [64], b4 [8] as FP32.  Row strides are padded so
//   that the eight rows a fragment load touches fall in distinct shared-memory banks.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace amr {
namespace mlp {

constexpr int H = 64, NIN = 7, NOUT = 2;
constexpr int NPARAM = H * NIN + H + 2 * (H * H + H) + NOUT * H + NOUT;   // 8962
// flat FP32 parameter offsets (same order as the oracle's theta)
constexpr int OW1 = 0, OB1 = OW1 + H * NIN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + NOUT * H;
// packed layout (element offsets in bf16 units for the matrices)
constexpr int S1 = 24;     // W1 row stride (16 used)
constexpr int S = 72;      // 64-wide rows
constexpr int S4T = 24;    // W4T row stride (8 used)
constexpr int PW1 = 0, PW2 = PW1 + H * S1, PW3 = PW2 + H * S, PW4 = PW3 + H * S, PW2T = PW4 + 8 * S,
              PW3T = PW2T + H * S, PW4T = PW3T + H * S, PEND = PW4T + H * S4T;
constexpr int PBIAS_BYTES = (3 * H + 8) * 4;
constexpr size_t PACKED_BYTES = size_t(PEND) * 2 + PBIAS_BYTES;   // biases follow the matrices

struct Packed {
    const __nv_bfloat16 *w;    // matrices
    const float *b;            // b1 | b2 | b3 | b4(8)
};

__host__ __device__ inline Packed view(const void *p)
{
    Packed q;
    q.w = static_cast<const __nv_bfloat16 *>(p);
    q.b = reinterpret_cast<const float *>(static_cast<const char *>(p) + size_t(PEND) * 2);
    return q;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

// D += A(16x16, row) * B(16x8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU(z) = z sigma(z) = (z/2) (1 + tanh(z/2)): one hardware tanh per value.  The hidden
// activations are computed on BF16 pairs (they are BF16 A fragments of the next layer
// anyway); the backward pass uses the FP32 derivative sigma (1 + z (1 - sigma)).
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu(float z) { return 0.5f * z * (1.0f + tanh_approx(0.5f * z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 0.5f + 0.5f * tanh_approx(0.5f * z);
    return s * (1.0f + z * (1.0f - s));
}
// two SiLUs on a BF16 pair: h = z/2, silu = h + h tanh(h)
__device__ __forceinline__ uint32_t silu_bf16x2(float z0, float z1)
{
    const uint32_t h = pack_bf16(0.5f * z0, 0.5f * z1);
    uint32_t t, r;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(h), "r"(t));
    return r;
}

// B fragment of a row-major [N][stride] weight block for n-tile nt, k-tile kt
__device__ __forceinline__ void bfrag(const __nv_bfloat16 *W, int stride, int nt, int kt, int lane, uint32_t &b0,
                                      uint32_t &b1)
{
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *row = W + (nt * 8 + g) * stride + kt * 16 + 2 * t;
    b0 = ld32(row);
    b1 = ld32(row + 8);
}

// accumulator n-tiles (2kt, 2kt+1) -> A fragment k-tile kt through SiLU on BF16 pairs
__device__ __forceinline__ void acc_to_a_silu(const float acc[8][4], uint32_t a[4][4])
{
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        a[kt][0] = silu_bf16x2(acc[2 * kt][0], acc[2 * kt][1]);
        a[kt][1] = silu_bf16x2(acc[2 * kt][2], acc[2 * kt][3]);
        a[kt][2] = silu_bf16x2(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
        a[kt][3] = silu_bf16x2(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
    }
}

// accumulator n-tiles (2kt, 2kt+1) -> A fragment k-tile kt, with an elementwise map
template <typename F>
__device__ __forceinline__ void acc_to_a(const float acc[8][4], uint32_t a[4][4], F f)
{
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        a[kt][0] = pack_bf16(f(acc[2 * kt][0]), f(acc[2 * kt][1]));
        a[kt][1] = pack_bf16(f(acc[2 * kt][2]), f(acc[2 * kt][3]));
        a[kt][2] = pack_bf16(f(acc[2 * kt + 1][0]), f(acc[2 * kt + 1][1]));
        a[kt][3] = pack_bf16(f(acc[2 * kt + 1][2]), f(acc[2 * kt + 1][3]));
    }
}

__device__ __forceinline__ void bias_init(float acc[8][4], const float *b, int lane)
{
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        acc[nt][0] = b[nt * 8 + 2 * t];
        acc[nt][1] = b[nt * 8 + 2 * t + 1];
        acc[nt][2] = acc[nt][0];
        acc[nt][3] = acc[nt][1];
    }
}

// hidden layer: acc = b + A * W^T over K = 64 (4 k-tiles), 8 n-tiles
__device__ __forceinline__ void hidden64(const uint32_t a[4][4], const __nv_bfloat16 *W, const float *b,
                                         float acc[8][4], int lane)
{
    bias_init(acc, b, lane);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            uint32_t b0, b1;
            bfrag(W, S, nt, kt, lane, b0, b1);
            mma16816(acc[nt], a[kt], b0, b1);
        }
}

// A fragment of the 16 x 16 input block (7 features, zero padded); x16 points at row 0
// of 16 consecutive samples of 8 floats each (feature 7 unused)
__device__ __forceinline__ void input_frag(const float *x16, int lane, uint32_t a[4])
{
    const int g = lane >> 2, t = lane & 3;
    const float *r0 = x16 + g * 8, *r1 = x16 + (g + 8) * 8;
    const int c0 = 2 * t, c1 = 2 * t + 1;
    const float x00 = r0[c0], x01 = c1 < NIN ? r0[c1] : 0.0f;
    const float x10 = r1[c0], x11 = c1 < NIN ? r1[c1] : 0.0f;
    a[0] = pack_bf16(x00, x01);
    a[1] = pack_bf16(x10, x11);
    a[2] = 0u;
    a[3] = 0u;
}

// Forward pass of 16 samples.  Output: lanes with t == 0 hold y[g] (y0[0], y0[1]) and
// y[g+8] (y1[0], y1[1]).  If z is given, the pre-activations of the three hidden layers
// are kept (accumulator layout) for a backward pass.
__device__ __forceinline__ void forward16(const Packed &P, const float *x16, int lane, float out[4],
                                          float (*z)[8][4] = nullptr)
{
    uint32_t a0[4];
    input_frag(x16, lane, a0);
    float acc[8][4];
    bias_init(acc, P.b, lane);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        bfrag(P.w + PW1, S1, nt, 0, lane, b0, b1);
        mma16816(acc[nt], a0, b0, b1);
    }
    uint32_t a[4][4];
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
        if (z) {
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) z[layer][nt][i] = acc[nt][i];
        }
        acc_to_a_silu(acc, a);
        hidden64(a, P.w + (layer == 0 ? PW2 : PW3), P.b + H * (layer + 1), acc, lane);
    }
    if (z) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) z[2][nt][i] = acc[nt][i];
    }
    acc_to_a_silu(acc, a);
    const int t = lane & 3;
    float o[4] = {P.b[3 * H + 2 * t], P.b[3 * H + 2 * t + 1], P.b[3 * H + 2 * t], P.b[3 * H + 2 * t + 1]};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        uint32_t b0, b1;
        bfrag(P.w + PW4, S, 0, kt, lane, b0, b1);
        mma16816(o, a[kt], b0, b1);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = o[i];
}

// ---- features of a face-normal Riemann problem (Galilean + scaling invariance) ------
// rho_ref = rho_L, p_ref = max(p_L, p_R), c_ref = sqrt(p_ref/rho_ref), ubar = (u_L+u_R)/2;
// x = [log(rho_L/rho_ref), (u_L-ubar)/c_ref, log(p_L/p_ref), log(rho_R/rho_ref),
//      (u_R-ubar)/c_ref, log(p_R/p_ref), gamma],  y = [log(p*/p_ref), (u*-ubar)/c_ref]
template <typename R>
__device__ __forceinline__ void features(R rL, R uL, R pL, R rR, R uR, R pR, R g, R x[7], R &pref, R &ubar, R &cref)
{
    const R rref = rL;
    pref = pL > pR ? pL : pR;
    cref = sqrt(pref / rref);
    ubar = R(0.5) * (uL + uR);
    x[0] = log(rL / rref);
    x[1] = (uL - ubar) / cref;
    x[2] = log(pL / pref);
    x[3] = log(rR / rref);
    x[4] = (uR - ubar) / cref;
    x[5] = log(pR / pref);
    x[6] = g;
}

}  // namespace mlp
}  // namespace amr
