// Learned Riemann surrogate: dataset labelling with the exact FP64 solver, BF16 tensor-core
// inference, and training (forward, backward, weight gradients on the tensor cores, Adam).
// The paper has no learned component; the network replaces the iterative exact solver
// (Toro 2009, Ch. 4) inside the Godunov update and is checked by a residual test.
#include <cstring>
#include "hydro_math.cuh"
#include "mlp_warp.cuh"

namespace amr {
using namespace mlp;

// states [n][6] = (rho_L, u_L, p_L, rho_R, u_R, p_R) in FP64 -> features x [n][8] (slot 7
// unused) and targets y [n][2] from the exact FP64 solution
__global__ void k_make_dataset(const double *__restrict__ st, int64_t n, double gamma, float *x, float *y,
                               int32_t *status)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const double *s = st + 6 * i;
    double WL[NV] = {s[0], s[1], 0.0, 0.0, s[2]}, WR[NV] = {s[3], s[4], 0.0, 0.0, s[5]};
    double xf[7], pref, ubar, cref;
    mlp::features(s[0], s[1], s[2], s[3], s[4], s[5], gamma, xf, pref, ubar, cref);
    double ps, us;
    const int e = exact_star(WL, WR, gamma, 1e-14, 50, ps, us);
    if (e != 0) {
        set_error(status, e);
        ps = pref; us = ubar;      // marked by the status word; the caller drops the set
    }
    for (int k = 0; k < 7; ++k) x[8 * i + k] = float(xf[k]);
    x[8 * i + 7] = 0.0f;
    y[2 * i] = float(log(ps / pref));
    y[2 * i + 1] = float((us - ubar) / cref);
}

// FP32 master parameters -> packed BF16 matrices (+ transposes) and FP32 biases
__global__ void k_pack(const float *__restrict__ th, __nv_bfloat16 *w, float *b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < PEND) {
        float v = 0.0f;
        if (i < PW2) {                                   // W1 [64][S1], in 7
            const int n = i / S1, k = i % S1;
            v = k < NIN ? th[OW1 + n * NIN + k] : 0.0f;
        } else if (i < PW3) {
            const int j = i - PW2, n = j / S, k = j % S;
            v = k < H ? th[OW2 + n * H + k] : 0.0f;
        } else if (i < PW4) {
            const int j = i - PW3, n = j / S, k = j % S;
            v = k < H ? th[OW3 + n * H + k] : 0.0f;
        } else if (i < PW2T) {                           // W4 [8][S], out 2
            const int j = i - PW4, n = j / S, k = j % S;
            v = (n < NOUT && k < H) ? th[OW4 + n * H + k] : 0.0f;
        } else if (i < PW3T) {                           // W2T[k][n] = W2[n][k]
            const int j = i - PW2T, k = j / S, n = j % S;
            v = n < H ? th[OW2 + n * H + k] : 0.0f;
        } else if (i < PW4T) {
            const int j = i - PW3T, k = j / S, n = j % S;
            v = n < H ? th[OW3 + n * H + k] : 0.0f;
        } else {                                         // W4T [64][S4T]
            const int j = i - PW4T, k = j / S4T, n = j % S4T;
            v = n < NOUT ? th[OW4 + n * H + k] : 0.0f;
        }
        w[i] = __float2bfloat16_rn(v);
    } else if (i < PEND + 3 * H + 8) {
        const int j = i - PEND;
        float v;
        if (j < H) v = th[OB1 + j];
        else if (j < 2 * H) v = th[OB2 + j - H];
        else if (j < 3 * H) v = th[OB3 + j - 2 * H];
        else v = (j - 3 * H) < NOUT ? th[OB4 + j - 3 * H] : 0.0f;
        b[j] = v;
    }
}

// inference: x [n][8] -> y [n][2]; one warp per 16 samples
__global__ void __launch_bounds__(256) k_forward(const void *packed, const float *__restrict__ x, float *y, int64_t n)
{
    const Packed P = view(packed);
    __shared__ float sx[8][16 * 8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nwarp = int64_t(gridDim.x) * 8;
    for (int64_t base = (blockIdx.x * 8 + w) * int64_t(16); base < n; base += nwarp * 16) {
        for (int j = lane; j < 16 * 8; j += 32) {
            const int64_t s = base + j / 8;
            sx[w][j] = s < n ? x[s * 8 + (j & 7)] : 0.0f;
        }
        __syncwarp();
        float o[4];
        forward16(P, sx[w], lane, o);
        const int g = lane >> 2, t = lane & 3;
        if (t == 0) {
            if (base + g < n) { y[2 * (base + g)] = o[0]; y[2 * (base + g) + 1] = o[1]; }
            if (base + g + 8 < n) { y[2 * (base + g + 8)] = o[2]; y[2 * (base + g + 8) + 1] = o[3]; }
        }
        __syncwarp();
    }
}

// ---- training: gradients of the loss over a batch --------------------------------------
// Each CTA (8 warps) takes chunks of 128 samples.  Per warp: forward of 16 samples keeping
// the pre-activations, backward through the layers in registers (dz -> dz W with the
// transposed weights).  Weight gradients dW = dz^T a are tensor-core products over the
// 128 samples of the chunk, staged transposed in shared memory; a constant-1 row in a^T
// gives the bias gradient.  Accumulators stay in registers across chunks; each CTA writes
// its partial gradient, and k_grad_reduce sums the partials in a fixed order.
constexpr int TB = 128;        // samples per chunk
constexpr int TS = TB + 8;     // staged row stride (bf16)
struct TrainSmem {
    __nv_bfloat16 dzT[H][TS];   // dz^T of the current layer (rows = outputs)
    __nv_bfloat16 aT[72][TS];   // a^T of the layer input (rows = inputs, then the ones row)
    float sx[8][16 * 8];
    float sy[8][16 * 2];
    float loss[8];
};

// tiles of dW for layer L: (m-tiles of outputs) x (n-tiles of inputs + ones row)
template <int L> struct Lay;
template <> struct Lay<1> { static constexpr int MT = 4, NT = 2, K = NIN, OW = OW1, OB = OB1, NOUTS = H; };
template <> struct Lay<2> { static constexpr int MT = 4, NT = 9, K = H, OW = OW2, OB = OB2, NOUTS = H; };
template <> struct Lay<3> { static constexpr int MT = 4, NT = 9, K = H, OW = OW3, OB = OB3, NOUTS = H; };
template <> struct Lay<4> { static constexpr int MT = 1, NT = 9, K = H, OW = OW4, OB = OB4, NOUTS = NOUT; };
template <int L> __host__ __device__ constexpr int slots() { return (Lay<L>::MT * Lay<L>::NT + 7) / 8; }

template <int L>
__device__ __forceinline__ void grad_gemm(const TrainSmem &sm, float acc[][4], int w, int lane)
{
    using Y = Lay<L>;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int sl = 0; sl < slots<L>(); ++sl) {
        const int j = w + 8 * sl;
        if (j >= Y::MT * Y::NT) break;
        const int mt = j / Y::NT, nt = j % Y::NT;
#pragma unroll
        for (int kt = 0; kt < TB / 16; ++kt) {
            uint32_t a[4];
            const __nv_bfloat16 *A0 = &sm.dzT[mt * 16 + g][kt * 16 + 2 * t];
            const __nv_bfloat16 *A1 = &sm.dzT[mt * 16 + g + 8][kt * 16 + 2 * t];
            a[0] = ld32(A0); a[1] = ld32(A1); a[2] = ld32(A0 + 8); a[3] = ld32(A1 + 8);
            const __nv_bfloat16 *B = &sm.aT[nt * 8 + g][kt * 16 + 2 * t];
            mma16816(acc[sl], a, ld32(B), ld32(B + 8));
        }
    }
}

// write a warp's dW tiles of layer L into a flat FP32 gradient vector
template <int L>
__device__ __forceinline__ void grad_store(const float acc[][4], float *out, int w, int lane)
{
    using Y = Lay<L>;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int sl = 0; sl < slots<L>(); ++sl) {
        const int j = w + 8 * sl;
        if (j >= Y::MT * Y::NT) break;
        const int mt = j / Y::NT, nt = j % Y::NT;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = mt * 16 + g + (i >= 2 ? 8 : 0);
            const int k = nt * 8 + 2 * t + (i & 1);
            if (n >= Y::NOUTS) continue;
            // layer 1: inputs 0..6, ones row at 7; other layers: inputs 0..63, ones row at 64
            const int kones = (L == 1) ? NIN : H;
            if (k < Y::K) out[Y::OW + n * Y::K + k] = acc[sl][i];
            else if (k == kones) out[Y::OB + n] = acc[sl][i];
        }
    }
}

// stage the BF16 SiLU activations (as the forward pass computes them) transposed
__device__ __forceinline__ void stage_T_silu(__nv_bfloat16 (*dst)[TS], const float v[8][4], int w, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t p = silu_bf16x2(v[nt][2 * h], v[nt][2 * h + 1]);
            const int row = 16 * w + g + (h ? 8 : 0);
            const int col = nt * 8 + 2 * t;
            dst[col][row] = *reinterpret_cast<const __nv_bfloat16 *>(&p);
            dst[col + 1][row] = *(reinterpret_cast<const __nv_bfloat16 *>(&p) + 1);
        }
}

// stage an accumulator-layout [16 samples][64] block of warp w as bf16 transposed rows
template <typename F>
__device__ __forceinline__ void stage_T(__nv_bfloat16 (*dst)[TS], const float v[8][4], int w, int lane, F f)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int col = nt * 8 + 2 * t + (i & 1), row = 16 * w + g + (i >= 2 ? 8 : 0);
            dst[col][row] = __float2bfloat16_rn(f(v[nt][i]));
        }
}

// mode 0: loss = sum over samples and outputs of (y - target)^2 / n, dy = 2 (y - t) / n
// mode 1: dy given (gradient of sum dy . y)
__global__ void __launch_bounds__(256, 1) k_train_grad(const void *packed, const float *__restrict__ x,
                                                       const float *__restrict__ tgt, int64_t n, int mode,
                                                       float *partial, float *loss_partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smraw);
    const Packed P = view(packed);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    // constant rows of a^T: the ones row (64 for layers 2-4; 7 for layer 1 is set per chunk)
    for (int j = threadIdx.x; j < 8 * TS; j += blockDim.x) sm.aT[64 + j / TS][j % TS] = __float2bfloat16_rn(j / TS == 0 ? 1.0f : 0.0f);
    float g1[slots<1>()][4], g2[slots<2>()][4], g3[slots<3>()][4], g4[slots<4>()][4];
    for (int s = 0; s < slots<1>(); ++s) for (int i = 0; i < 4; ++i) g1[s][i] = 0.0f;
    for (int s = 0; s < slots<2>(); ++s) for (int i = 0; i < 4; ++i) g2[s][i] = 0.0f;
    for (int s = 0; s < slots<3>(); ++s) for (int i = 0; i < 4; ++i) g3[s][i] = 0.0f;
    for (int s = 0; s < slots<4>(); ++s) for (int i = 0; i < 4; ++i) g4[s][i] = 0.0f;
    float myloss = 0.0f;
    const float inv_n = 1.0f / float(n);

    for (int64_t chunk = int64_t(blockIdx.x) * TB; chunk < n; chunk += int64_t(gridDim.x) * TB) {
        const int64_t base = chunk + 16 * w;
        for (int j = lane; j < 16 * 8; j += 32) {
            const int64_t s = base + j / 8;
            sm.sx[w][j] = s < n ? x[s * 8 + (j & 7)] : 0.0f;
        }
        for (int j = lane; j < 16 * 2; j += 32) {
            const int64_t s = base + j / 2;
            sm.sy[w][j] = s < n ? tgt[s * 2 + (j & 1)] : 0.0f;
        }
        __syncwarp();
        float z[3][8][4], o[4];
        forward16(P, sm.sx[w], lane, o, z);
        // dy in the output-fragment layout (lanes t == 0 own outputs 0, 1)
        float dz4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (t == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = g + (i >= 2 ? 8 : 0), k = i & 1;
                const bool valid = base + row < n;
                const float ty = sm.sy[w][row * 2 + k];
                if (mode == 0) {
                    const float d = o[i] - ty;
                    dz4[i] = valid ? 2.0f * d * inv_n : 0.0f;
                    myloss += valid ? d * d * inv_n : 0.0f;
                } else {
                    dz4[i] = valid ? ty : 0.0f;
                }
            }
        }
        // ---- layer 4: dW4 = dz4^T a3, da3 = dz4 W4
        float v8[8][4];
        __syncthreads();   // previous chunk's gradient products are done with the buffers
        // rows 0..15 of dz^T for this warp's 16 sample columns: outputs 0, 1 and zero padding
        for (int j = lane; j < 16 * 16; j += 32) sm.dzT[j / 16][16 * w + (j % 16)] = __float2bfloat16_rn(0.0f);
        __syncwarp();
        if (t == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) sm.dzT[i & 1][16 * w + g + (i >= 2 ? 8 : 0)] = __float2bfloat16_rn(dz4[i]);
        }
        stage_T_silu(sm.aT, z[2], w, lane);
        __syncthreads();
        grad_gemm<4>(sm, g4, w, lane);
        {
            uint32_t a[4];
            a[0] = pack_bf16(dz4[0], dz4[1]);
            a[1] = pack_bf16(dz4[2], dz4[3]);
            a[2] = 0u; a[3] = 0u;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                v8[nt][0] = v8[nt][1] = v8[nt][2] = v8[nt][3] = 0.0f;
                uint32_t b0, b1;
                bfrag(P.w + PW4T, S4T, nt, 0, lane, b0, b1);
                mma16816(v8[nt], a, b0, b1);
            }
        }
        // ---- layers 3, 2: dz = da * silu'(z); dW = dz^T a_prev; da_prev = dz W
#pragma unroll
        for (int L = 3; L >= 2; --L) {
            const float(*zl)[4] = z[L - 1];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) v8[nt][i] *= dsilu(zl[nt][i]);
            __syncthreads();
            stage_T(sm.dzT, v8, w, lane, [](float q) { return q; });
            stage_T_silu(sm.aT, z[L - 2], w, lane);
            __syncthreads();
            if (L == 3) grad_gemm<3>(sm, g3, w, lane);
            else grad_gemm<2>(sm, g2, w, lane);
            uint32_t a[4][4];
            acc_to_a(v8, a, [](float q) { return q; });
            const __nv_bfloat16 *WT = P.w + (L == 3 ? PW3T : PW2T);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                v8[nt][0] = v8[nt][1] = v8[nt][2] = v8[nt][3] = 0.0f;
#pragma unroll
                for (int kt = 0; kt < 4; ++kt) {
                    uint32_t b0, b1;
                    bfrag(WT, S, nt, kt, lane, b0, b1);
                    mma16816(v8[nt], a[kt], b0, b1);
                }
            }
        }
        // ---- layer 1: dz1 = da1 * silu'(z1); dW1 = dz1^T x (ones row at input 7)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) v8[nt][i] *= dsilu(z[0][nt][i]);
        __syncthreads();
        stage_T(sm.dzT, v8, w, lane, [](float q) { return q; });
        for (int j = lane; j < 16 * 16; j += 32) {
            const int row = j / 16, k = j % 16;     // sample row, input k
            float v = 0.0f;
            if (k < NIN) v = sm.sx[w][row * 8 + k];
            else if (k == NIN) v = 1.0f;
            sm.aT[k][16 * w + row] = __float2bfloat16_rn(v);
        }
        __syncthreads();
        grad_gemm<1>(sm, g1, w, lane);
    }
    __syncthreads();
    float *out = partial + int64_t(blockIdx.x) * NPARAM;
    grad_store<1>(g1, out, w, lane);
    grad_store<2>(g2, out, w, lane);
    grad_store<3>(g3, out, w, lane);
    grad_store<4>(g4, out, w, lane);
    for (int off = 16; off > 0; off >>= 1) myloss += __shfl_xor_sync(0xffffffffu, myloss, off);
    if (lane == 0) sm.loss[w] = myloss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int k = 0; k < 8; ++k) s += sm.loss[k];
        loss_partial[blockIdx.x] = s;
    }
}

// sum the per-CTA partials in CTA order; entries no tile wrote stay 0 (cleared first)
__global__ void k_grad_reduce(const float *__restrict__ partial, int nblk, float *grad, const float *__restrict__ lp,
                              float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) {
        float s = 0.0f;
        for (int b = 0; b < nblk; ++b) s += partial[int64_t(b) * NPARAM + i];
        grad[i] = s;
    }
    if (i == 0 && loss) {
        float s = 0.0f;
        for (int b = 0; b < nblk; ++b) s += lp[b];
        *loss = s;
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; t counts from 1
__global__ void k_adam(float *th, float *m, float *v, const float *__restrict__ grad, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gr = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gr;
    const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static int grad_blocks(int64_t n)
{
    const int64_t b = (n + TB - 1) / TB;
    return int(b < 148 ? (b > 0 ? b : 1) : 148);
}

}  // namespace amr

using namespace amr;

extern "C" size_t mlp_packed_bytes(void) { return mlp::PACKED_BYTES; }
extern "C" int mlp_nparams(void) { return mlp::NPARAM; }
extern "C" size_t mlp_scratch_bytes(int64_t n)
{
    return (size_t(grad_blocks(n)) * (mlp::NPARAM + 1) + mlp::NPARAM + 64) * sizeof(float);
}

extern "C" amr_status mlp_pack(const float *d_theta, void *d_packed, amr_stream stream)
{
    if (!d_theta || !d_packed || (uintptr_t(d_packed) & 15)) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Packed P = view(d_packed);
    const int tot = mlp::PEND + 3 * mlp::H + 8;
    k_pack<<<(tot + 255) / 256, 256, 0, st>>>(d_theta, const_cast<__nv_bfloat16 *>(P.w), const_cast<float *>(P.b));
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status mlp_make_dataset(const double *d_states, int64_t n, double gamma, float *d_x, float *d_y,
                                       int32_t *d_status, amr_stream stream)
{
    if (!d_states || !d_x || !d_y || n < 0 || !(gamma > 1.0)) return AMR_EINVAL;
    if (n == 0) return AMR_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_make_dataset<<<unsigned((n + 255) / 256), 256, 0, st>>>(d_states, n, gamma, d_x, d_y, d_status);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status mlp_forward(const void *d_packed, const float *d_x, float *d_y, int64_t n, amr_stream stream)
{
    if (!d_packed || n < 0) return AMR_EINVAL;
    if (n == 0) return AMR_OK;                       // no samples: the buffers are not used
    if (!d_x || !d_y) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t warps = (n + 15) / 16;
    const int64_t blocks = (warps + 7) / 8;
    k_forward<<<unsigned(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(d_packed, d_x, d_y, n);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

static amr_status grad_launch(const void *d_packed, const float *d_x, const float *d_t, int64_t n, int mode,
                              float *d_grad, float *d_loss, float *d_scratch, size_t scratch_bytes, cudaStream_t st)
{
    if (scratch_bytes < mlp_scratch_bytes(n)) return AMR_ECAPACITY;
    const int nb = grad_blocks(n);
    float *partial = d_scratch, *lp = d_scratch + size_t(nb) * mlp::NPARAM;
    AMR_CUDA_TRY(cudaMemsetAsync(partial, 0, size_t(nb) * mlp::NPARAM * sizeof(float), st));
    const size_t smem = sizeof(TrainSmem);
    AMR_CUDA_TRY(cudaFuncSetAttribute(k_train_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    k_train_grad<<<nb, 256, smem, st>>>(d_packed, d_x, d_t, n, mode, partial, lp);
    AMR_CUDA_TRY(cudaGetLastError());
    k_grad_reduce<<<(mlp::NPARAM + 255) / 256, 256, 0, st>>>(partial, nb, d_grad, lp, d_loss);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status mlp_grad(const void *d_packed, const float *d_x, const float *d_dy, int64_t n, float *d_grad,
                               float *d_scratch, size_t scratch_bytes, amr_stream stream)
{
    if (!d_packed || !d_x || !d_dy || !d_grad || !d_scratch || n <= 0) return AMR_EINVAL;
    return grad_launch(d_packed, d_x, d_dy, n, 1, d_grad, nullptr, d_scratch, scratch_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

extern "C" amr_status mlp_train_step(float *d_theta, float *d_adam_m, float *d_adam_v, void *d_packed,
                                     const float *d_x, const float *d_y, int64_t n, float lr, int64_t t,
                                     float *d_loss, float *d_scratch, size_t scratch_bytes, amr_stream stream)
{
    if (!d_theta || !d_adam_m || !d_adam_v || !d_packed || !d_x || !d_y || !d_scratch || n <= 0 || t < 1)
        return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float *grad = d_scratch + size_t(grad_blocks(n)) * (mlp::NPARAM + 1);
    amr_status r = grad_launch(d_packed, d_x, d_y, n, 0, grad, d_loss, d_scratch, scratch_bytes, st);
    if (r != AMR_OK) return r;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, float(t)), c2 = 1.0f - powf(b2, float(t));
    k_adam<<<(mlp::NPARAM + 255) / 256, 256, 0, st>>>(d_theta, d_adam_m, d_adam_v, grad, lr, b1, b2, 1e-8f, c1, c2);
    AMR_CUDA_TRY(cudaGetLastError());
    return mlp_pack(d_theta, d_packed, stream);
}
