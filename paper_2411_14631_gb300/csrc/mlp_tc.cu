// Inference of the learned Riemann surrogate on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), over tiles of 128 samples.
//
// The network is the one of mlp_warp.cuh (7 -> 64 -> 64 -> 64 -> 2, SiLU on the hidden
// layers, BF16 weights and activations, FP32 accumulation), the project's stand-in for
// the iterative exact Riemann solver (Toro 2009, Ch. 4).  One CTA of 128 threads takes a
// tile of 128 samples (UMMA M = 128): the operands sit in shared memory in the K-major
// layout without swizzle (8-row x 16-byte core matrices), one elected thread issues the
// MMAs of a layer (K = 16 per instruction) into 64 TMEM columns and commits them to an
// mbarrier; each warp then reads its 32 rows back (tcgen05.ld), adds the bias and applies
// SiLU on BF16 pairs (the same arithmetic as the mma.sync path) and writes the next
// layer's operand.  Waits are bounded: one that runs out writes AMR_ETIMEOUT, and the CTA
// frees its tensor memory and returns.
#include <cstdint>
#include <cuda_bf16.h>
#include "common.cuh"
#include "mlp_warp.cuh"

namespace amr {
namespace mlp {

constexpr int TM = 128;            // samples per tile (UMMA M)
constexpr int TMEM_COLS = 64;      // FP32 accumulator columns (the widest layer)

// byte offset of element (r, k) of a K-major operand with K columns (BF16), no swizzle:
// core matrix (r/8, k/8) at (r/8) * SBO + (k/8) * LBO, LBO = 128 B, SBO = 16 K bytes
__host__ __device__ constexpr int cofs(int r, int k, int K) { return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

struct TcSmem {
    alignas(128) uint8_t w1[64 * 16 * 2];   // B operands (N x K): W1 64 x 16 (7 used)
    alignas(128) uint8_t w2[64 * 64 * 2];
    alignas(128) uint8_t w3[64 * 64 * 2];
    alignas(128) uint8_t w4[16 * 64 * 2];   // W4 padded to N = 16 (2 used)
    alignas(128) uint8_t x[TM * 16 * 2];    // A operands (M x K): the input tile (K 16, 7 used)
    alignas(128) uint8_t h[TM * 64 * 2];    // hidden activations
    float b[3 * H + 8];
    alignas(8) uint64_t mbar;
    uint32_t tmem;
    int32_t fail;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, int K)
{
    uint64_t d = uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t((128 >> 4) & 0x3FFF) << 16;
    d |= uint64_t(((K * 16) >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// bounded wait for the mbarrier phase (about half a second of SM clock); false if it ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase)
{
    const uint32_t a = smem_u32(mbar);
    const long long t0 = clock64();
    while (clock64() - t0 < 1000000000ll) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 FP32 accumulator columns of the warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(TM) k_forward_tc(const void *packed, const float *__restrict__ x, float *y, int64_t n,
                                                   int32_t *status)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the operand arrays want 128-byte alignment in the shared window (the launch adds 1 KB)
    const uint32_t mis = smem_u32(smem_raw) & 1023u;
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw + (mis ? 1024u - mis : 0u));
    const Packed P = view(packed);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t ntile = (n + TM - 1) / TM;

    // weights and biases into the operand layout (once per CTA)
    auto put = [](uint8_t *base, int r, int k, int K, __nv_bfloat16 v) {
        *reinterpret_cast<__nv_bfloat16 *>(base + cofs(r, k, K)) = v;
    };
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int i = tid; i < 64 * 16; i += TM) put(sm.w1, i >> 4, i & 15, 16, P.w[PW1 + (i >> 4) * S1 + (i & 15)]);
    for (int i = tid; i < 64 * 64; i += TM) {
        put(sm.w2, i >> 6, i & 63, 64, P.w[PW2 + (i >> 6) * S + (i & 63)]);
        put(sm.w3, i >> 6, i & 63, 64, P.w[PW3 + (i >> 6) * S + (i & 63)]);
    }
    for (int i = tid; i < 16 * 64; i += TM) {
        const int r = i >> 6, k = i & 63;
        put(sm.w4, r, k, 64, r < 8 ? P.w[PW4 + r * S + k] : zero);
    }
    for (int i = tid; i < 3 * H + 8; i += TM) sm.b[i] = P.b[i];
    if (tid == 0) {
        sm.fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.mbar)), "r"(1) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t lane_base = uint32_t(32 * warp) << 16;   // this warp's TMEM lanes
    const uint32_t xa = smem_u32(sm.x), ha = smem_u32(sm.h);
    const uint32_t wa[4] = {smem_u32(sm.w1), smem_u32(sm.w2), smem_u32(sm.w3), smem_u32(sm.w4)};
    uint32_t phase = 0;

    // one layer: MMAs over K/16 slices by thread 0, commit, wait (bounded)
    auto layer = [&](uint32_t a, int K, uint32_t b, int N) -> bool {
        if (tid == 0) {
            const uint32_t idesc = umma_idesc(TM, N);
            for (int kk = 0; kk < K / 16; ++kk)
                mma_bf16(tmem, umma_desc(a + kk * 256, K), umma_desc(b + kk * 256, K), idesc, kk > 0);
            mma_commit(&sm.mbar);
        }
        // the same answer in every thread: no thread leaves the tile loop alone
        const bool ok = __syncthreads_and(mbar_wait(&sm.mbar, phase)) != 0;
        phase ^= 1u;
        fence_after();
        return ok;
    };
    // hidden-layer epilogue of this thread's row: bias, SiLU on BF16 pairs, into sm.h
    auto hidden_out = [&](const float *bias) {
        const int r = tid;
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + uint32_t(c), v);
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = silu_bf16x2(v[2 * i] + bias[c + 2 * i], v[2 * i + 1] + bias[c + 2 * i + 1]);
            *reinterpret_cast<uint4 *>(sm.h + cofs(r, c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(sm.h + cofs(r, c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
    };

    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        // the input tile: 7 features (slot 7 of the 8 stored is unused), zero padded to K = 16
        {
            const int64_t s = t * TM + tid;
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = (s < n && k < NIN) ? x[s * 8 + k] : 0.0f;
            *reinterpret_cast<uint4 *>(sm.x + cofs(tid, 0, 16)) =
                make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
            *reinterpret_cast<uint4 *>(sm.x + cofs(tid, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        ok = layer(xa, 16, wa[0], 64);
        if (!ok) break;
        hidden_out(sm.b);
        ok = layer(ha, 64, wa[1], 64);
        if (!ok) break;
        hidden_out(sm.b + H);
        ok = layer(ha, 64, wa[2], 64);
        if (!ok) break;
        hidden_out(sm.b + 2 * H);
        ok = layer(ha, 64, wa[3], 16);
        if (!ok) break;
        {
            float v[16];
            tmem_ld16(tmem + lane_base, v);
            const int64_t s = t * TM + tid;
            if (s < n) {
                y[2 * s] = v[0] + sm.b[3 * H];
                y[2 * s + 1] = v[1] + sm.b[3 * H + 1];
            }
        }
        fence_before();
        __syncthreads();     // TMEM columns free for the next tile's first layer
        fence_after();
    }
    if (!ok) {
        set_error(status, AMR_ETIMEOUT);
        // the MMAs may still be in flight: one more bounded wait before the memory is freed
        mbar_wait(&sm.mbar, phase);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace mlp
}  // namespace amr

using namespace amr;

extern "C" amr_status mlp_forward_tc(const void *d_packed, const float *d_x, float *d_y, int64_t n, int32_t *d_status,
                                     amr_stream stream)
{
    if (!d_packed || !d_x || !d_y || n < 0) return AMR_EINVAL;
    if (n == 0) return AMR_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = sizeof(mlp::TcSmem) + 1024;
    AMR_CUDA_TRY(cudaFuncSetAttribute(mlp::k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntile = (n + mlp::TM - 1) / mlp::TM;
    const int64_t grid = ntile < int64_t(4) * nsm ? ntile : int64_t(4) * nsm;
    mlp::k_forward_tc<<<unsigned(grid), mlp::TM, smem, st>>>(d_packed, d_x, d_y, n, d_status);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}
