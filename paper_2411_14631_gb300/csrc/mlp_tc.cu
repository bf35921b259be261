// Inference of the learned Riemann surrogate on the 5th-generation tensor cores
// (tcgen05.mma, accumulators and activations in tensor memory), over tiles of 128 samples.
//
// The network is the one of mlp_warp.cuh (7 -> 64 -> 64 -> 64 -> 2, SiLU on the hidden
// layers, BF16 weights and activations, FP32 accumulation), the project's stand-in for
// the iterative exact Riemann solver (Toro 2009, Ch. 4).  One persistent CTA per SM holds
// the weights once in shared memory (K-major, no swizzle: 8-row x 16-byte core matrices)
// and runs five independent groups of four warps, each on its own tile of 128 samples
// (UMMA M = 128) with its own 96 TMEM columns: 64 FP32 accumulators and the next layer's
// A operand (64 BF16 activations per row).  The group's first thread issues a layer's
// MMAs (the first layer's A from shared memory, the others' from tensor memory) and
// commits them to the group's mbarrier; the group's warps then read the accumulators
// (tcgen05.ld), apply SiLU on BF16 pairs (the arithmetic of the mma.sync path) and write
// the activations back (tcgen05.st), while the tensor cores run the other groups'
// layers.  The hidden biases are folded into the MMAs; the next input tile arrives by
// bulk copy during the current one.
//
// The bound is the SiLU's tanh: the MUFU unit returns 16 tanh results per clock per SM
// (bf16x2 and f32 forms alike), 192 per sample, against about 60 tensor-core cycles per
// 128 samples per layer.  Waits are bounded: one that runs out writes AMR_ETIMEOUT, and
// the group stops after its copies and MMAs in flight have landed (bounded again); the
// CTA frees its tensor memory.
#include <cstdint>
#include <cuda_bf16.h>
#include "common.cuh"
#include "mlp_warp.cuh"

namespace amr {
namespace mlp {

constexpr int TM = 128;            // samples per tile (UMMA M)
constexpr int NG = 5;              // independent tile groups per CTA (4 warps each)
constexpr int NT = 128 * NG;       // threads per CTA (one CTA per SM)
constexpr int GCOLS = 96;          // TMEM columns per group: 64 FP32 accumulators, then the
                                   // next layer's A operand (64 BF16 per row, two per column)
constexpr int TMEM_COLS = 512;     // the allocation (a power of two >= NG * GCOLS)

// byte offset of element (r, k) of a K-major operand with K columns (BF16), no swizzle:
// core matrix (r/8, k/8) at (r/8) * SBO + (k/8) * LBO, LBO = 128 B, SBO = 16 K bytes
__host__ __device__ constexpr int cofs(int r, int k, int K) { return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// The hidden layers' biases ride in the MMAs: a column pair of ones in the A operand
// (k = 8, 9 of the input tile; a shared 128 x 16 "ones" tile for the other layers) meets
// the bias split into two BF16 terms in B, hi = bf16(b) and lo = bf16(b - hi) (|hi + lo - b|
// <= 2^-17 |b|), so the accumulator holds W x + b.  The hidden weights and biases are stored
// halved (exact), so the accumulator is z/2, the argument of SiLU's tanh form.
struct TcSmem {
    alignas(128) uint8_t w1[64 * 16 * 2];    // B operands (N x K): W1|b1
    alignas(128) uint8_t w2[64 * 64 * 2];    // W2, W3
    alignas(128) uint8_t w3[64 * 64 * 2];
    alignas(128) uint8_t wb2[64 * 16 * 2];   // b2, b3 as (hi, lo) columns
    alignas(128) uint8_t wb3[64 * 16 * 2];
    alignas(128) uint8_t w4[16 * 64 * 2];    // W4 padded to N = 16 (2 used)
    alignas(128) uint8_t ones[TM * 16 * 2];  // A operand of the bias MMAs
    alignas(128) uint8_t x[NG][TM * 16 * 2]; // per group: the input tile (A of the first layer)
    alignas(128) float stage[NG][TM * 8];    // per group: the next input tile, FP32, by bulk copy
    alignas(8) uint64_t mma_bar[NG], x_bar[NG];
    float b4[2];
    uint32_t tmem;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle; +16 per K slice of 16
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

// the same with the A operand in tensor memory (row i in lane i, two BF16 per column)
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc));
}

// completion of this thread's prior MMAs arrives on the mbarrier
__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// bounded wait for the mbarrier phase (about half a second of SM clock); false if it ran
// out.  Each try may suspend the thread for up to 20 us until the phase completes.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase)
{
    const uint32_t a = smem_u32(mbar);
    const long long t0 = clock64();
    while (clock64() - t0 < 1000000000ll) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(phase), "r"(20000)
            : "memory");
        if (done) return true;
    }
    return false;
}

// the mbarrier phase is complete (no wait): the acquire of the data it guards, for the
// threads that learned of the completion through a barrier
__device__ __forceinline__ void mbar_acquire(uint64_t *mbar, uint32_t phase)
{
    asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%0], %1;\n}\n" ::"r"(smem_u32(mbar)),
                 "r"(phase)
                 : "memory");
}

// bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory; completion (bytes) arrives on the mbarrier
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// barrier of the 128 threads of group g (named barrier 1 + g), AND of the predicate
__device__ __forceinline__ bool group_sync_and(int g, bool v)
{
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, 128, p;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"(uint32_t(v)), "r"(1 + g)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

// 32 FP32 accumulator columns of the warp's 32 lanes (one row per thread), then the wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 16 32-bit columns of the warp's 32 lanes from registers (one row per thread)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t r[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t r[2])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// SiLU of a pre-activation pair given as halves h = z/2: h + h tanh(h) on BF16 pairs, the
// arithmetic of silu_bf16x2
__device__ __forceinline__ uint32_t silu_half_bf16x2(float h0, float h1)
{
    const uint32_t h = pack_bf16(h0, h1);
    uint32_t t, r;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(h), "r"(t));
    return r;
}

// One CTA per SM; its eight groups of four warps run independent tiles (group g takes
// tiles g, g + NG, ... of the CTA's share), each with its own 64 TMEM columns, operand
// buffer, mbarriers and named barrier, so the tensor cores work on one group's layer while
// the others run their epilogues.  Per tile: the input tile (bulk-copied one tile ahead)
// is converted to the BF16 operand; then four layers, each MMAs issued by the group's
// first thread and committed to the group's mbarrier, then (hidden layers) TMEM ->
// SiLU -> the next operand, in place.
__global__ void __launch_bounds__(NT, 1) k_forward_tc(const void *packed, const float *__restrict__ x, float *y, int64_t n,
                                                      int32_t *status)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the operand arrays want 128-byte alignment in the shared window (the launch adds 1 KB)
    const uint32_t mis = smem_u32(smem_raw) & 1023u;
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw + (mis ? 1024u - mis : 0u));
    const Packed P = view(packed);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = warp >> 2, gt = tid & 127;     // group, thread (= tile row) in the group
    const int64_t ntile = (n + TM - 1) / TM;

    // weights and biases into the operand layout (once per CTA)
    auto put = [](uint8_t *base, int r, int k, int K, __nv_bfloat16 v) {
        *reinterpret_cast<__nv_bfloat16 *>(base + cofs(r, k, K)) = v;
    };
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f), one = __float2bfloat16_rn(1.0f),
                        half = __float2bfloat16_rn(0.5f);
    // (hi, lo) BF16 terms of b/2
    auto bias_terms = [](float b, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
        const float bh = 0.5f * b;
        hi = __float2bfloat16_rn(bh);
        lo = __float2bfloat16_rn(bh - __bfloat162float(hi));
    };
    for (int i = tid; i < 64 * 16; i += NT) {
        const int r = i >> 4, k = i & 15;
        __nv_bfloat16 hi, lo, v1 = zero, v2 = zero, v3 = zero;
        bias_terms(P.b[r], hi, lo);
        if (k < NIN) v1 = __hmul(P.w[PW1 + r * S1 + k], half);
        else if (k == 8) v1 = hi;
        else if (k == 9) v1 = lo;
        bias_terms(P.b[H + r], hi, lo);
        if (k < 2) v2 = k == 0 ? hi : lo;
        bias_terms(P.b[2 * H + r], hi, lo);
        if (k < 2) v3 = k == 0 ? hi : lo;
        put(sm.w1, r, k, 16, v1);
        put(sm.wb2, r, k, 16, v2);
        put(sm.wb3, r, k, 16, v3);
        put(sm.w4, k, r, 64, k < 8 ? P.w[PW4 + k * S + r] : zero);
    }
    for (int i = tid; i < 64 * 64; i += NT) {
        const int r = i >> 6, k = i & 63;
        put(sm.w2, r, k, 64, __hmul(P.w[PW2 + r * S + k], half));
        put(sm.w3, r, k, 64, __hmul(P.w[PW3 + r * S + k], half));
    }
    for (int i = tid; i < TM * 16; i += NT) put(sm.ones, i >> 4, i & 15, 16, (i & 15) < 2 ? one : zero);
    if (tid < 2) sm.b4[tid] = P.b[3 * H + tid];
    if (tid == 0) {
        for (int q = 0; q < NG; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.mma_bar[q])), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.x_bar[q])), "r"(1) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

    const bool leader = gt == 0;
    const uint32_t tacc = sm.tmem + uint32_t(GCOLS * g);                       // the group's accumulators
    const uint32_t tact = tacc + 64u;                                          // and activations
    const uint32_t lanes = uint32_t(32 * (warp & 3)) << 16;                    // this warp's lanes
    uint8_t *const xg = sm.x[g];
    float *const stg = sm.stage[g];
    const uint64_t d_x = umma_desc(smem_u32(xg), 16), d_w1 = umma_desc(smem_u32(sm.w1), 16),
                   d_w2 = umma_desc(smem_u32(sm.w2), 64), d_w3 = umma_desc(smem_u32(sm.w3), 64),
                   d_b2 = umma_desc(smem_u32(sm.wb2), 16), d_b3 = umma_desc(smem_u32(sm.wb3), 16),
                   d_w4 = umma_desc(smem_u32(sm.w4), 64), d_one = umma_desc(smem_u32(sm.ones), 16);
    constexpr uint32_t I64 = umma_idesc(TM, 64), I16 = umma_idesc(TM, 16);
    uint32_t mphase = 0, xphase = 0;       // (every thread) the next phase of each mbarrier
    bool mpend = false, xpend = false;     // (leader) an MMA commit / a bulk copy not yet waited for

    const int64_t tstep = int64_t(gridDim.x) * NG;
    auto issue_x = [&](int64_t t) {        // leader: bulk copy of tile t's inputs into the stage
        const int64_t rows = n - t * TM < TM ? n - t * TM : TM;
        bulk_load(stg, x + t * TM * 8, uint32_t(rows * 32), &sm.x_bar[g]);
        xpend = true;
    };
    // leader waits for the group's MMAs; every thread of the group gets the answer
    auto wait_mma = [&]() -> bool {
        bool ok = true;
        if (leader) {
            ok = mbar_wait(&sm.mma_bar[g], mphase);
            if (ok) mpend = false;
        }
        ok = group_sync_and(g, ok);
        if (ok) {
            if (!leader) mbar_acquire(&sm.mma_bar[g], mphase);
            mphase ^= 1u;
        }
        fence_after();
        return ok;
    };
    // hidden-layer epilogue of this thread's row: SiLU of the 64 accumulators into the
    // next layer's A operand in tensor memory
    auto hidden_out = [&]() {
#pragma unroll
        for (int c = 0; c < 64; c += 32) {
            uint32_t v[32], q[16];
            tmem_ld32(tacc + lanes + uint32_t(c), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) q[i] = silu_half_bf16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
            tmem_st16(tact + lanes + uint32_t(c / 2), q);
        }
        tmem_wait_st();
        fence_before();
        group_sync(g);
        fence_after();
    };

    int64_t t = int64_t(blockIdx.x) * NG + g;
    bool ok = true;
    if (leader && t < ntile) issue_x(t);
    for (; t < ntile; t += tstep) {
        // the input tile: FP32 stage -> BF16 operand (features 0-6, slot 7 zeroed, ones at 8, 9)
        if (leader) {
            ok = mbar_wait(&sm.x_bar[g], xphase);
            if (ok) xpend = false;
        }
        ok = group_sync_and(g, ok);
        if (!ok) break;
        if (!leader) mbar_acquire(&sm.x_bar[g], xphase);
        xphase ^= 1u;
        {
            const float4 a = *reinterpret_cast<const float4 *>(stg + gt * 8);
            const float4 b = *reinterpret_cast<const float4 *>(stg + gt * 8 + 4);
            *reinterpret_cast<uint4 *>(xg + cofs(gt, 0, 16)) =
                make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(b.x, b.y), pack_bf16(b.z, 0.0f));
            *reinterpret_cast<uint4 *>(xg + cofs(gt, 8, 16)) = make_uint4(0x3F803F80u, 0u, 0u, 0u);
        }
        fence_async_smem();
        fence_before();
        group_sync(g);
        fence_after();
        if (leader) {
            if (t + tstep < ntile) issue_x(t + tstep);      // the stage is free again
            mma_bf16(tacc, d_x, d_w1, I64, 0);
            mma_commit(&sm.mma_bar[g]);
            mpend = true;
        }
        if (!(ok = wait_mma())) break;
        hidden_out();
        if (leader) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_bf16_ta(tacc, tact + 8 * kk, d_w2 + 16 * kk, I64, kk > 0);
            mma_bf16(tacc, d_one, d_b2, I64, 1);
            mma_commit(&sm.mma_bar[g]);
            mpend = true;
        }
        if (!(ok = wait_mma())) break;
        hidden_out();
        if (leader) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_bf16_ta(tacc, tact + 8 * kk, d_w3 + 16 * kk, I64, kk > 0);
            mma_bf16(tacc, d_one, d_b3, I64, 1);
            mma_commit(&sm.mma_bar[g]);
            mpend = true;
        }
        if (!(ok = wait_mma())) break;
        hidden_out();
        if (leader) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_bf16_ta(tacc, tact + 8 * kk, d_w4 + 16 * kk, I16, kk > 0);
            mma_commit(&sm.mma_bar[g]);
            mpend = true;
        }
        if (!(ok = wait_mma())) break;
        {
            uint32_t v[2];
            tmem_ld2(tacc + lanes, v);
            const int64_t s = t * TM + gt;
            if (s < n)
                *reinterpret_cast<float2 *>(y + 2 * s) =
                    make_float2(__uint_as_float(v[0]) + sm.b4[0], __uint_as_float(v[1]) + sm.b4[1]);
        }
        fence_before();
        group_sync(g);       // the group's TMEM columns and input buffer free for the next tile
        fence_after();
    }
    if (!ok) {
        if (leader) set_error(status, AMR_ETIMEOUT);
        // copies or MMAs may still be in flight: one more bounded wait for each before the
        // memory is released
        if (leader && xpend) mbar_wait(&sm.x_bar[g], xphase);
        if (leader && mpend) mbar_wait(&sm.mma_bar[g], mphase);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(TMEM_COLS) : "memory");
}

// Throughput of the MUFU tanh, the bound of the kernel above: every thread runs eight
// independent chains of tanh.approx.bf16x2 (the SiLU's instruction); each CTA times its
// chains with the SM clock and the longest time is kept.
constexpr int TANH_ITERS = 1024;
__global__ void __launch_bounds__(512) k_tanh_rate(unsigned long long *cycles)
{
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 0x3C003C00u ^ uint32_t(threadIdx.x * 8 + i);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < TANH_ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) asm volatile("tanh.approx.bf16x2 %0, %0;" : "+r"(a[i]));
    }
    // the results feed a branch (an atomic that adds nothing), so that the chains are
    // neither removed nor left in flight when the clock is read after the barrier
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x9E3779B9u) atomicAdd(cycles, 0ull);
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

}  // namespace mlp
}  // namespace amr

using namespace amr;

extern "C" amr_status mlp_forward_tc(const void *d_packed, const float *d_x, float *d_y, int64_t n, int32_t *d_status,
                                     amr_stream stream)
{
    if (!d_packed || n < 0) return AMR_EINVAL;
    if (n == 0) return AMR_OK;                       // no samples: the buffers are not used
    if (!d_x || !d_y) return AMR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_x) & 15) || (reinterpret_cast<uintptr_t>(d_y) & 7)) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // at least 116 KB of shared memory: one CTA per SM, which the 512-column TMEM
    // allocation assumes
    const size_t smem = sizeof(mlp::TcSmem) + 1024 > 116 * 1024 ? sizeof(mlp::TcSmem) + 1024 : 116 * 1024;
    AMR_CUDA_TRY(cudaFuncSetAttribute(mlp::k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ngroup = (n + mlp::TM - 1) / mlp::TM;
    const int64_t want = (ngroup + mlp::NG - 1) / mlp::NG;
    const int64_t grid = want < nsm ? want : nsm;
    mlp::k_forward_tc<<<unsigned(grid), mlp::NT, smem, st>>>(d_packed, d_x, d_y, n, d_status);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

extern "C" amr_status mlp_tanh_rate(unsigned long long *d_cycles, int64_t *h_results, amr_stream stream)
{
    if (!d_cycles || !h_results) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 4 * nsm, threads = 512;        // four CTAs per SM, all resident at once
    *h_results = int64_t(blocks) * threads * 8 * mlp::TANH_ITERS * 2;
    AMR_CUDA_TRY(cudaMemsetAsync(d_cycles, 0, sizeof(unsigned long long), st));
    mlp::k_tanh_rate<<<blocks, threads, 0, st>>>(d_cycles);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}
