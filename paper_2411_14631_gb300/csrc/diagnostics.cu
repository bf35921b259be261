// Global conservation diagnostics on the device: the totals of the conserved variables
// over the leaf cells, sum_leaf U_v dV (mass, momentum, total energy), per box in batch
// mode.  These are the conservation bookkeeping of the level step (Table 1: godunov_fine
// with its refluxing keeps them constant up to rounding in a periodic box); the paper
// prints no formula for them, the definition above is the plain one.
//
// Deterministic and independent of the launch shape: the octs are cut into fixed chunks
// of 256 (per box in batch mode); a chunk's partial sums are formed in a fixed order (per
// oct its eight cells in cell order, then a fixed reduction tree over the chunk's 256
// octs); a second pass sums each box's chunk partials in a fixed order.  FP64 throughout,
// no atomics, no host synchronisation.
#include "common.cuh"

namespace amr {

constexpr int CONS_CHUNK = 256;   // octs per chunk = threads per CTA

// chunk offsets: chunk_off[b] = first chunk of box b (octree mode: one box of all octs)
__global__ void k_cons_chunks(int32_t n_inst, int64_t noct, const int64_t *__restrict__ inst_oct_off,
                              int64_t *__restrict__ chunk_off)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    chunk_off[0] = 0;
    if (n_inst == 0) {
        chunk_off[1] = (noct + CONS_CHUNK - 1) / CONS_CHUNK;
        return;
    }
    int64_t c = 0;
    for (int b = 0; b < n_inst; ++b) {
        c += (inst_oct_off[b + 1] - inst_oct_off[b] + CONS_CHUNK - 1) / CONS_CHUNK;
        chunk_off[b + 1] = c;
    }
}

// sum of the 2 x NV values over the CTA's 256 threads in a fixed order: a butterfly per
// warp (IEEE addition is commutative, so every lane ends with the same bits), then the
// eight warp sums in warp order
__device__ __forceinline__ void cta_sum10(double s[2 * NV], double (*red)[2 * NV], double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 2 * NV; ++k)
        for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 2 * NV; ++k) red[warp][k] = s[k];
    __syncthreads();
    if (threadIdx.x < 2 * NV) {
        double acc = red[0][threadIdx.x];
        for (int w = 1; w < CONS_CHUNK / 32; ++w) acc += red[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

// per chunk: [sum_leaf U_v dV, sum_leaf |U_v| dV] (v = 0..4) into part[chunk][10]
__global__ void __launch_bounds__(CONS_CHUNK) k_cons_partial(TreeView tv, const int64_t *__restrict__ inst_oct_off,
                                                             const int64_t *__restrict__ chunk_off,
                                                             const double *__restrict__ u, double *__restrict__ part)
{
    __shared__ double red[CONS_CHUNK / 32][2 * NV];
    const int nbox = tv.n_inst > 0 ? tv.n_inst : 1;
    const int64_t nch = chunk_off[nbox];
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        int b = 0;
        if (tv.n_inst > 0) {
            int lo = 0, hi = nbox - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (chunk_off[mid] <= ch) lo = mid; else hi = mid - 1;
            }
            b = lo;
        }
        const int64_t obox = tv.n_inst > 0 ? inst_oct_off[b] : 0;
        const int64_t oend = tv.n_inst > 0 ? inst_oct_off[b + 1] : tv.noct;
        const int64_t o = obox + (ch - chunk_off[b]) * CONS_CHUNK + threadIdx.x;
        double s[2 * NV];
#pragma unroll
        for (int k = 0; k < 2 * NV; ++k) s[k] = 0.0;
        if (o < oend) {
            double dV;
            unsigned rm = 0;
            if (tv.n_inst > 0) {
                const double dx = tv.inst_dx[b];
                dV = dx * dx * dx;
            } else {
                dV = pow2(-3 * tv.lvl[o]);
                rm = tv.refmask[o];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                // the oct's eight cells of variable v: four 16-byte loads
                const double2 *row = reinterpret_cast<const double2 *>(u + v * tv.ncell + o * 8);
                double x[8];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const double2 q = row[h];
                    x[2 * h] = q.x;
                    x[2 * h + 1] = q.y;
                }
                double sv = 0.0, av = 0.0;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if ((rm >> c) & 1u) continue;          // refined: not a leaf
                    sv += x[c];
                    av += fabs(x[c]);
                }
                s[v] = sv * dV;
                s[NV + v] = av * dV;
            }
        }
        cta_sum10(s, red, part + ch * 2 * NV);
    }
}

// per box: its chunk partials in chunk order (thread t takes chunks t, t + 256, ...), then
// the fixed CTA tree
__global__ void __launch_bounds__(CONS_CHUNK) k_cons_final(const int64_t *__restrict__ chunk_off,
                                                           const double *__restrict__ part, double *__restrict__ totals)
{
    __shared__ double red[CONS_CHUNK / 32][2 * NV];
    const int b = blockIdx.x;
    double s[2 * NV];
#pragma unroll
    for (int k = 0; k < 2 * NV; ++k) s[k] = 0.0;
    for (int64_t ch = chunk_off[b] + threadIdx.x; ch < chunk_off[b + 1]; ch += CONS_CHUNK)
#pragma unroll
        for (int k = 0; k < 2 * NV; ++k) s[k] += part[ch * 2 * NV + k];
    cta_sum10(s, red, totals + int64_t(b) * 2 * NV);
}

}  // namespace amr

using namespace amr;

static size_t cons_off_bytes(const amr_tree *t)
{
    const int64_t nbox = t->n_inst > 0 ? t->n_inst : 1;
    return (size_t(nbox + 1) * sizeof(int64_t) + 255) & ~size_t(255);
}

extern "C" size_t hydro_conservation_work_bytes(const amr_tree *t)
{
    if (!t || t->noct <= 0) return 0;
    const int64_t nbox = t->n_inst > 0 ? t->n_inst : 1;
    const int64_t nch = t->noct / CONS_CHUNK + nbox + 1;   // at least the sum of the per-box ceilings
    return cons_off_bytes(t) + size_t(nch) * 2 * NV * sizeof(double);
}

extern "C" amr_status hydro_conservation(const amr_tree *t, const double *d_u, double *d_totals, void *d_work,
                                         size_t work_bytes, int32_t blocks, amr_stream stream)
{
    if (!t || t->noct <= 0 || !d_u || !d_totals || !d_work || blocks < 0) return AMR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_work) & 255) != 0 || (reinterpret_cast<uintptr_t>(d_u) & 15) != 0)
        return AMR_EINVAL;
    if (work_bytes < hydro_conservation_work_bytes(t)) return AMR_ECAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nbox = t->n_inst > 0 ? t->n_inst : 1;
    int64_t *chunk_off = static_cast<int64_t *>(d_work);
    double *part = reinterpret_cast<double *>(static_cast<char *>(d_work) + cons_off_bytes(t));
    k_cons_chunks<<<1, 32, 0, st>>>(t->n_inst, t->noct, t->inst_oct_off, chunk_off);
    AMR_CUDA_TRY(cudaGetLastError());
    int nb = blocks;
    if (nb == 0) {
        int dev = 0, nsm = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        nb = 4 * nsm;
    }
    k_cons_partial<<<unsigned(nb), CONS_CHUNK, 0, st>>>(make_view(t), t->inst_oct_off, chunk_off, d_u, part);
    AMR_CUDA_TRY(cudaGetLastError());
    k_cons_final<<<unsigned(nbox), CONS_CHUNK, 0, st>>>(chunk_off, part, d_totals);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}
