// Internal device helpers shared by the amrhydro kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cmath>
#include <cuda_runtime.h>
#include "../../include/amrhydro.h"

namespace amr {

constexpr int NV = 5;
constexpr int32_t OUTSIDE = INT32_MIN;   // nb27 / slot entry beyond an outflow face

#define AMR_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return AMR_ECUDA;            \
    } while (0)

// First error wins; 0 means no error.
__device__ __forceinline__ void set_error(int32_t *word, int32_t code)
{
    if (word) atomicCAS(word, 0, code);
}

// Peano-Hilbert key of oct coordinates (x,y,z) with `bits` bits each (Sec. 1 of the
// paper: space is ordered along the Peano-Hilbert curve).  Skilling's transposition
// (AIP Conf. Proc. 707, 2004): per bit plane from the top, an inversion or an exchange
// of the lower bits; then a Gray code; the transposed index is interleaved x-first.
__host__ __device__ inline uint64_t hilbert3(int bits, uint32_t x, uint32_t y, uint32_t z)
{
    if (bits <= 0) return 0;
    uint32_t a[3] = {x, y, z};
    for (uint32_t q = 1u << (bits - 1); q > 1; q >>= 1) {
        const uint32_t low = q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (a[i] & q) {
                a[0] ^= low;
            } else {
                const uint32_t sw = (a[0] ^ a[i]) & low;
                a[0] ^= sw;
                a[i] ^= sw;
            }
        }
    }
    a[1] ^= a[0];
    a[2] ^= a[1];
    uint32_t flip = 0;
    for (uint32_t q = 1u << (bits - 1); q > 1; q >>= 1)
        if (a[2] & q) flip ^= q - 1;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b) {
#pragma unroll
        for (int i = 0; i < 3; ++i) key = (key << 1) | (((a[i] ^ flip) >> b) & 1u);
    }
    return key;
}

// 2^e and x * 2^e (x > 0 and normal) by exponent arithmetic on the bit pattern: exact,
// and off the FP64 pipe
__host__ __device__ inline double pow2(int e)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)(1023 + e) << 52);
#else
    return ldexp(1.0, e);
#endif
}
__device__ __forceinline__ double scale_pow2(double x, int e)
{
    return __longlong_as_double(__double_as_longlong(x) + ((long long)e << 52));
}

// Oct index of (l, x, y, z) in the level-sorted key array, or -1.
__device__ __forceinline__ int64_t find_oct(const uint64_t *__restrict__ key, const int64_t *lvl_off, int l,
                                            int64_t x, int64_t y, int64_t z)
{
    if (l < 1 || l > AMR_MAXLEV) return -1;
    const int64_t m = int64_t(1) << (l - 1);
    if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) return -1;
    const uint64_t k = hilbert3(l - 1, uint32_t(x), uint32_t(y), uint32_t(z));
    int64_t lo = lvl_off[l], hi = lvl_off[l + 1] - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const uint64_t km = key[mid];
        if (km == k) return mid;
        if (km < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Periodic wrap (returns 0) or "beyond an outflow face" (returns 1) for a coordinate
// at a level with n cells per dimension.
__device__ __forceinline__ int bc_apply(const int32_t *bc, int axis, int64_t n, int64_t &c)
{
    if (c >= 0 && c < n) return 0;
    const int face = 2 * axis + (c >= n ? 1 : 0);
    if (bc[face] == AMR_BC_PERIODIC) {
        c = ((c % n) + n) % n;
        return 0;
    }
    return 1;
}

// Arguments shared by the hydro kernels (passed by value).
struct TreeView {
    int64_t noct, ncell;
    int32_t levelmin, levelmax;
    int32_t bc[6];
    int64_t lvl_off[AMR_MAXLEV + 2];
    int64_t reg_base;
    const int32_t *lvl, *ix, *iy, *iz;
    const int32_t *son, *nbor, *father;
    const uint8_t *refmask, *fused;
    const uint64_t *key;                 // Hilbert keys (octs sorted by level, then key)
    const int32_t *nb27;                 // same-level neighbour octs (refinement)
    const int32_t *ghost_cell;           // coarse leaves the tiles interpolate from
    int32_t n_inst;                      // batch mode: number of boxes (0: octree)
    const int32_t *inst_n;
    const double *inst_dx;
};

// The flux-register buffer: rows [oct - reg_base][6 faces][NV] of FP64, then (256-byte
// aligned) the interpolated children of the ghost fathers, [n_ghost][8][NV] values of the
// working precision (room for FP64).
inline size_t reg_rows_bytes(const amr_tree *t)
{
    const int64_t rows = t->noct - t->reg_base;
    return (size_t(rows > 0 ? rows : 1) * 6 * NV * sizeof(double) + 255) & ~size_t(255);
}
inline size_t reg_total_bytes(const amr_tree *t)
{
    return reg_rows_bytes(t) + size_t(t->n_ghost > 0 ? t->n_ghost : 0) * 8 * NV * sizeof(double);
}

inline TreeView make_view(const amr_tree *t)
{
    TreeView v;
    v.noct = t->noct;
    v.ncell = 8 * t->noct;
    v.levelmin = t->levelmin;
    v.levelmax = t->levelmax;
    for (int i = 0; i < 6; ++i) v.bc[i] = t->bc[i];
    for (int i = 0; i < AMR_MAXLEV + 2; ++i) v.lvl_off[i] = t->lvl_off[i];
    v.reg_base = t->reg_base;
    v.lvl = t->lvl; v.ix = t->ix; v.iy = t->iy; v.iz = t->iz;
    v.son = t->son; v.nbor = t->nbor; v.father = t->father; v.refmask = t->refmask; v.fused = t->fused;
    v.key = t->key; v.nb27 = t->nb27; v.ghost_cell = t->ghost_cell;
    v.n_inst = t->n_inst; v.inst_n = t->inst_n; v.inst_dx = t->inst_dx;
    return v;
}

}  // namespace amr
