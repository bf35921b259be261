// refine_fine (Table 1): refinement of the octree between steps, on the device.
//
//   1. k_ref_flag: a cell at level l (levelmin <= l < lmax) is refined iff its mass
//      rho dx_l^3 exceeds the threshold; cells above levelmin always are.
//   2. k_ref_balance, one launch per level from the finest up: every refined cell refines
//      the parent-level cells that contain its 26 neighbours (2 per axis, its own father
//      among them), found through the old tree's same-level neighbour table of its
//      father's oct.  After this pass the new tree obeys the 2:1 rule.
//   3. k_ref_exists, one launch per level from the coarsest down: a cell whose father is
//      not refined does not exist in the new tree (a no-op after step 2, kept so that the
//      list is a tree whatever the state).
//   4. An exclusive scan of the flags places the child oct of each refined cell; the new
//      list is the root oct plus those children, counted per level from the scan at the
//      level boundaries of the old tree (cells are in level order).
// The list then goes to amr_build_octree_device (Hilbert keys, sort, tables), and
// k_remap moves the state: an oct present in both trees is copied, a new oct is
// interpolated from its father cell in the old tree with the ghost-cell formula.
#include <cub/device/device_scan.cuh>
#include "godunov_impl.cuh"

namespace amr {

__global__ void k_ref_flag(TreeView tv, const double *__restrict__ rho, double thr, int lmax, int32_t *flag)
{
    const int64_t ncell = tv.ncell;
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < ncell; c += int64_t(gridDim.x) * blockDim.x) {
        const int l = tv.lvl[c >> 3];
        int32_t f;
        if (l < tv.levelmin) f = 1;
        else if (l >= lmax) f = 0;
        else f = rho[c] * pow2(-3 * l) > thr;
        flag[c] = f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) flag[ncell] = 0;    // the scan's extra entry
}

// refined cells of level l mark the level-(l-1) cells containing their neighbours
__global__ void k_ref_balance(TreeView tv, int l, int32_t *flag, int32_t *err)
{
    const int64_t c0 = tv.lvl_off[l] * 8, c1 = tv.lvl_off[l + 1] * 8;
    for (int64_t c = c0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < c1;
         c += int64_t(gridDim.x) * blockDim.x) {
        if (!flag[c]) continue;
        const int64_t o = c >> 3;
        const int cc = int(c & 7);
        const int32_t F = tv.father[o];
        const int64_t P = F >> 3;                        // the oct of the father cell (level l-1)
        const int32_t fx = tv.ix[o], fy = tv.iy[o], fz = tv.iz[o];   // father cell coordinates
        const int32_t X = 2 * fx + (cc & 1), Y = 2 * fy + ((cc >> 1) & 1), Z = 2 * fz + ((cc >> 2) & 1);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            // parents (X -+ 1) >> 1 of the neighbours along each axis (floor shifts)
            const int32_t Tx = (X + ((t & 1) ? 1 : -1)) >> 1, Ty = (Y + ((t & 2) ? 1 : -1)) >> 1,
                          Tz = (Z + ((t & 4) ? 1 : -1)) >> 1;
            const int dx = (Tx >> 1) - (fx >> 1), dy = (Ty >> 1) - (fy >> 1), dz = (Tz >> 1) - (fz >> 1);
            const int32_t N = tv.nb27[P * 27 + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
            if (N == INT32_MIN) continue;                // beyond an outflow face: nothing needed
            if (N < 0) { set_error(err, AMR_EUNBALANCED); continue; }
            flag[int64_t(N) * 8 + (Tx & 1) + 2 * (Ty & 1) + 4 * (Tz & 1)] = 1;
        }
    }
}

__global__ void k_ref_exists(TreeView tv, int l, int32_t *flag)
{
    const int64_t c0 = tv.lvl_off[l] * 8, c1 = tv.lvl_off[l + 1] * 8;
    for (int64_t c = c0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < c1;
         c += int64_t(gridDim.x) * blockDim.x)
        if (flag[c] && !flag[tv.father[c >> 3]]) flag[c] = 0;
}

__global__ void k_ref_emit(TreeView tv, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                           int32_t *lxyz)
{
    const int64_t ncell = tv.ncell;
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < ncell; c += int64_t(gridDim.x) * blockDim.x) {
        if (!flag[c]) continue;
        const int64_t o = c >> 3;
        const int cc = int(c & 7);
        int32_t *e = lxyz + 4 * (1 + int64_t(pos[c]));
        e[0] = tv.lvl[o] + 1;
        e[1] = 2 * tv.ix[o] + (cc & 1);
        e[2] = 2 * tv.iy[o] + ((cc >> 1) & 1);
        e[3] = 2 * tv.iz[o] + ((cc >> 2) & 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        lxyz[0] = 1; lxyz[1] = 0; lxyz[2] = 0; lxyz[3] = 0;        // the root oct
    }
}

// pos at the first cell of each level (and the end), for the per-level counts
__global__ void k_ref_bounds(TreeView tv, const int32_t *__restrict__ pos, int32_t *out)
{
    const int l = threadIdx.x;
    if (l < AMR_MAXLEV + 2) out[l] = pos[tv.lvl_off[l] * 8];
}

// the oct of level l with Hilbert key k in a tree sorted by (level, key), or -1
__device__ __forceinline__ int64_t find_oct(const TreeView &tv, int l, uint64_t k)
{
    if (l < 1 || l > tv.levelmax) return -1;
    int64_t lo = tv.lvl_off[l], hi = tv.lvl_off[l + 1] - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const uint64_t km = tv.key[mid];
        if (km == k) return mid;
        if (km < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__global__ void k_remap(TreeView to, const double *__restrict__ u_old, TreeView tn, double *__restrict__ u_new,
                        int32_t *err)
{
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < tn.noct; o += int64_t(gridDim.x) * blockDim.x) {
        const int l = tn.lvl[o];
        const int64_t p = find_oct(to, l, tn.key[o]);
        if (p >= 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int c = 0; c < 8; ++c) u_new[v * tn.ncell + o * 8 + c] = u_old[v * to.ncell + p * 8 + c];
            continue;
        }
        // a new oct: its father cell exists in the old tree (a leaf there)
        const int32_t Fn = tn.father[o];
        const int64_t Po = Fn >= 0 ? find_oct(to, l - 1, tn.key[Fn >> 3]) : -1;
        if (Po < 0) {
            set_error(err, AMR_EUNBALANCED);
            continue;
        }
        const int64_t Fo = Po * 8 + (Fn & 7);
        for (int c = 0; c < 8; ++c) {
            double U[NV];
            interp_child<double>(to, u_old, Fo, c, U);
#pragma unroll
            for (int v = 0; v < NV; ++v) u_new[v * tn.ncell + o * 8 + c] = U[v];
        }
    }
}

struct RefineWs {
    size_t flag, pos, bounds, err, cub, total, cub_bytes;
};

static RefineWs refine_ws(int64_t ncell)
{
    RefineWs W;
    size_t o = 0;
    auto put = [&](size_t b) { size_t at = o; o += (b + 255) & ~size_t(255); return at; };
    W.flag = put(4 * size_t(ncell + 1));
    W.pos = put(4 * size_t(ncell + 1));
    W.bounds = put(4 * (AMR_MAXLEV + 2));
    W.err = put(4);
    size_t cb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, cb, (int32_t *)nullptr, (int32_t *)nullptr, int(ncell + 1));
    W.cub_bytes = cb;
    W.cub = put(cb);
    W.total = o;
    return W;
}

static int grid_for(int64_t n) { return int(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096); }

}  // namespace amr

using namespace amr;

extern "C" size_t amr_refine_work_bytes(const amr_tree *t)
{
    if (!t || t->noct <= 0 || t->n_inst != 0) return 0;
    return refine_ws(8 * t->noct).total;
}

extern "C" amr_status amr_refine(const amr_tree *t, const amr_refine_params *p, const double *d_u, void *d_work,
                                 size_t work_bytes, int32_t *d_lxyz, int64_t cap, int64_t *h_level_counts,
                                 int64_t *h_n, amr_stream stream)
{
    if (!t || !p || !d_u || !d_work || !d_lxyz || !h_level_counts || !h_n) return AMR_EINVAL;
    if (t->noct <= 0 || t->n_inst != 0) return AMR_EINVAL;
    if (p->levelmax < t->levelmin || p->levelmax > 20 || !(p->mass_thr >= 0.0)) return AMR_EINVAL;
    if (uintptr_t(d_work) & 255) return AMR_EINVAL;
    const int64_t ncell = 8 * t->noct;
    const RefineWs W = refine_ws(ncell);
    if (work_bytes < W.total) return AMR_ECAPACITY;
    if (cap < ncell + 1) return AMR_ECAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *S = static_cast<char *>(d_work);
    int32_t *flag = (int32_t *)(S + W.flag), *pos = (int32_t *)(S + W.pos), *bounds = (int32_t *)(S + W.bounds);
    int32_t *err = (int32_t *)(S + W.err);
    const TreeView tv = make_view(t);
    AMR_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));
    k_ref_flag<<<grid_for(ncell), 256, 0, st>>>(tv, d_u, p->mass_thr, p->levelmax, flag);
    for (int l = t->levelmax; l > t->levelmin; --l) {
        const int64_t nl = 8 * (t->lvl_off[l + 1] - t->lvl_off[l]);
        if (nl > 0) k_ref_balance<<<grid_for(nl), 256, 0, st>>>(tv, l, flag, err);
    }
    for (int l = t->levelmin + 1; l <= t->levelmax; ++l) {
        const int64_t nl = 8 * (t->lvl_off[l + 1] - t->lvl_off[l]);
        if (nl > 0) k_ref_exists<<<grid_for(nl), 256, 0, st>>>(tv, l, flag);
    }
    size_t cb = W.cub_bytes;
    AMR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(S + W.cub, cb, flag, pos, int(ncell + 1), st));
    k_ref_emit<<<grid_for(ncell), 256, 0, st>>>(tv, flag, pos, d_lxyz);
    k_ref_bounds<<<1, 32, 0, st>>>(tv, pos, bounds);
    int32_t hb[AMR_MAXLEV + 2], herr = 0;
    AMR_CUDA_TRY(cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    AMR_CUDA_TRY(cudaStreamSynchronize(st));
    AMR_CUDA_TRY(cudaGetLastError());
    if (herr != 0) return amr_status(herr);
    // refined cells of level l become the octs of level l+1
    for (int l = 0; l <= AMR_MAXLEV; ++l) h_level_counts[l] = 0;
    h_level_counts[1] = 1;
    int64_t n = 1;
    for (int l = 1; l <= t->levelmax && l < AMR_MAXLEV; ++l) {
        const int64_t k = int64_t(hb[l + 1]) - hb[l];
        h_level_counts[l + 1] = k;
        n += k;
    }
    *h_n = n;
    return AMR_OK;
}

extern "C" amr_status amr_remap_state(const amr_tree *t_old, const double *d_u_old, const amr_tree *t_new,
                                      double *d_u_new, int32_t *d_status, amr_stream stream)
{
    if (!t_old || !d_u_old || !t_new || !d_u_new || t_old->n_inst != 0 || t_new->n_inst != 0) return AMR_EINVAL;
    if (t_old->noct <= 0 || t_new->noct <= 0 || d_u_old == d_u_new) return AMR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_remap<<<grid_for(t_new->noct), 256, 0, st>>>(make_view(t_old), d_u_old, make_view(t_new), d_u_new, d_status);
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}
