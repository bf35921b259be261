// amr_build_octree: the fully threaded octree of Sec. 1 (cells split into eight
// octants), numbered along the Peano-Hilbert curve, with its neighbour tables and the
// stencil-slot tables of the oct tiles the hydro kernels update.
#include <cstring>
#include <vector>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include "common.cuh"

namespace amr {

constexpr int LMAX_BUILD = 20;          // 3*(l-1) key bits + level must fit 64 bits
constexpr int32_t UNNEEDED = INT32_MIN + 1;

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct TreeLayout {
    size_t lvl, ix, iy, iz, key, son, father, nbor, nb27, refmask, fused, grid, root[2], slot[2], ghost, rlist, total;
    int64_t tile_bound[2];
};

static int nslot(int depth) { const int s = (1 << depth) + 2; return s * s * s; }

static TreeLayout tree_layout(int64_t n, const int64_t cnt[AMR_MAXLEV + 2], int levelmin, int lmax)
{
    TreeLayout L;
    for (int d = 0; d < 2; ++d) {
        int64_t b = 0;
        for (int l = levelmin; l <= lmax; ++l) {
            const int r = l - (d + 1);
            if (r >= 1) b += cnt[r] < cnt[l] ? cnt[r] : cnt[l];
        }
        L.tile_bound[d] = b;
    }
    size_t o = 0;
    auto put = [&](size_t bytes) { size_t at = o; o += al256(bytes); return at; };
    L.lvl = put(4 * n); L.ix = put(4 * n); L.iy = put(4 * n); L.iz = put(4 * n);
    L.key = put(8 * n); L.son = put(32 * n); L.father = put(4 * n); L.nbor = put(24 * n);
    L.nb27 = put(108 * n); L.refmask = put(n); L.fused = put(n);
    // dense oct grid of the deepest complete level
    int lg = lmax;
    while (lg > levelmin && cnt[lg] != (int64_t(1) << (3 * (lg - 1)))) --lg;
    L.grid = put(4 * cnt[lg]);
    for (int d = 0; d < 2; ++d) {
        L.root[d] = put(4 * L.tile_bound[d]);
        L.slot[d] = put(4 * L.tile_bound[d] * nslot(d + 1));
    }
    // ghost fathers: coarse leaves of levels levelmin..lmax-1 at most
    int64_t coarse = 0;
    for (int l = levelmin; l < lmax; ++l) coarse += 8 * cnt[l];
    L.ghost = put(4 * (coarse > 0 ? coarse : 1));
    // cells of the same levels with reflux or restriction work in a step, at most all of them
    L.rlist = put(4 * (coarse > 0 ? coarse : 1));
    L.total = o;
    return L;
}

struct WsLayout { size_t lxyz, sk0, sk1, id0, id1, flag, pos, gflag, gpos, small, cub, total; size_t cub_bytes; };

static size_t cub_bytes_needed(int64_t n)
{
    size_t a = 0, b = 0, c = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, a, (uint64_t *)nullptr, (uint64_t *)nullptr, (int32_t *)nullptr,
                                    (int32_t *)nullptr, (int)n, 0, 64);
    cub::DeviceScan::ExclusiveSum(nullptr, b, (int32_t *)nullptr, (int32_t *)nullptr, (int)n);
    cub::DeviceScan::ExclusiveSum(nullptr, c, (int32_t *)nullptr, (int32_t *)nullptr, (int)(8 * n + 1));
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

static WsLayout ws_layout(int64_t n)
{
    WsLayout W;
    size_t o = 0;
    auto put = [&](size_t bytes) { size_t at = o; o += al256(bytes); return at; };
    W.lxyz = put(16 * n); W.sk0 = put(8 * n); W.sk1 = put(8 * n); W.id0 = put(4 * n); W.id1 = put(4 * n);
    W.flag = put(4 * (n + 1)); W.pos = put(4 * (n + 1));
    W.gflag = put(4 * (8 * n + 1)); W.gpos = put(4 * (8 * n + 1));   // ghost fathers, per cell
    W.small = put(2048);   // err, tile counts, level histogram, ghost offsets
    W.cub_bytes = cub_bytes_needed(n);
    W.cub = put(W.cub_bytes);
    W.total = o;
    return W;
}

static amr_status count_levels(const int32_t *h, int64_t n, int64_t cnt[AMR_MAXLEV + 2], int *lmax)
{
    for (int l = 0; l < AMR_MAXLEV + 2; ++l) cnt[l] = 0;
    *lmax = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int l = h[4 * i];
        if (l < 1 || l > LMAX_BUILD) return AMR_EINVAL;
        cnt[l]++;
        if (l > *lmax) *lmax = l;
    }
    return AMR_OK;
}

static amr_status check_geom(const amr_geom *g, int64_t n)
{
    if (!g || n <= 0 || n > (int64_t(1) << 27)) return AMR_EINVAL;   // 8*noct < 2^31 - 2
    if (g->levelmin < 2 || g->levelmin > LMAX_BUILD) return AMR_EINVAL;
    for (int f = 0; f < 6; ++f)
        if (g->bc[f] != AMR_BC_PERIODIC && g->bc[f] != AMR_BC_OUTFLOW) return AMR_EINVAL;
    for (int a = 0; a < 3; ++a)
        if ((g->bc[2 * a] == AMR_BC_PERIODIC) != (g->bc[2 * a + 1] == AMR_BC_PERIODIC)) return AMR_EINVAL;
    return AMR_OK;
}

// ---- kernels --------------------------------------------------------------------
__global__ void k_keys(const int32_t *__restrict__ lxyz, int64_t n, uint64_t *sk, int32_t *id, int32_t *err)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int l = lxyz[4 * i];
    const int32_t x = lxyz[4 * i + 1], y = lxyz[4 * i + 2], z = lxyz[4 * i + 3];
    const int64_t m = int64_t(1) << ((l >= 1 && l <= LMAX_BUILD ? l : 1) - 1);
    if (l < 1 || l > LMAX_BUILD || x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) {
        set_error(err, AMR_EINVAL);
        sk[i] = ~uint64_t(0);
    } else {
        sk[i] = (uint64_t(l) << 58) | hilbert3(l - 1, x, y, z);
    }
    id[i] = int32_t(i);
}

// octs per level of a device oct list (checked against the counts the caller gave)
__global__ void k_level_hist(const int32_t *__restrict__ lxyz, int64_t n, unsigned long long *hist)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int l = lxyz[4 * i];
    if (l >= 0 && l < AMR_MAXLEV + 2) atomicAdd(hist + l, 1ull);
}

__global__ void k_scatter(const uint64_t *__restrict__ sk, const int32_t *__restrict__ id,
                          const int32_t *__restrict__ lxyz, int64_t n, int32_t *lvl, int32_t *ix, int32_t *iy,
                          int32_t *iz, uint64_t *key, int32_t *err)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int32_t s = id[i];
    lvl[i] = lxyz[4 * s];
    ix[i] = lxyz[4 * s + 1];
    iy[i] = lxyz[4 * s + 2];
    iz[i] = lxyz[4 * s + 3];
    key[i] = sk[i] & ((uint64_t(1) << 58) - 1);
    if (i > 0 && sk[i] == sk[i - 1]) set_error(err, AMR_EINVAL);   // duplicate oct
}

struct BuildView {
    int64_t n;
    int32_t levelmin, levelmax;
    int32_t bc[6];
    int64_t lvl_off[AMR_MAXLEV + 2];
    const int32_t *lvl, *ix, *iy, *iz;
    const uint64_t *key;
};

// level-l cell (X,Y,Z) (inside the box) -> cell id, or -1 if its oct is absent
__device__ int64_t cell_of(const BuildView &b, int l, int64_t X, int64_t Y, int64_t Z)
{
    const int64_t o = find_oct(b.key, b.lvl_off, l, X >> 1, Y >> 1, Z >> 1);
    return o < 0 ? -1 : o * 8 + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1);
}

// Tables by search (son, father, nbor, nb27, refmask) for the octs [0, o1): levels 1 and 2,
// whose neighbours cannot come from a coarser oct's table (the root's has no wrap).
__global__ void k_tables(BuildView b, int64_t o1, int32_t *son, int32_t *father, int32_t *nbor, int32_t *nb27,
                         uint8_t *refmask, int32_t *err)
{
    const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o >= o1) return;
    const int l = b.lvl[o];
    const int64_t x = b.ix[o], y = b.iy[o], z = b.iz[o];
    uint32_t mask = 0;
    for (int c = 0; c < 8; ++c) {
        const int64_t s = find_oct(b.key, b.lvl_off, l + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1));
        son[8 * o + c] = int32_t(s);
        if (s >= 0) mask |= 1u << c;
    }
    refmask[o] = uint8_t(mask);
    if (l < b.levelmin && mask != 0xFFu) set_error(err, AMR_EINVAL);   // levels below levelmin have no leaves
    if (l == 1) {
        father[o] = -1;
        for (int k = 0; k < 6; ++k) nbor[6 * o + k] = -1;
        for (int k = 0; k < 27; ++k) nb27[27 * o + k] = (k == 13) ? int32_t(o) : OUTSIDE;
        return;
    }
    const int64_t f = cell_of(b, l - 1, x, y, z);
    if (f < 0) set_error(err, AMR_EINVAL);                             // oct without its father cell
    father[o] = int32_t(f);
    const int64_t nf = int64_t(1) << (l - 1);
    for (int k = 0; k < 6; ++k) {
        int64_t P[3] = {x, y, z};
        P[k >> 1] += (k & 1) ? 1 : -1;
        int out = 0;
        for (int a = 0; a < 3; ++a) out |= bc_apply(b.bc, a, nf, P[a]);
        if (out) { nbor[6 * o + k] = -1; continue; }
        const int64_t cid = cell_of(b, l - 1, P[0], P[1], P[2]);
        if (cid < 0) set_error(err, AMR_EUNBALANCED);
        nbor[6 * o + k] = int32_t(cid);
    }
    for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        int64_t P[3] = {x + dx, y + dy, z + dz};
        int out = 0;
        for (int a = 0; a < 3; ++a) out |= bc_apply(b.bc, a, nf, P[a]);
        if (out) { nb27[27 * o + k] = OUTSIDE; continue; }
        const int64_t cid = cell_of(b, l - 1, P[0], P[1], P[2]);   // 2:1 rule: must exist
        if (cid < 0) { set_error(err, AMR_EUNBALANCED); nb27[27 * o + k] = OUTSIDE; continue; }
        const int64_t s = find_oct(b.key, b.lvl_off, l, P[0], P[1], P[2]);
        nb27[27 * o + k] = s >= 0 ? int32_t(s) : int32_t(-1 - cid);
    }
}

// An oct whose eight cells are leaves and have no refined same-level face neighbour:
// its cells are final after the Godunov update (no reflux, no restriction reaches them),
// so the update kernel can also restrict its father cell.
// Every oct's father cell (one search) and, scattered from it, the son table.
__global__ void k_father_son(BuildView b, int32_t *son, int32_t *father, int32_t *err)
{
    const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o >= b.n) return;
    const int l = b.lvl[o];
    if (l == 1) {
        father[o] = -1;
        return;
    }
    const int64_t f = cell_of(b, l - 1, b.ix[o], b.iy[o], b.iz[o]);
    if (f < 0) set_error(err, AMR_EINVAL);                             // oct without its father cell
    father[o] = int32_t(f);
    if (f >= 0) son[f] = int32_t(o);
}

// Tables of the level-l octs (l >= 3) from the tables of their fathers' octs: the level-(l-1)
// cell next to an oct's father lies in the father oct or one of its 26 neighbours, and the
// level-l neighbour oct is that cell's son.  Same entries as k_tables, without searching.
__global__ void k_tables_level(BuildView b, int l, const int32_t *__restrict__ son, const int32_t *__restrict__ father,
                               int32_t *nbor, int32_t *nb27, uint8_t *refmask, int32_t *err)
{
    const int64_t o = b.lvl_off[l] + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o >= b.lvl_off[l + 1]) return;
    const int32_t x = b.ix[o], y = b.iy[o], z = b.iz[o];   // father cell coordinates (level l-1)
    uint32_t mask = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (son[8 * o + c] >= 0) mask |= 1u << c;
    refmask[o] = uint8_t(mask);
    if (l < b.levelmin && mask != 0xFFu) set_error(err, AMR_EINVAL);   // levels below levelmin have no leaves
    const int32_t f = father[o];
    if (f < 0) return;                                                 // reported by k_father_son
    const int32_t *pn = nb27 + 27 * int64_t(f >> 3);                   // the father's oct (level l-1)
    // level-(l-1) cell (X, Y, Z) next to the father: its oct among the father oct's 27
    auto cell_near = [&](int32_t X, int32_t Y, int32_t Z, int32_t &cid) -> int {
        const int k = ((X >> 1) - (x >> 1) + 1) + 3 * ((Y >> 1) - (y >> 1) + 1) + 9 * ((Z >> 1) - (z >> 1) + 1);
        const int32_t po = pn[k];
        if (po == OUTSIDE) return 1;                                   // beyond an outflow face
        if (po < 0) return 2;                                          // missing: 2:1 rule broken
        cid = po * 8 + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1);
        return 0;
    };
    for (int k = 0; k < 6; ++k) {
        int32_t P[3] = {x, y, z};
        P[k >> 1] += (k & 1) ? 1 : -1;
        int32_t cid = -1;
        const int r = cell_near(P[0], P[1], P[2], cid);
        if (r == 2) set_error(err, AMR_EUNBALANCED);
        nbor[6 * o + k] = r == 0 ? cid : -1;
    }
    for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        int32_t cid = -1;
        const int r = cell_near(x + dx, y + dy, z + dz, cid);
        if (r != 0) {
            if (r == 2) set_error(err, AMR_EUNBALANCED);
            nb27[27 * o + k] = OUTSIDE;
            continue;
        }
        const int32_t sn = son[cid];
        nb27[27 * o + k] = sn >= 0 ? sn : -1 - cid;
    }
}

__global__ void k_fused(BuildView b, const int32_t *__restrict__ son, const int32_t *__restrict__ nbor,
                        const uint8_t *__restrict__ refmask, uint8_t *fused)
{
    const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o >= b.n) return;
    uint8_t ok = b.lvl[o] >= 2 && refmask[o] == 0;
    for (int f = 0; f < 6 && ok; ++f) {
        const int32_t N = nbor[6 * o + f];
        if (N < 0) continue;
        const int32_t so = son[N];
        if (so < 0) continue;
        const int d = f >> 1, side = f & 1;
        // cells of the neighbour oct facing this oct sit at position 1 - side along d
        for (int c = 0; c < 8; ++c)
            if (((c >> d) & 1) == 1 - side && ((refmask[so] >> c) & 1)) ok = 0;
    }
    fused[o] = ok;
}

// flag octs that root a tile of the given depth: a descendant `depth` levels down
__global__ void k_tile_flags(BuildView b, const int32_t *__restrict__ son, const uint8_t *__restrict__ refmask,
                             int depth, int32_t *flag)
{
    const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o > b.n) return;
    if (o == b.n) { flag[o] = 0; return; }
    const int l = b.lvl[o] + depth;   // level the tile updates
    int f = 0;
    if (l >= b.levelmin && l <= b.levelmax) {
        if (depth == 1) {
            f = refmask[o] != 0;
        } else {
            for (int c = 0; c < 8; ++c) {
                const int32_t s = son[8 * o + c];
                if (s >= 0 && refmask[s] != 0) f = 1;
            }
        }
    }
    flag[o] = f;
}

__global__ void k_grid(int64_t o0, int64_t o1, int l, const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                       const int32_t *__restrict__ iz, int32_t *grid)
{
    const int64_t o = o0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o >= o1) return;
    const int64_t M = int64_t(1) << (l - 1);
    const int64_t x = ix[o], y = iy[o], z = iz[o];
    if (x < 0 || y < 0 || z < 0 || x >= M || y >= M || z >= M) return;   // invalid input: reported by k_keys
    grid[x + M * (y + M * z)] = int32_t(o);
}

__global__ void k_tile_compact(int64_t n, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                               int32_t *root)
{
    const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o < n && flag[o]) root[pos[o]] = int32_t(o);
}

// tiles updating level l are the compacted roots at level l - depth:
// [pos[lvl_off[l - depth]], pos[lvl_off[l - depth + 1]])
__global__ void k_tile_counts(BuildView b, const int32_t *__restrict__ pos, int depth, int64_t *out)
{
    const int l = threadIdx.x;
    if (l >= AMR_MAXLEV + 2) return;
    const int r = l - depth < 0 ? 0 : l - depth;
    const int64_t at = b.lvl_off[r] < b.n ? b.lvl_off[r] : b.n;
    out[l] = pos[at];
}

// Stencil slots of each tile: a depth-D tile covers 2^D x 2^D x 2^D level-l octs and
// its stencil (2^D + 2)^3 oct positions, one layer of octs (two cells) around it; the
// eight corner positions are marked unneeded.
__global__ void k_tile_slots(BuildView b, int depth, int64_t ntile, const int32_t *__restrict__ root,
                             const int32_t *__restrict__ son, int32_t *slot)
{
    const int ns = (1 << depth) + 2, nsl = ns * ns * ns;
    const int64_t gi = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (gi >= ntile * nsl) return;
    const int64_t t = gi / nsl;
    const int s = int(gi % nsl);
    const int32_t r = root[t];
    const int l = b.lvl[r] + depth;
    const int sx = s % ns, sy = (s / ns) % ns, sz = s / (ns * ns);
    // the eight corner slots: the update reads none of their cells (its faces need the
    // predicted states of face neighbours only), so they get no ghost father either
    if (int(sx == 0 || sx == ns - 1) + int(sy == 0 || sy == ns - 1) + int(sz == 0 || sz == ns - 1) == 3) {
        slot[gi] = UNNEEDED;
        return;
    }
    // level-l oct coordinates == level-(l-1) father cell coordinates
    int64_t P[3] = {int64_t(b.ix[r]) * (1 << depth) - 1 + sx, int64_t(b.iy[r]) * (1 << depth) - 1 + sy,
                    int64_t(b.iz[r]) * (1 << depth) - 1 + sz};
    const int64_t nf = int64_t(1) << (l - 1);
    int out = 0;
    for (int a = 0; a < 3; ++a) out |= bc_apply(b.bc, a, nf, P[a]);
    int32_t v;
    if (out) {
        v = OUTSIDE;
    } else {
        const int64_t F = cell_of(b, l - 1, P[0], P[1], P[2]);
        if (F < 0) v = UNNEEDED;                    // no updated oct of the tile reaches it (2:1 rule)
        else v = son[F] >= 0 ? son[F] : int32_t(-1 - F);
    }
    slot[gi] = v;
}

// Ghost fathers: every coarse leaf a tile slot interpolates from gets one index, in cell
// order; the slots are rewritten to refer to that index.
__global__ void k_ghost_mark(int64_t nslots, const int32_t *__restrict__ slot, int32_t *gflag)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= nslots) return;
    const int32_t v = slot[i];
    if (v < 0 && v != OUTSIDE && v != UNNEEDED) gflag[-1 - int64_t(v)] = 1;
}

__global__ void k_ghost_compact(int64_t ncell, const int32_t *__restrict__ gflag, const int32_t *__restrict__ gpos,
                                int32_t *ghost_cell)
{
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c < ncell && gflag[c]) ghost_cell[gpos[c]] = int32_t(c);
}

__global__ void k_ghost_rewrite(int64_t nslots, const int32_t *__restrict__ gpos, int32_t *slot)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= nslots) return;
    const int32_t v = slot[i];
    if (v < 0 && v != OUTSIDE && v != UNNEEDED) slot[i] = -1 - gpos[-1 - int64_t(v)];
}

__global__ void k_ghost_bounds(BuildView b, const int32_t *__restrict__ gpos, int64_t *out)
{
    const int l = threadIdx.x;
    if (l < AMR_MAXLEV + 2) out[l] = gpos[b.lvl_off[l] * 8];
}

// Cells of levels levelmin .. levelmax-1 that the step's reflux pass (not restricting
// everything) has work for: a refined cell whose child oct is not restricted inside the
// update kernel, or a leaf with a refined face neighbour (the same tests as the pass).
__global__ void k_reflux_flag(BuildView b, const int32_t *__restrict__ son, const int32_t *__restrict__ nbor,
                              const uint8_t *__restrict__ fused, int32_t *flag)
{
    const int64_t c0 = b.lvl_off[b.levelmin] * 8, c1 = b.lvl_off[b.levelmax] * 8;
    const int64_t cell = c0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (cell >= c1) return;
    const int32_t s = son[cell];
    int32_t need = 0;
    if (s >= 0) {
        need = !fused[s];
    } else {
        const int64_t o = cell >> 3;
        const int c = int(cell & 7);
        for (int f = 0; f < 6 && !need; ++f) {
            const int d = f >> 1, side = f & 1;
            int64_t nb;
            if (((c >> d) & 1) != side) {
                nb = o * 8 + (c ^ (1 << d));
            } else {
                const int32_t N = nbor[6 * o + f];
                if (N < 0) continue;
                const int32_t so = son[N];
                if (so < 0) continue;
                nb = int64_t(so) * 8 + (c ^ (1 << d));
            }
            need = son[nb] >= 0;
        }
    }
    flag[cell] = need;
}

__global__ void k_reflux_compact(int64_t c0, int64_t c1, const int32_t *__restrict__ flag,
                                 const int32_t *__restrict__ pos, int32_t *list)
{
    const int64_t c = c0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c < c1 && flag[c]) list[pos[c]] = int32_t(c);
}

// ---- batch mode: independent uniform boxes -------------------------------------------
struct BoxLayout {
    size_t lvl, ix, iy, iz, refmask, fused, inst_n, inst_dx, inst_oct_off, col_off, root[2], slot[2], tinst[2], total;
    int64_t noct, ntile[2];
};

static amr_status box_counts(const amr_geom *g, int64_t *noct, int64_t ntile[2])
{
    if (!g->h_inst_n || g->n_inst <= 0 || g->n_inst > (1 << 20)) return AMR_EINVAL;
    int64_t n = 0, t1 = 0, t2 = 0;
    bool d2 = true;
    for (int i = 0; i < g->n_inst; ++i) {
        const int64_t N = g->h_inst_n[i];
        if (N < 4 || N % 4 || N > (1 << 16)) return AMR_EINVAL;
        n += (N / 2) * (N / 2) * (N / 2);
        t1 += (N / 4) * (N / 4) * (N / 4);
        if (N % 8) d2 = false; else t2 += (N / 8) * (N / 8) * (N / 8);
    }
    if (n > (int64_t(1) << 27)) return AMR_EINVAL;
    *noct = n;
    ntile[0] = t1;
    ntile[1] = d2 ? t2 : 0;
    return AMR_OK;
}

static BoxLayout box_layout(const amr_geom *g, int64_t n, const int64_t nt[2])
{
    BoxLayout L;
    L.noct = n; L.ntile[0] = nt[0]; L.ntile[1] = nt[1];
    size_t o = 0;
    auto put = [&](size_t bytes) { size_t at = o; o += al256(bytes); return at; };
    L.lvl = put(4 * n); L.ix = put(4 * n); L.iy = put(4 * n); L.iz = put(4 * n);
    L.refmask = put(n); L.fused = put(n);
    L.inst_n = put(4 * size_t(g->n_inst)); L.inst_dx = put(8 * size_t(g->n_inst));
    L.inst_oct_off = put(8 * (size_t(g->n_inst) + 1));
    L.col_off = put(8 * (size_t(g->n_inst) + 1));
    for (int d = 0; d < 2; ++d) {
        L.root[d] = put(4 * nt[d]);
        L.slot[d] = put(4 * nt[d] * nslot(d + 1));
        L.tinst[d] = put(4 * nt[d]);
    }
    L.total = o;
    return L;
}

__device__ __forceinline__ int find_box(const int64_t *off, int n_inst, int64_t i)
{
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_box_octs(int n_inst, const int64_t *__restrict__ off, const int32_t *__restrict__ N, int64_t n,
                           int32_t *lvl, int32_t *ix, int32_t *iy, int32_t *iz, uint8_t *refmask, uint8_t *fused)
{
    const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (o >= n) return;
    const int b = find_box(off, n_inst, o);
    const int64_t M = N[b] / 2, j = o - off[b];
    lvl[o] = b;
    ix[o] = int32_t(j % M);
    iy[o] = int32_t((j / M) % M);
    iz[o] = int32_t(j / (M * M));
    refmask[o] = 0;
    fused[o] = 0;
}

// tiles of depth d: 2^d octs per axis; tile_off[b] = first tile of box b
__global__ void k_box_tiles(int n_inst, const int64_t *__restrict__ toff, const int64_t *__restrict__ ooff,
                            const int32_t *__restrict__ N, int depth, int64_t ntile, const int32_t *bc,
                            int32_t *root, int32_t *tinst, int32_t *slot)
{
    const int ns = (1 << depth) + 2, nsl = ns * ns * ns;
    const int64_t gi = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (gi >= ntile * nsl) return;
    const int64_t t = gi / nsl;
    const int s = int(gi % nsl);
    const int b = find_box(toff, n_inst, t);
    const int64_t M = N[b] / 2, T = M >> depth, j = t - toff[b];
    const int64_t c[3] = {(j % T) << depth, ((j / T) % T) << depth, (j / (T * T)) << depth};
    if (s == 0) {
        root[t] = int32_t(ooff[b] + c[0] + M * (c[1] + M * c[2]));
        tinst[t] = b;
    }
    int64_t P[3] = {c[0] - 1 + s % ns, c[1] - 1 + (s / ns) % ns, c[2] - 1 + s / (ns * ns)};
    int out = 0;
    for (int a = 0; a < 3; ++a) out |= bc_apply(bc, a, M, P[a]);
    slot[gi] = out ? OUTSIDE : int32_t(ooff[b] + P[0] + M * (P[1] + M * P[2]));
}

static amr_status build_boxes(const amr_geom *g, void *d_tree_mem, size_t tree_bytes, void *d_ws, size_t ws_bytes,
                              amr_tree *out, cudaStream_t st)
{
    int64_t n, nt[2];
    if (box_counts(g, &n, nt) != AMR_OK) return AMR_EINVAL;
    const BoxLayout L = box_layout(g, n, nt);
    const size_t wsz = al256(8 * (size_t(g->n_inst) + 1)) * 3 + 256;
    if (tree_bytes < L.total || ws_bytes < wsz) return AMR_ECAPACITY;
    char *T = static_cast<char *>(d_tree_mem), *S = static_cast<char *>(d_ws);
    std::memset(out, 0, sizeof(*out));
    out->noct = n;
    for (int f = 0; f < 6; ++f) out->bc[f] = g->bc[f];
    for (int l = 1; l < AMR_MAXLEV + 2; ++l) out->lvl_off[l] = n;
    out->reg_base = n;
    out->lvl = (int32_t *)(T + L.lvl); out->ix = (int32_t *)(T + L.ix); out->iy = (int32_t *)(T + L.iy);
    out->iz = (int32_t *)(T + L.iz); out->refmask = (uint8_t *)(T + L.refmask); out->fused = (uint8_t *)(T + L.fused);
    out->n_inst = g->n_inst;
    out->inst_n = (int32_t *)(T + L.inst_n);
    out->inst_dx = (double *)(T + L.inst_dx);
    out->inst_oct_off = (int64_t *)(T + L.inst_oct_off);
    std::vector<int64_t> ooff(g->n_inst + 1), toff[2], coff(g->n_inst + 1);
    std::vector<double> dx(g->n_inst);
    bool col_ok = true;
    coff[0] = 0;
    toff[0].resize(g->n_inst + 1); toff[1].resize(g->n_inst + 1);
    ooff[0] = toff[0][0] = toff[1][0] = 0;
    for (int i = 0; i < g->n_inst; ++i) {
        const int64_t N = g->h_inst_n[i];
        ooff[i + 1] = ooff[i] + (N / 2) * (N / 2) * (N / 2);
        toff[0][i + 1] = toff[0][i] + (N / 4) * (N / 4) * (N / 4);
        toff[1][i + 1] = toff[1][i] + (nt[1] ? (N / 8) * (N / 8) * (N / 8) : 0);
        dx[i] = 1.0 / double(N);
        if (N % 16) col_ok = false;
        coff[i + 1] = coff[i] + (N / 8) * (N / 8) * (N / 16);   // 8x8 footprints x 16-cell segments
    }
    out->inst_col_off = (int64_t *)(T + L.col_off);
    out->col_work = col_ok ? coff[g->n_inst] : 0;
    AMR_CUDA_TRY(cudaMemcpyAsync(out->inst_col_off, coff.data(), 8 * coff.size(), cudaMemcpyHostToDevice, st));
    int64_t *t0 = (int64_t *)S, *t1 = (int64_t *)(S + al256(8 * (size_t(g->n_inst) + 1)));
    int32_t *dbc = (int32_t *)(S + 2 * al256(8 * (size_t(g->n_inst) + 1)));
    AMR_CUDA_TRY(cudaMemcpyAsync(out->inst_n, g->h_inst_n, 4 * size_t(g->n_inst), cudaMemcpyHostToDevice, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(out->inst_dx, dx.data(), 8 * size_t(g->n_inst), cudaMemcpyHostToDevice, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(out->inst_oct_off, ooff.data(), 8 * ooff.size(), cudaMemcpyHostToDevice, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(t0, toff[0].data(), 8 * toff[0].size(), cudaMemcpyHostToDevice, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(t1, toff[1].data(), 8 * toff[1].size(), cudaMemcpyHostToDevice, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(dbc, g->bc, 6 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int TB = 256;
    k_box_octs<<<unsigned((n + TB - 1) / TB), TB, 0, st>>>(g->n_inst, out->inst_oct_off, out->inst_n, n, out->lvl,
                                                           out->ix, out->iy, out->iz, out->refmask, out->fused);
    for (int d = 0; d < 2; ++d) {
        out->tile_root[d] = (int32_t *)(T + L.root[d]);
        out->tile_slot[d] = (int32_t *)(T + L.slot[d]);
        out->tile_inst[d] = (int32_t *)(T + L.tinst[d]);
        out->tile_off[d][0] = 0;
        for (int l = 1; l < AMR_MAXLEV + 2; ++l) out->tile_off[d][l] = nt[d];
        if (nt[d] > 0) {
            const int64_t tot = nt[d] * nslot(d + 1);
            k_box_tiles<<<unsigned((tot + TB - 1) / TB), TB, 0, st>>>(g->n_inst, d == 0 ? t0 : t1, out->inst_oct_off,
                                                                     out->inst_n, d + 1, nt[d], dbc,
                                                                     out->tile_root[d], out->tile_inst[d],
                                                                     out->tile_slot[d]);
        }
    }
    AMR_CUDA_TRY(cudaStreamSynchronize(st));
    AMR_CUDA_TRY(cudaGetLastError());
    return AMR_OK;
}

}  // namespace amr

using namespace amr;

extern "C" amr_status amr_build_octree_query(const amr_geom *geom, const int32_t *h_oct_lxyz, int64_t n_oct,
                                             size_t *tree_bytes, size_t *workspace_bytes)
{
    if (geom && geom->n_inst > 0) {
        if (!tree_bytes || !workspace_bytes) return AMR_EINVAL;
        for (int f = 0; f < 6; ++f)
            if (geom->bc[f] != AMR_BC_PERIODIC && geom->bc[f] != AMR_BC_OUTFLOW) return AMR_EINVAL;
        int64_t n, nt[2];
        if (box_counts(geom, &n, nt) != AMR_OK) return AMR_EINVAL;
        *tree_bytes = box_layout(geom, n, nt).total;
        *workspace_bytes = al256(8 * (size_t(geom->n_inst) + 1)) * 3 + 256;
        return AMR_OK;
    }
    if (check_geom(geom, n_oct) != AMR_OK || !h_oct_lxyz || !tree_bytes || !workspace_bytes) return AMR_EINVAL;
    int64_t cnt[AMR_MAXLEV + 2];
    int lmax;
    if (count_levels(h_oct_lxyz, n_oct, cnt, &lmax) != AMR_OK) return AMR_EINVAL;
    *tree_bytes = tree_layout(n_oct, cnt, geom->levelmin, lmax).total;
    *workspace_bytes = ws_layout(n_oct).total;
    return AMR_OK;
}

// The octree from an oct list in host memory (h_lxyz) or device memory (d_lxyz), with its
// per-level counts already known.
static amr_status build_tree(const amr_geom *geom, const int32_t *h_lxyz, const int32_t *d_lxyz, int64_t n,
                             const int64_t cnt[AMR_MAXLEV + 2], int lmax, void *d_tree_mem, size_t tree_bytes,
                             void *d_workspace, size_t workspace_bytes, amr_tree *out, cudaStream_t st)
{
    const int lmin = geom->levelmin;
    if (lmax < lmin) return AMR_EINVAL;
    for (int l = 1; l <= lmin; ++l)
        if (cnt[l] != (int64_t(1) << (3 * (l - 1)))) return AMR_EINVAL;   // levels 1..levelmin complete
    const TreeLayout L = tree_layout(n, cnt, lmin, lmax);
    const WsLayout W = ws_layout(n);
    if (tree_bytes < L.total || workspace_bytes < W.total) return AMR_ECAPACITY;
    char *T = static_cast<char *>(d_tree_mem), *S = static_cast<char *>(d_workspace);

    std::memset(out, 0, sizeof(*out));
    out->noct = n;
    out->levelmin = lmin;
    out->levelmax = lmax;
    for (int f = 0; f < 6; ++f) out->bc[f] = geom->bc[f];
    int64_t acc = 0;
    for (int l = 0; l < AMR_MAXLEV + 2; ++l) { out->lvl_off[l] = acc; acc += (l <= AMR_MAXLEV) ? cnt[l] : 0; }
    out->lvl_off[AMR_MAXLEV + 1] = n;
    out->reg_base = out->lvl_off[lmin + 1];
    out->lvl = (int32_t *)(T + L.lvl); out->ix = (int32_t *)(T + L.ix); out->iy = (int32_t *)(T + L.iy);
    out->iz = (int32_t *)(T + L.iz); out->key = (uint64_t *)(T + L.key); out->son = (int32_t *)(T + L.son);
    out->father = (int32_t *)(T + L.father); out->nbor = (int32_t *)(T + L.nbor);
    out->nb27 = (int32_t *)(T + L.nb27); out->refmask = (uint8_t *)(T + L.refmask);
    out->fused = (uint8_t *)(T + L.fused);
    for (int d = 0; d < 2; ++d) {
        out->tile_root[d] = (int32_t *)(T + L.root[d]);
        out->tile_slot[d] = (int32_t *)(T + L.slot[d]);
    }
    const int32_t *lxyz = d_lxyz ? d_lxyz : (const int32_t *)(S + W.lxyz);
    uint64_t *sk0 = (uint64_t *)(S + W.sk0), *sk1 = (uint64_t *)(S + W.sk1);
    int32_t *id0 = (int32_t *)(S + W.id0), *id1 = (int32_t *)(S + W.id1);
    int32_t *flag = (int32_t *)(S + W.flag), *pos = (int32_t *)(S + W.pos);
    int32_t *err = (int32_t *)(S + W.small);
    int64_t *tcnt = (int64_t *)(S + W.small + 256);
    void *cubtmp = S + W.cub;

    const int TB = 256;
    const unsigned nb = unsigned((n + TB - 1) / TB), nb1 = unsigned((n + TB) / TB);
    if (h_lxyz)
        AMR_CUDA_TRY(cudaMemcpyAsync(S + W.lxyz, h_lxyz, 16 * size_t(n), cudaMemcpyHostToDevice, st));
    AMR_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    if (d_lxyz) {
        // the caller's per-level counts must describe the list (they size the layout)
        unsigned long long *hist = (unsigned long long *)(S + W.small + 1024);
        unsigned long long hh[AMR_MAXLEV + 2];
        AMR_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(hh), st));
        k_level_hist<<<nb, TB, 0, st>>>(lxyz, n, hist);
        AMR_CUDA_TRY(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, st));
        AMR_CUDA_TRY(cudaStreamSynchronize(st));
        for (int l = 0; l < AMR_MAXLEV + 2; ++l)
            if (int64_t(hh[l]) != (l <= AMR_MAXLEV ? cnt[l] : 0)) return AMR_EINVAL;
    }
    k_keys<<<nb, TB, 0, st>>>(lxyz, n, sk0, id0, err);
    size_t cb = W.cub_bytes;
    AMR_CUDA_TRY(cub::DeviceRadixSort::SortPairs(cubtmp, cb, sk0, sk1, id0, id1, (int)n, 0, 64, st));
    k_scatter<<<nb, TB, 0, st>>>(sk1, id1, lxyz, n, out->lvl, out->ix, out->iy, out->iz, out->key, err);

    BuildView bv;
    bv.n = n; bv.levelmin = lmin; bv.levelmax = lmax;
    for (int f = 0; f < 6; ++f) bv.bc[f] = geom->bc[f];
    for (int l = 0; l < AMR_MAXLEV + 2; ++l) bv.lvl_off[l] = out->lvl_off[l];
    bv.lvl = out->lvl; bv.ix = out->ix; bv.iy = out->iy; bv.iz = out->iz; bv.key = out->key;
    // son and father for every oct, the other tables of levels 1-2 by search, then level by
    // level from the coarser tables
    AMR_CUDA_TRY(cudaMemsetAsync(out->son, 0xFF, 32 * size_t(n), st));
    k_father_son<<<nb, TB, 0, st>>>(bv, out->son, out->father, err);
    {
        const int64_t o12 = out->lvl_off[3 <= AMR_MAXLEV + 1 ? 3 : AMR_MAXLEV + 1];
        if (o12 > 0)
            k_tables<<<unsigned((o12 + TB - 1) / TB), TB, 0, st>>>(bv, o12, out->son, out->father, out->nbor,
                                                                    out->nb27, out->refmask, err);
        for (int l = 3; l <= lmax; ++l) {
            const int64_t nl = out->lvl_off[l + 1] - out->lvl_off[l];
            if (nl > 0)
                k_tables_level<<<unsigned((nl + TB - 1) / TB), TB, 0, st>>>(bv, l, out->son, out->father, out->nbor,
                                                                         out->nb27, out->refmask, err);
        }
    }
    k_fused<<<nb, TB, 0, st>>>(bv, out->son, out->nbor, out->refmask, out->fused);
    {
        // the deepest complete level (levelmin at least): its oct grid for the z-column kernel
        int lg = lmax;
        while (lg > lmin && cnt[lg] != (int64_t(1) << (3 * (lg - 1)))) --lg;
        out->grid_level = lg;
        out->grid = (int32_t *)(T + L.grid);
        const int64_t nl = cnt[lg];
        k_grid<<<unsigned((nl + TB - 1) / TB), TB, 0, st>>>(out->lvl_off[lg], out->lvl_off[lg + 1], lg, out->ix,
                                                            out->iy, out->iz, out->grid);
    }

    for (int d = 0; d < 2; ++d) {
        const int depth = d + 1;
        k_tile_flags<<<nb1, TB, 0, st>>>(bv, out->son, out->refmask, depth, flag);
        cb = W.cub_bytes;
        AMR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(cubtmp, cb, flag, pos, (int)(n + 1), st));
        k_tile_compact<<<nb, TB, 0, st>>>(n, flag, pos, out->tile_root[d]);
        k_tile_counts<<<1, 32, 0, st>>>(bv, pos, depth, tcnt + d * 32);
    }
    int64_t hc[64];
    int32_t herr = 0;
    AMR_CUDA_TRY(cudaMemcpyAsync(hc, tcnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    AMR_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    AMR_CUDA_TRY(cudaStreamSynchronize(st));
    AMR_CUDA_TRY(cudaGetLastError());
    if (herr != 0) return amr_status(herr);
    for (int d = 0; d < 2; ++d) {
        for (int l = 0; l < AMR_MAXLEV + 2; ++l) out->tile_off[d][l] = hc[d * 32 + l];
        const int64_t ntile = out->tile_off[d][AMR_MAXLEV + 1];
        if (ntile > L.tile_bound[d]) return AMR_ECAPACITY;
        if (ntile > 0) {
            const int64_t tot = ntile * nslot(d + 1);
            k_tile_slots<<<unsigned((tot + TB - 1) / TB), TB, 0, st>>>(bv, d + 1, ntile, out->tile_root[d], out->son,
                                                                      out->tile_slot[d]);
        }
    }
    // the reflux pass's work list: per level, in cell order
    out->reflux_cell = (int32_t *)(T + L.rlist);
    for (int l = 0; l < AMR_MAXLEV + 2; ++l) out->reflux_off[l] = 0;
    if (lmax > lmin) {
        const int64_t ncell = 8 * n;
        int32_t *rflag = (int32_t *)(S + W.gflag), *rpos = (int32_t *)(S + W.gpos);
        int64_t *roff = (int64_t *)(S + W.small + 1280);
        AMR_CUDA_TRY(cudaMemsetAsync(rflag, 0, 4 * size_t(ncell + 1), st));
        const int64_t c0 = out->lvl_off[lmin] * 8, c1 = out->lvl_off[lmax] * 8;
        k_reflux_flag<<<unsigned((c1 - c0 + TB - 1) / TB), TB, 0, st>>>(bv, out->son, out->nbor, out->fused, rflag);
        cb = W.cub_bytes;
        AMR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(cubtmp, cb, rflag, rpos, (int)(ncell + 1), st));
        k_reflux_compact<<<unsigned((c1 - c0 + TB - 1) / TB), TB, 0, st>>>(c0, c1, rflag, rpos, out->reflux_cell);
        k_ghost_bounds<<<1, 32, 0, st>>>(bv, rpos, roff);
        AMR_CUDA_TRY(cudaMemcpyAsync(out->reflux_off, roff, sizeof(out->reflux_off), cudaMemcpyDeviceToHost, st));
        AMR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // ghost fathers: one index per coarse leaf the tiles interpolate from, in cell order
    {
        const int64_t ncell = 8 * n;
        int32_t *gflag = (int32_t *)(S + W.gflag), *gpos = (int32_t *)(S + W.gpos);
        int64_t *goff = (int64_t *)(S + W.small + 1280);
        out->ghost_cell = (int32_t *)(T + L.ghost);
        AMR_CUDA_TRY(cudaMemsetAsync(gflag, 0, 4 * size_t(ncell + 1), st));
        for (int d = 0; d < 2; ++d) {
            const int64_t ns = out->tile_off[d][AMR_MAXLEV + 1] * nslot(d + 1);
            if (ns > 0) k_ghost_mark<<<unsigned((ns + TB - 1) / TB), TB, 0, st>>>(ns, out->tile_slot[d], gflag);
        }
        cb = W.cub_bytes;
        AMR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(cubtmp, cb, gflag, gpos, (int)(ncell + 1), st));
        k_ghost_compact<<<unsigned((ncell + TB - 1) / TB), TB, 0, st>>>(ncell, gflag, gpos, out->ghost_cell);
        for (int d = 0; d < 2; ++d) {
            const int64_t ns = out->tile_off[d][AMR_MAXLEV + 1] * nslot(d + 1);
            if (ns > 0) k_ghost_rewrite<<<unsigned((ns + TB - 1) / TB), TB, 0, st>>>(ns, gpos, out->tile_slot[d]);
        }
        k_ghost_bounds<<<1, 32, 0, st>>>(bv, gpos, goff);
        AMR_CUDA_TRY(cudaMemcpyAsync(out->ghost_off, goff, sizeof(out->ghost_off), cudaMemcpyDeviceToHost, st));
    }
    AMR_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
    AMR_CUDA_TRY(cudaStreamSynchronize(st));
    AMR_CUDA_TRY(cudaGetLastError());
    if (herr != 0) return amr_status(herr);
    out->n_ghost = out->ghost_off[AMR_MAXLEV + 1];
    int64_t coarse = 0;
    for (int l = lmin; l < lmax; ++l) coarse += 8 * cnt[l];
    if (out->n_ghost > (coarse > 0 ? coarse : 1)) return AMR_ECAPACITY;   // cannot happen for a valid tree
    return AMR_OK;
}

extern "C" amr_status amr_build_octree(const amr_geom *geom, const int32_t *h_oct_lxyz, int64_t n,
                                       void *d_tree_mem, size_t tree_bytes, void *d_workspace,
                                       size_t workspace_bytes, amr_tree *out, amr_stream stream)
{
    if (geom && geom->n_inst > 0) {
        if (!d_tree_mem || !d_workspace || !out) return AMR_EINVAL;
        for (int f = 0; f < 6; ++f)
            if (geom->bc[f] != AMR_BC_PERIODIC && geom->bc[f] != AMR_BC_OUTFLOW) return AMR_EINVAL;
        for (int a = 0; a < 3; ++a)
            if ((geom->bc[2 * a] == AMR_BC_PERIODIC) != (geom->bc[2 * a + 1] == AMR_BC_PERIODIC)) return AMR_EINVAL;
        if ((uintptr_t(d_tree_mem) & 255) || (uintptr_t(d_workspace) & 255)) return AMR_EINVAL;
        return build_boxes(geom, d_tree_mem, tree_bytes, d_workspace, workspace_bytes, out,
                           reinterpret_cast<cudaStream_t>(stream));
    }
    if (check_geom(geom, n) != AMR_OK || !h_oct_lxyz || !d_tree_mem || !d_workspace || !out) return AMR_EINVAL;
    if ((uintptr_t(d_tree_mem) & 255) || (uintptr_t(d_workspace) & 255)) return AMR_EINVAL;
    int64_t cnt[AMR_MAXLEV + 2];
    int lmax;
    if (count_levels(h_oct_lxyz, n, cnt, &lmax) != AMR_OK) return AMR_EINVAL;
    return build_tree(geom, h_oct_lxyz, nullptr, n, cnt, lmax, d_tree_mem, tree_bytes, d_workspace, workspace_bytes,
                      out, reinterpret_cast<cudaStream_t>(stream));
}

static amr_status device_counts(const amr_geom *geom, const int64_t *h_level_counts, int64_t cnt[AMR_MAXLEV + 2],
                                int64_t *n, int *lmax)
{
    if (!geom || geom->n_inst != 0 || !h_level_counts) return AMR_EINVAL;
    *n = 0;
    *lmax = 0;
    for (int l = 0; l < AMR_MAXLEV + 2; ++l) {
        cnt[l] = l <= AMR_MAXLEV ? h_level_counts[l] : 0;
        if (cnt[l] < 0 || (cnt[l] > 0 && (l < 1 || l > LMAX_BUILD))) return AMR_EINVAL;
        if (cnt[l] > 0) *lmax = l;
        *n += cnt[l];
    }
    return check_geom(geom, *n);
}

extern "C" amr_status amr_build_octree_device_query(const amr_geom *geom, const int64_t *h_level_counts,
                                                    size_t *tree_bytes, size_t *workspace_bytes)
{
    int64_t cnt[AMR_MAXLEV + 2], n;
    int lmax;
    if (!tree_bytes || !workspace_bytes || device_counts(geom, h_level_counts, cnt, &n, &lmax) != AMR_OK)
        return AMR_EINVAL;
    if (lmax < geom->levelmin) return AMR_EINVAL;
    *tree_bytes = tree_layout(n, cnt, geom->levelmin, lmax).total;
    *workspace_bytes = ws_layout(n).total;
    return AMR_OK;
}

extern "C" amr_status amr_build_octree_device(const amr_geom *geom, const int32_t *d_oct_lxyz,
                                              const int64_t *h_level_counts, void *d_tree_mem, size_t tree_bytes,
                                              void *d_workspace, size_t workspace_bytes, amr_tree *out,
                                              amr_stream stream)
{
    int64_t cnt[AMR_MAXLEV + 2], n;
    int lmax;
    if (device_counts(geom, h_level_counts, cnt, &n, &lmax) != AMR_OK) return AMR_EINVAL;
    if (!d_oct_lxyz || !d_tree_mem || !d_workspace || !out) return AMR_EINVAL;
    if ((uintptr_t(d_tree_mem) & 255) || (uintptr_t(d_workspace) & 255)) return AMR_EINVAL;
    return build_tree(geom, nullptr, d_oct_lxyz, n, cnt, lmax, d_tree_mem, tree_bytes, d_workspace, workspace_bytes,
                      out, reinterpret_cast<cudaStream_t>(stream));
}
