// Poisson solve of Sec. 2.3: preconditioned pipelined CG (Ghysels & Vanroose 2014,
// Algorithm 4) with the 7-point incomplete-Poisson preconditioner (13/12, 1/6) and the
// convergence measure of Eq. 3.  FP64 throughout.
//
// One iteration is one kernel.  A thread block owns a 32 x TY column of cells and marches
// up a segment of z planes, keeping rings of w planes (with a two-cell in-plane halo) and
// of m = M^-1 w planes (one-cell halo) in shared memory, so that m_i = M^-1 w_i and
// n_i = A m_i never touch HBM.  Each cell then runs the eight recurrences of the
// iteration (z, q, s, p with beta_i; x, r, u, w with alpha_i) and adds its share of
// gamma_{i+1} = r_{i+1} . u_{i+1} and delta_{i+1} = w_{i+1} . u_{i+1}.  The last block to
// finish reduces the per-block partials in a fixed order (so results do not depend on
// scheduling) and computes eps_{i+1}, beta_{i+1}, alpha_{i+1} for the next launch: the
// kernel boundary is the iteration's single global synchronisation, the role the
// all-reduce plays in the distributed algorithm.  w is double-buffered because
// neighbouring blocks read its halo; every other vector is read and written only at the
// thread's own cell.
//
// The solver applies 6 M^-1 (centre 6.5, neighbours 1), one FP64 instruction per
// application fewer than the 13/12, 1/6 stencil.  Scaling the preconditioner by c > 0
// leaves x_i and eps_i unchanged in exact arithmetic (u, w, gamma scale by c; m, q, n, z,
// delta by c^2; alpha by 1/c; beta not at all), and FP64 arithmetic is the bound of the
// iteration kernel on this GPU.
//
// Without a preconditioner (M^-1 = I) the recurrences give m = w, q = s and u = r
// exactly, so that variant keeps r, s, w, z, p only and applies A to w directly.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ppcg.h"

namespace {

constexpr int TX = 32;            // tile width (one warp per tile row)
constexpr int INIT_THREADS = 256;
constexpr int INIT_BLOCKS = 1216; // 152 SMs x 8
constexpr int MIN_SEG = 4;

struct PState {
    double gamma0, gamma, alpha, beta, tol, eps;
    int32_t it, max_iter, done, status;
    uint32_t count;               // blocks of the current launch that have finished
    int32_t pad[3];
};
static_assert(sizeof(PState) == 80, "state layout");

struct Dims {
    int nx, ny, nz;
    int64_t sy, sz, n;
};

struct Vecs {
    double *r, *u, *w0, *w1, *z, *q, *s, *p;
};

struct Work {
    PState *st;
    double *part;
    int64_t part_cap;
    Vecs v;
};

constexpr int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

int64_t part_capacity(int nx, int ny, int nz)
{
    int64_t cols = (int64_t)((nx + TX - 1) / TX) * ((ny + 7) / 8);
    return cols * ((nz + MIN_SEG - 1) / MIN_SEG) + INIT_BLOCKS;
}

size_t work_bytes(int nx, int ny, int nz)
{
    int64_t n = (int64_t)nx * ny * nz;
    return (size_t)(align256(sizeof(PState)) + align256(2 * part_capacity(nx, ny, nz) * 8) + 8 * align256(n * 8));
}

Work carve(void *base, int nx, int ny, int nz)
{
    int64_t n = (int64_t)nx * ny * nz;
    char *p = (char *)base;
    Work w;
    w.st = (PState *)p;
    p += align256(sizeof(PState));
    w.part_cap = part_capacity(nx, ny, nz);
    w.part = (double *)p;
    p += align256(2 * w.part_cap * 8);
    double **v[8] = {&w.v.r, &w.v.u, &w.v.w0, &w.v.w1, &w.v.z, &w.v.q, &w.v.s, &w.v.p};
    for (int i = 0; i < 8; i++) {
        *v[i] = (double *)p;
        p += align256(n * 8);
    }
    return w;
}

__device__ __forceinline__ double nb_sum(const double *__restrict__ v, const Dims &d, int i, int j, int k, int64_t c)
{
    double s = 0.0;
    if (i > 0) s += v[c - 1];
    if (i < d.nx - 1) s += v[c + 1];
    if (j > 0) s += v[c - d.sy];
    if (j < d.ny - 1) s += v[c + d.sy];
    if (k > 0) s += v[c - d.sz];
    if (k < d.nz - 1) s += v[c + d.sz];
    return s;
}

__device__ __forceinline__ void cell_of(const Dims &d, int64_t c, int &i, int &j, int &k)
{
    int64_t t = c / d.nx;
    i = (int)(c - t * d.nx);
    j = (int)(t % d.ny);
    k = (int)(t / d.ny);
}

// y = A x (op 0) or M^-1 x (op 1)
__global__ void k_apply(Dims d, int op, const double *__restrict__ x, double *__restrict__ y)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d.n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(d, c, i, j, k);
        double s = nb_sum(x, d, i, j, k, c);
        y[c] = op == POISSON_OP_A ? fma(6.0, x[c], -s) : fma(s, 1.0 / 6.0, (13.0 / 12.0) * x[c]);
    }
}

// r = b - A x
__global__ void k_resid(Dims d, const double *__restrict__ b, const double *__restrict__ x, double *__restrict__ r)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d.n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_of(d, c, i, j, k);
        r[c] = b[c] - fma(6.0, x[c], -nb_sum(x, d, i, j, k, c));
    }
}

// Sum (a, b) over the block in a fixed order; the totals land in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        red[2 * wid] = a;
        red[2 * wid + 1] = b;
    }
    __syncthreads();
    if (tid == 0) {
        a = red[0];
        b = red[1];
        for (int w = 1; w < NT / 32; w++) {
            a += red[2 * w];
            b += red[2 * w + 1];
        }
    }
    __syncthreads();
}

// Every block adds its partials (a, b); returns true in thread 0 of the last block to
// finish, with the grid totals in (a, b), summed over blocks in index order.
template <int NT>
__device__ bool grid_sum2(double &a, double &b, double *red, double *part, PState *st, int nblocks, int bid)
{
    __shared__ int last;
    block_sum2<NT>(a, b, red);
    if (threadIdx.x == 0) {
        part[2 * bid] = a;
        part[2 * bid + 1] = b;
        __threadfence();
        last = atomicAdd(&st->count, 1u) == (unsigned)(nblocks - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += NT) {
        sa += __ldcg(part + 2 * i);
        sb += __ldcg(part + 2 * i + 1);
    }
    block_sum2<NT>(sa, sb, red);
    a = sa;
    b = sb;
    return threadIdx.x == 0;
}

// u = M^-1 r (or u = r), w0 = A u, gamma_0, delta_0, first step length.
template <bool PC>
__global__ void __launch_bounds__(INIT_THREADS) k_start(Dims d, const double *__restrict__ r, double *__restrict__ u,
                                                        double *__restrict__ w0, PState *st, double *part,
                                                        double *eps, double tol, int max_iter)
{
    __shared__ double red[2 * INIT_THREADS / 32];
    double ga = 0.0, da = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)INIT_THREADS + threadIdx.x; c < d.n; c += (int64_t)gridDim.x * INIT_THREADS) {
        int i, j, k;
        cell_of(d, c, i, j, k);
        // u at the cell and its neighbours, then w = A u
        double uc, s;
        if (PC) {
            double rc = r[c];
            auto minv = [&](int64_t e, int ii, int jj, int kk) {   // 6 M^-1
                return fma(6.5, r[e], nb_sum(r, d, ii, jj, kk, e));
            };
            uc = minv(c, i, j, k);
            s = 0.0;
            if (i > 0) s += minv(c - 1, i - 1, j, k);
            if (i < d.nx - 1) s += minv(c + 1, i + 1, j, k);
            if (j > 0) s += minv(c - d.sy, i, j - 1, k);
            if (j < d.ny - 1) s += minv(c + d.sy, i, j + 1, k);
            if (k > 0) s += minv(c - d.sz, i, j, k - 1);
            if (k < d.nz - 1) s += minv(c + d.sz, i, j, k + 1);
            u[c] = uc;
            ga = fma(rc, uc, ga);
        } else {
            uc = r[c];
            s = nb_sum(r, d, i, j, k, c);
            ga = fma(uc, uc, ga);
        }
        double wc = fma(6.0, uc, -s);
        w0[c] = wc;
        da = fma(wc, uc, da);
    }
    if (grid_sum2<INIT_THREADS>(ga, da, red, part, st, gridDim.x, blockIdx.x)) {
        st->count = 0;
        st->it = 0;
        st->tol = tol;
        st->max_iter = max_iter;
        st->gamma0 = ga;
        st->eps = ga > 0.0 ? 1.0 : 0.0;
        if (eps) eps[0] = st->eps;
        st->status = AMR_ENOCONV;
        st->done = 0;
        if (!(ga > 0.0)) {
            st->status = AMR_OK;
            st->done = 1;
        } else if (max_iter == 0) {
            st->done = 1;
        } else {
            double alpha = ga / da;
            if (!(alpha > 0.0) || !isfinite(alpha)) {
                st->status = AMR_EBREAKDOWN;
                st->done = 1;
            }
            st->alpha = alpha;
            st->beta = 0.0;
            st->gamma = ga;
        }
    }
}

template <int TY, bool PC>
struct IterSmem {
    static constexpr int H = PC ? 2 : 1;          // in-plane halo of the w tile
    static constexpr int WX = TX + 2 * H, WY = TY + 2 * H;
    static constexpr int MX = TX + 2, MY = TY + 2;
    static constexpr int RW = 5;                  // w planes in flight or in use
    double w[RW][WY * WX];
    double m[PC ? 3 : 1][PC ? MY * MX : 1];
    double red[2 * TX * TY / 32];
};

// 8-byte asynchronous global -> shared copy; zero-filled when !valid (nothing is read)
__device__ __forceinline__ void cp_async8(double *dst, const double *src, bool valid)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One PPCG iteration (see the file comment).  Grid: (ceil(nx/32), ceil(ny/TY), ceil(nz/seg)).
// Step k of a block's z march: the copy of w plane k+3 (k+2 without preconditioner) is
// started and the seven vectors of cell (x, y, k) are loaded before the block waits for
// w plane k+2 and computes m plane k+1, so both kinds of memory latency overlap the
// previous plane's arithmetic.
template <int TY, bool PC>
__global__ void __launch_bounds__(TX *TY, 1024 / (TX * TY)) k_iter(Dims d, Vecs v, double *__restrict__ x, PState *st,
                                                                  double *part, double *eps, int seg)
{
    constexpr int NT = TX * TY;
    using S = IterSmem<TY, PC>;
    constexpr int H = S::H, WX = S::WX, WY = S::WY, MX = S::MX, MY = S::MY, RW = S::RW;
    constexpr int AHEAD = PC ? 3 : 2;             // w plane started at step k: k + AHEAD
    __shared__ S sm;
    if (st->done) return;
    const int it = st->it;
    const double alpha = st->alpha, beta = st->beta;
    const bool first = it == 0;
    const double *__restrict__ win = (it & 1) ? v.w1 : v.w0;
    double *__restrict__ wout = (it & 1) ? v.w0 : v.w1;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * seg, z1 = min(z0 + seg, d.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < d.nx && gy < d.ny;

    // start copying w plane k (zero outside the box) with the in-plane halo into slot k mod RW
    auto load_w = [&](int k) {
        double *dst = sm.w[(k + RW) % RW];
        const bool zin = k >= 0 && k < d.nz;
        for (int e = tid; e < WX * WY; e += NT) {
            const int ex = e % WX, ey = e / WX;
            const int ix = x0 - H + ex, iy = y0 - H + ey;
            const bool ok = zin && ix >= 0 && ix < d.nx && iy >= 0 && iy < d.ny;
            cp_async8(dst + e, ok ? win + (ix + d.sy * iy + d.sz * k) : win, ok);
        }
    };
    // m = 6 M^-1 w on plane k with a one-cell halo (zero outside the box), into slot k mod 3
    auto comp_m = [&](int k) {
        double *dst = sm.m[(k + 3) % 3];
        const double *wm = sm.w[(k - 1 + RW) % RW], *wc = sm.w[(k + RW) % RW], *wp = sm.w[(k + 1) % RW];
        const bool zin = k >= 0 && k < d.nz;
        for (int e = tid; e < MX * MY; e += NT) {
            const int ex = e % MX, ey = e / MX;
            const int ix = x0 - 1 + ex, iy = y0 - 1 + ey;
            double val = 0.0;
            if (zin && ix >= 0 && ix < d.nx && iy >= 0 && iy < d.ny) {
                const int wi = (ey + 1) * WX + ex + 1;
                const double s = ((wc[wi - 1] + wc[wi + 1]) + (wc[wi - WX] + wc[wi + WX])) + (wm[wi] + wp[wi]);
                val = fma(6.5, wc[wi], s);
            }
            dst[e] = val;
        }
    };

    double ga = 0.0, da = 0.0;
    for (int k = z0 - H; k < z0 + AHEAD; k++) load_w(k);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if (PC) {
        comp_m(z0 - 1);
        comp_m(z0);
        __syncthreads();
    }
    for (int k = z0; k < z1; k++) {
        load_w(k + AHEAD);
        cp_async_commit();
        const int64_t c = gx + d.sy * gy + d.sz * k;
        double rc = 0.0, xc = 0.0, uc = 0.0, zo = 0.0, so = 0.0, po = 0.0, qo = 0.0;
        if (own) {
            rc = v.r[c];
            xc = x[c];
            if (PC) uc = v.u[c];
            if (!first) {
                zo = v.z[c];
                so = v.s[c];
                po = v.p[c];
                if (PC) qo = v.q[c];
            }
        }
        cp_async_wait<1>();
        __syncthreads();
        if (PC) {
            comp_m(k + 1);
            __syncthreads();
        }
        if (!own) continue;
        const double *wk = sm.w[k % RW];
        const double wc = wk[(ty + H) * WX + tx + H];
        double mc, nval;
        if (PC) {
            const double *mk = sm.m[k % 3], *mm = sm.m[(k + 2) % 3], *mp = sm.m[(k + 1) % 3];
            const int mi = (ty + 1) * MX + tx + 1;
            mc = mk[mi];
            const double s = ((mk[mi - 1] + mk[mi + 1]) + (mk[mi - MX] + mk[mi + MX])) + (mm[mi] + mp[mi]);
            nval = fma(6.0, mc, -s);
        } else {
            const int wi = (ty + H) * WX + tx + H;
            const double s = ((wk[wi - 1] + wk[wi + 1]) + (wk[wi - WX] + wk[wi + WX])) +
                             (sm.w[(k + RW - 1) % RW][wi] + sm.w[(k + 1) % RW][wi]);
            mc = wc;
            nval = fma(6.0, wc, -s);
            uc = rc;
        }
        double zz, ss, pp, qq;
        if (first) {
            zz = nval; ss = wc; pp = uc; qq = mc;
        } else {
            zz = fma(beta, zo, nval);
            ss = fma(beta, so, wc);
            pp = fma(beta, po, uc);
            qq = PC ? fma(beta, qo, mc) : ss;
        }
        xc = fma(alpha, pp, xc);
        rc = fma(-alpha, ss, rc);
        const double wn = fma(-alpha, zz, wc);
        v.z[c] = zz; v.s[c] = ss; v.p[c] = pp;
        x[c] = xc; v.r[c] = rc; wout[c] = wn;
        if (PC) {
            uc = fma(-alpha, qq, uc);
            v.q[c] = qq; v.u[c] = uc;
        } else {
            uc = rc;
        }
        ga = fma(rc, uc, ga);
        da = fma(wn, uc, da);
    }
    cp_async_wait<0>();
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (grid_sum2<NT>(ga, da, sm.red, part, st, nb, bid)) {
        // gamma_{i+1}, delta_{i+1}; then eps_{i+1} (Eq. 3) and the next step length
        const int i1 = it + 1;
        st->count = 0;
        st->it = i1;
        const double e = sqrt(ga / st->gamma0);
        st->eps = e;
        if (eps) eps[i1] = e;
        if (e <= st->tol) {
            st->status = AMR_OK;
            st->done = 1;
        } else if (i1 >= st->max_iter) {
            st->done = 1;
        } else {
            const double b1 = ga / st->gamma;
            const double a1 = ga / (da - b1 * ga / alpha);
            if (!(a1 > 0.0) || !isfinite(a1)) {
                st->status = AMR_EBREAKDOWN;
                st->done = 1;
            }
            st->beta = b1;
            st->alpha = a1;
            st->gamma = ga;
        }
    }
}

struct Launch {
    dim3 grid;
    int ty, seg;
};

amr_status plan(const ppcg_params *prm, Launch &L)
{
    L.ty = prm->tile_y ? prm->tile_y : 8;
    if (L.ty != 8 && L.ty != 16) return AMR_EINVAL;
    const int cx = (prm->nx + TX - 1) / TX, cy = (prm->ny + L.ty - 1) / L.ty;
    int seg = prm->seg;
    if (seg == 0) {
        const int64_t cols = (int64_t)cx * cy;
        int64_t nseg = (INIT_BLOCKS + cols - 1) / cols;
        seg = (int)((prm->nz + nseg - 1) / nseg);
        if (seg < MIN_SEG) seg = MIN_SEG;
    }
    if (seg < MIN_SEG) return AMR_EINVAL;
    const int cz = (prm->nz + seg - 1) / seg;
    if (cy > 65535 || cz > 65535) return AMR_EINVAL;
    L.seg = seg;
    L.grid = dim3(cx, cy, cz);
    return AMR_OK;
}

Dims dims_of(int nx, int ny, int nz)
{
    Dims d;
    d.nx = nx; d.ny = ny; d.nz = nz;
    d.sy = nx;
    d.sz = (int64_t)nx * ny;
    d.n = d.sz * nz;
    return d;
}

bool size_ok(int nx, int ny, int nz)
{
    return nx >= 1 && ny >= 1 && nz >= 1 && (int64_t)nx * ny * nz <= (int64_t(1) << 40);
}

amr_status check_prm(const ppcg_params *prm, const void *d_work, size_t work_bytes_given)
{
    if (!prm || !d_work || !size_ok(prm->nx, prm->ny, prm->nz)) return AMR_EINVAL;
    if (prm->precond != PPCG_PRECOND_NONE && prm->precond != PPCG_PRECOND_IP) return AMR_EINVAL;
    if (!(prm->tol >= 0.0) || prm->max_iter < 0 || prm->check_every < 0) return AMR_EINVAL;
    if (((uintptr_t)d_work & 255) != 0) return AMR_EINVAL;
    if (work_bytes_given < work_bytes(prm->nx, prm->ny, prm->nz)) return AMR_ECAPACITY;
    return AMR_OK;
}

int init_grid(int64_t n)
{
    int64_t b = (n + INIT_THREADS - 1) / INIT_THREADS;
    return (int)(b < INIT_BLOCKS ? (b < 1 ? 1 : b) : INIT_BLOCKS);
}

amr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? AMR_OK : AMR_ECUDA; }

} // namespace

extern "C" size_t ppcg_workspace_bytes(int32_t nx, int32_t ny, int32_t nz)
{
    return size_ok(nx, ny, nz) ? work_bytes(nx, ny, nz) : 0;
}

extern "C" amr_status poisson_apply(int32_t nx, int32_t ny, int32_t nz, int32_t op, const double *d_in, double *d_out,
                                    amr_stream stream)
{
    if (!size_ok(nx, ny, nz) || !d_in || !d_out || d_in == d_out) return AMR_EINVAL;
    if (op != POISSON_OP_A && op != POISSON_OP_MINV) return AMR_EINVAL;
    Dims d = dims_of(nx, ny, nz);
    k_apply<<<init_grid(d.n), INIT_THREADS, 0, (cudaStream_t)stream>>>(d, op, d_in, d_out);
    return cuda_status(cudaGetLastError());
}

extern "C" amr_status ppcg_start(const ppcg_params *prm, const double *d_b, const double *d_x, void *d_work,
                                 size_t work_bytes_given, double *d_eps, amr_stream stream)
{
    amr_status s = check_prm(prm, d_work, work_bytes_given);
    if (s != AMR_OK) return s;
    if (!d_b || !d_x) return AMR_EINVAL;
    Launch L;
    if ((s = plan(prm, L)) != AMR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Dims d = dims_of(prm->nx, prm->ny, prm->nz);
    Work w = carve(d_work, prm->nx, prm->ny, prm->nz);
    if (cudaMemsetAsync(w.st, 0, sizeof(PState), st) != cudaSuccess) return AMR_ECUDA;
    const int g = init_grid(d.n);
    k_resid<<<g, INIT_THREADS, 0, st>>>(d, d_b, d_x, w.v.r);
    if (prm->precond == PPCG_PRECOND_IP)
        k_start<true><<<g, INIT_THREADS, 0, st>>>(d, w.v.r, w.v.u, w.v.w0, w.st, w.part, d_eps, prm->tol,
                                                    prm->max_iter);
    else
        k_start<false><<<g, INIT_THREADS, 0, st>>>(d, w.v.r, w.v.u, w.v.w0, w.st, w.part, d_eps, prm->tol,
                                                     prm->max_iter);
    return cuda_status(cudaGetLastError());
}

extern "C" amr_status ppcg_iterate(const ppcg_params *prm, double *d_x, void *d_work, size_t work_bytes_given,
                                   double *d_eps, int32_t count, amr_stream stream)
{
    amr_status s = check_prm(prm, d_work, work_bytes_given);
    if (s != AMR_OK) return s;
    if (!d_x || count < 0) return AMR_EINVAL;
    Launch L;
    if ((s = plan(prm, L)) != AMR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Dims d = dims_of(prm->nx, prm->ny, prm->nz);
    Work w = carve(d_work, prm->nx, prm->ny, prm->nz);
    const bool pc = prm->precond == PPCG_PRECOND_IP;
    for (int i = 0; i < count; i++) {
        if (L.ty == 16) {
            if (pc) k_iter<16, true><<<L.grid, TX * 16, 0, st>>>(d, w.v, d_x, w.st, w.part, d_eps, L.seg);
            else k_iter<16, false><<<L.grid, TX * 16, 0, st>>>(d, w.v, d_x, w.st, w.part, d_eps, L.seg);
        } else {
            if (pc) k_iter<8, true><<<L.grid, TX * 8, 0, st>>>(d, w.v, d_x, w.st, w.part, d_eps, L.seg);
            else k_iter<8, false><<<L.grid, TX * 8, 0, st>>>(d, w.v, d_x, w.st, w.part, d_eps, L.seg);
        }
    }
    return cuda_status(cudaGetLastError());
}

extern "C" amr_status ppcg_poll(const void *d_work, ppcg_info *h_info, amr_stream stream)
{
    if (!d_work || !h_info) return AMR_EINVAL;
    PState h;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, d_work, sizeof(PState), cudaMemcpyDeviceToHost, st) != cudaSuccess) return AMR_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return AMR_ECUDA;
    h_info->iters = h.it;
    h_info->done = h.done;
    h_info->status = h.status;
    h_info->pad = 0;
    h_info->eps = h.eps;
    return AMR_OK;
}

extern "C" amr_status ppcg_solve(const ppcg_params *prm, const double *d_b, double *d_x, void *d_work,
                                 size_t work_bytes_given, double *d_eps, ppcg_info *h_info, amr_stream stream)
{
    amr_status s = ppcg_start(prm, d_b, d_x, d_work, work_bytes_given, d_eps, stream);
    if (s != AMR_OK) return s;
    ppcg_info info;
    if ((s = ppcg_poll(d_work, &info, stream)) != AMR_OK) return s;
    const int chunk = prm->check_every ? prm->check_every : 16;
    int launched = 0;
    while (!info.done && launched < prm->max_iter) {
        int c = prm->max_iter - launched < chunk ? prm->max_iter - launched : chunk;
        if ((s = ppcg_iterate(prm, d_x, d_work, work_bytes_given, d_eps, c, stream)) != AMR_OK) return s;
        launched += c;
        if ((s = ppcg_poll(d_work, &info, stream)) != AMR_OK) return s;
    }
    if (h_info) *h_info = info;
    return (amr_status)info.status;
}
