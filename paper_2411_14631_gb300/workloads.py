"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module only generates inputs: oct lists ``(level, ix, iy, iz)`` (oct coordinates at
the oct's level, 2^(level-1) octs per dimension) and primitive fields
``W = (rho, u, v, w, p)`` sampled at cell centres.  It contains no step of the hydro
scheme; each side converts primitives to conserved variables with its own code.

Workloads (shapes of the paper's runs: clustered, multi-level, high density contrast,
Sec. 1 and Sec. 3.1 of arXiv 2411.14631; the paper's cosmological and galaxy initial
conditions are not available, these synthetic fields stand in for them):

* ``sod``          -- 3D Sod tube, split at x = 0.5 (Toro 2009, Sec. 4.3.3, test 1).
* ``turbulent``    -- periodic box, log-normal density from a Gaussian random field with
                      P(k) ~ k^-4, Gaussian velocity field of rms Mach 2, p = rho.
* ``plummer``      -- Plummer-like clumps (core 0.005, contrast 1e4) on a base level,
                      refined by a quasi-Lagrangian mass threshold, 2:1 balanced.
* ``sedov``        -- point blast, E = 1 deposited in one cell, rho = 1, p = 1e-5.
* ``random_tree``  -- tiny random balanced octrees for table tests.
* ``poisson_rhs``  -- right-hand side of the gravity solve on an N^3 Dirichlet box: the
                      plummer clumps (truncated at r = 0.1) as the source, -4 pi h^2 (rho - mean).
"""
import itertools

import numpy as np

PERIODIC, OUTFLOW = 0, 1


def _pack(x, y, z):
    return (x.astype(np.int64) << 42) | (y.astype(np.int64) << 21) | z.astype(np.int64)


def _unpack(k):
    m = (1 << 21) - 1
    return (k >> 42) & m, (k >> 21) & m, k & m


def full_level(level):
    """All octs of one complete level, as packed coordinates."""
    n = 1 << (level - 1)
    g = np.arange(n, dtype=np.int64)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.unique(_pack(x.ravel(), y.ravel(), z.ravel()))


def to_lxyz(levels):
    """dict level -> packed coords  ->  (n, 4) int32 array of (level, ix, iy, iz)."""
    out = []
    for l in sorted(levels):
        x, y, z = _unpack(levels[l])
        out.append(np.stack([np.full(x.shape, l), x, y, z], axis=1))
    return np.concatenate(out).astype(np.int32)


def balance(levels, periodic=True):
    """Add octs until every oct's father has all 26 father-level neighbours present
    (the 2:1 rule of a fully threaded octree), finest level first."""
    lmax = max(levels)
    for l in range(lmax, 1, -1):
        if l not in levels or levels[l].size == 0:
            continue
        x, y, z = _unpack(levels[l])
        n = 1 << (l - 1)           # father-level cells per dimension
        need = []
        for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
            px, py, pz = x + dx, y + dy, z + dz
            if periodic:
                px, py, pz = px % n, py % n, pz % n
                keep = slice(None)
            else:
                keep = (px >= 0) & (px < n) & (py >= 0) & (py < n) & (pz >= 0) & (pz < n)
            need.append(_pack(px[keep] >> 1, py[keep] >> 1, pz[keep] >> 1))
        levels[l - 1] = np.unique(np.concatenate([levels.get(l - 1, np.empty(0, np.int64))] + need))
    return levels


def uniform_tree(level):
    """Complete octree down to ``level`` (levels 1..level all full)."""
    return to_lxyz({l: full_level(l) for l in range(1, level + 1)})


def random_tree(base, extra, seed, p_refine=0.3, periodic=True):
    """Random balanced octree: complete to ``base``, then up to ``extra`` random levels."""
    rng = np.random.default_rng(seed)
    levels = {l: full_level(l) for l in range(1, base + 1)}
    cur = levels[base]
    for l in range(base + 1, base + extra + 1):
        x, y, z = _unpack(cur)
        kids = []
        for c in range(8):
            pick = rng.random(x.size) < p_refine
            kids.append(_pack(2 * x[pick] + (c & 1), 2 * y[pick] + ((c >> 1) & 1), 2 * z[pick] + ((c >> 2) & 1)))
        cur = np.unique(np.concatenate(kids))
        if cur.size == 0:
            break
        levels[l] = cur
    return to_lxyz(balance(levels, periodic))


def cell_centres(lxyz):
    """Cell centres (n*8, 3) for an oct list in the given order (cell = oct*8 + c)."""
    l = lxyz[:, 0].astype(np.int64)
    base = lxyz[:, 1:4].astype(np.float64) * 2
    c = np.arange(8)
    off = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
    dx = np.ldexp(1.0, -l)
    return ((base[:, None, :] + off[None] + 0.5) * dx[:, None, None]).reshape(-1, 3)


# ---- primitive fields, W[var][cell] -------------------------------------------------
def sod_prims(xyz, axis=0):
    left = xyz[:, axis] < 0.5
    W = np.zeros((5, xyz.shape[0]))
    W[0] = np.where(left, 1.0, 0.125)
    W[4] = np.where(left, 1.0, 0.1)
    return W


def uniform_prims(xyz, rho=1.0, vel=(0.0, 0.0, 0.0), p=1.0):
    W = np.empty((5, xyz.shape[0]))
    W[0] = rho
    W[1:4] = np.asarray(vel, dtype=np.float64)[:, None]
    W[4] = p
    return W


def grf(n, seed, slope=-4.0):
    """Unit-variance Gaussian random field on an n^3 periodic grid with P(k) ~ k^slope
    (integer wavenumbers, k = 0 removed): seeded white noise shaped in Fourier space."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n))
    f = np.fft.rfftn(noise)
    k1 = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)            # sqrt(P) = k^(slope/2)
    d = np.fft.irfftn(f * amp, s=(n, n, n), axes=(0, 1, 2))
    d -= d.mean()
    return d / d.std()


TURB_SEED = 241114631


def turbulent_fields(level, seed=TURB_SEED, sigma=1.0, mach=2.0):
    """Grid fields of the turbulent box: rho = exp(sigma*delta - sigma^2/2),
    velocities from three more fields scaled to 3D rms |v| = mach (c_s = 1), p = rho."""
    n = 1 << level
    delta = grf(n, seed)
    rho = np.exp(sigma * delta - 0.5 * sigma * sigma)
    v = np.stack([grf(n, seed + k) for k in (1, 2, 3)])
    v *= mach / np.sqrt(np.mean(np.sum(v * v, axis=0)))
    return rho, v


def grid_prims(xyz, level, rho, v, p=None):
    """Sample grid fields (level-l cells) at cell centres of level >= l."""
    n = 1 << level
    idx = np.minimum((xyz * n).astype(np.int64), n - 1)
    W = np.empty((5, xyz.shape[0]))
    W[0] = rho[idx[:, 0], idx[:, 1], idx[:, 2]]
    for d in range(3):
        W[1 + d] = v[d][idx[:, 0], idx[:, 1], idx[:, 2]]
    W[4] = W[0] if p is None else p[idx[:, 0], idx[:, 1], idx[:, 2]]
    return W


PLUMMER_A, PLUMMER_CONTRAST = 0.005, 1e4


def plummer_centres(nclump=64, seed=3):
    return np.random.default_rng(seed).random((nclump, 3))


def plummer_density(xyz, centres, a=PLUMMER_A, contrast=PLUMMER_CONTRAST, chunk=1 << 20):
    """rho = 1 + sum_clumps contrast * (1 + r^2/a^2)^(-5/2), periodic minimum image."""
    out = np.ones(xyz.shape[0])
    for s in range(0, xyz.shape[0], chunk):
        x = xyz[s:s + chunk]
        acc = np.zeros(x.shape[0])
        for c in centres:
            d = x - c
            d -= np.round(d)
            r2 = np.einsum("ij,ij->i", d, d)
            acc += contrast * (1.0 + r2 / (a * a)) ** -2.5
        out[s:s + chunk] += acc
    return out


def plummer_tree(base=7, lmax=12, nclump=64, seed=3):
    """Base level complete; a level-l cell (base <= l < lmax) is refined iff
    rho * dx_l^3 > dx_base^3 (a mass threshold of one background base cell, i.e.
    rho > 8^(l-base)), strict; then 2:1 balanced (periodic).  Above the base level only
    cells within the radius where one clump alone could pass the threshold are examined
    (the other clumps and the background add less than 2 there)."""
    centres = plummer_centres(nclump, seed)
    levels = {l: full_level(l) for l in range(1, base + 1)}
    cur = levels[base]                      # octs of level l (packed coordinates)
    a, K = PLUMMER_A, PLUMMER_CONTRAST
    for l in range(base, lmax):
        thr = 8.0 ** (l - base)
        n = 1 << l                          # cells per dimension at level l
        if l == base:
            x, y, z = _unpack(cur)
            c = np.arange(8)
            cx = (2 * x[:, None] + (c & 1)).ravel()
            cy = (2 * y[:, None] + ((c >> 1) & 1)).ravel()
            cz = (2 * z[:, None] + ((c >> 2) & 1)).ravel()
        else:
            rcut = a * np.sqrt((K / (thr - 2.0)) ** 0.4 - 1.0)
            R = int(np.ceil(rcut * n)) + 1
            off = np.arange(-R, R + 1)
            ox, oy, oz = np.meshgrid(off, off, off, indexing="ij")
            cand = []
            for cen in centres:
                ic = np.floor(cen * n).astype(np.int64)
                cand.append(_pack((ic[0] + ox.ravel()) % n, (ic[1] + oy.ravel()) % n, (ic[2] + oz.ravel()) % n))
            cells = np.unique(np.concatenate(cand))
            cx, cy, cz = _unpack(cells)
            inside = np.isin(_pack(cx >> 1, cy >> 1, cz >> 1), cur)   # the cell exists (its oct does)
            cx, cy, cz = cx[inside], cy[inside], cz[inside]
        xyz = (np.stack([cx, cy, cz], axis=1) + 0.5) / n
        rho = plummer_density(xyz, centres)
        pick = rho > thr
        cur = np.unique(_pack(cx[pick], cy[pick], cz[pick]))   # refined cells = octs of level l+1
        if cur.size == 0:
            break
        levels[l + 1] = cur
    return to_lxyz(balance(levels, periodic=True)), centres


def plummer_prims(xyz, centres):
    W = np.zeros((5, xyz.shape[0]))
    W[0] = plummer_density(xyz, centres)
    W[4] = W[0]
    return W


def sedov_prims(xyz, level, e_blast=1.0, rho=1.0, p=1e-5, gamma=1.4):
    """Uniform gas with the blast energy added, as pressure, to the cell whose lower
    corner is the box centre (index n/2 on each axis)."""
    n = 1 << level
    W = uniform_prims(xyz, rho=rho, p=p)
    idx = np.floor(xyz * n).astype(np.int64)
    hit = np.all(idx == n // 2, axis=1) & np.all(np.abs(xyz * n - (idx + 0.5)) < 1e-9, axis=1)
    W[4, hit] = p + (gamma - 1.0) * e_blast * n ** 3
    return W


SOD_GAMMA, TURB_GAMMA, PLUMMER_GAMMA, SEDOV_GAMMA = 1.4, 5.0 / 3.0, 5.0 / 3.0, 1.4


# ---- batches of independent uniform boxes ------------------------------------------
def sedov_batch_sizes(n=48, seed=5, lo=32, hi=192, step=16):
    """n box sizes drawn uniformly from {lo, lo+step, ..., hi} with default_rng(seed)."""
    choices = np.arange(lo, hi + 1, step)
    return np.random.default_rng(seed).choice(choices, size=n).astype(np.int32)


def box_cell_ijk(N):
    """(i, j, k) of every cell of one N^3 box in the batch layout: octs lexicographic
    (x fastest), cell c = cx + 2 cy + 4 cz inside the oct."""
    M = N // 2
    o = np.arange(M ** 3)
    ox, oy, oz = o % M, (o // M) % M, o // (M * M)
    c = np.arange(8)
    i = (2 * ox[:, None] + (c & 1)).ravel()
    j = (2 * oy[:, None] + ((c >> 1) & 1)).ravel()
    k = (2 * oz[:, None] + ((c >> 2) & 1)).ravel()
    return i, j, k


def box_batch_to_lex(N):
    """Index array: position in the batch layout -> lexicographic index i + N (j + N k)."""
    i, j, k = box_cell_ijk(N)
    return i + N * (j + N * k)


def sedov_box_prims_lex(N, e_blast=1.0, rho=1.0, p=1e-5, gamma=1.4):
    """Sedov data for one N^3 box in lexicographic order: the blast energy, as pressure,
    in cell (N/2, N/2, N/2)."""
    W = np.zeros((5, N ** 3))
    W[0] = rho
    W[4] = p
    c = N // 2
    W[4, c + N * (c + N * c)] = p + (gamma - 1.0) * e_blast * N ** 3
    return W


def batch_prims(sizes, per_box_lex):
    """Concatenate per-box lexicographic fields into the batch layout."""
    out = []
    for N in sizes:
        W = per_box_lex(int(N))
        out.append(W[:, box_batch_to_lex(int(N))])
    return np.concatenate(out, axis=1)


POISSON_CLUMP_RMAX = 0.1


def poisson_density(N, nclump=64, seed=3, a=PLUMMER_A, contrast=PLUMMER_CONTRAST):
    """rho = 1 + sum of Plummer clumps (as plummer_density, periodic minimum image), each
    truncated at r = POISSON_CLUMP_RMAX, at the cell centres of an N^3 box; the array is
    indexed i + N (j + N k)."""
    centres = plummer_centres(nclump, seed)
    rho = np.ones((N, N, N))                      # [k, j, i]
    R = int(np.ceil(POISSON_CLUMP_RMAX * N))
    off = np.arange(-R, R + 1)
    for c in centres:
        ic = np.floor(c * N).astype(np.int64)
        idx = [(ic[d] + off) % N for d in range(3)]
        dd = [((idx[d] + 0.5) / N - c[d]) for d in range(3)]
        dd = [x - np.round(x) for x in dd]
        r2 = dd[2][:, None, None] ** 2 + dd[1][None, :, None] ** 2 + dd[0][None, None, :] ** 2
        val = np.where(r2 <= POISSON_CLUMP_RMAX ** 2, contrast * (1.0 + r2 / (a * a)) ** -2.5, 0.0)
        rho[np.ix_(idx[2], idx[1], idx[0])] += val
    return rho.ravel()


def poisson_rhs(N, seed=0, nclump=64):
    """b = -4 pi h^2 (rho - mean rho), h = 1/N, G = 1: the source of A x = b with A the
    7-point -h^2 Laplacian and homogeneous Dirichlet boundaries (box of N^3 cells)."""
    rho = poisson_density(N, nclump=nclump, seed=3 + seed)
    return -4.0 * np.pi * (rho - rho.mean()) / float(N * N)
