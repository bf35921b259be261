"""Plain FP64 CPU oracle for the AMR Godunov hydro hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``.  The product library never imports it.  It
shares no code with the CUDA path; the C sources in this folder are compiled with
``-O2 -ffp-contract=off`` (no fused multiply-add, so every rounding step is the one
written in the source).

The scheme it writes out (the paper prints none; Table 1 only names godunov_fine,
newdt_fine and refine_fine) is documented at the top of ``hydro.c``; the Riemann
solvers in ``riemann.c``; the octree and Hilbert key in ``tree.c``; the surrogate
network in ``mlp.c``; the CG and PPCG Poisson solvers of Sec. 2.3 in ``poisson.c``.
"""
import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["riemann.c", "tree.c", "hydro.c", "mlp.c", "box.c", "poisson.c", "refine.c", "subcycle.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EUNBALANCED, ENONPHYSICAL, ENOCONV, EBREAKDOWN = 0, -1, -2, -6, -7, -8
PRECOND_NONE, PRECOND_IP = 0, 1
PERIODIC, OUTFLOW = 0, 1
HLLC, EXACT = 0, 1
OUTSIDE = -(2 ** 31)
MAXLEV = 21


def build(force=False):
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SRC] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        L.or_hilbert_key.restype = C.c_uint64
        L.or_hilbert_key.argtypes = [C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_tree_build.argtypes = [C.c_int32, P, P, C.c_int64, C.POINTER(C.c_void_p)]
        L.or_tree_free.argtypes = [P]
        L.or_tree_noct.restype = C.c_int64
        L.or_tree_noct.argtypes = [P]
        L.or_tree_export.argtypes = [P] + [P] * 10
        L.or_lookup.restype = C.c_int64
        L.or_lookup.argtypes = [P, C.c_int, C.c_int64, C.c_int64, C.c_int64]
        L.or_minmod.restype = C.c_double
        L.or_minmod.argtypes = [C.c_double, C.c_double]
        L.or_mc.restype = C.c_double
        L.or_mc.argtypes = [C.c_double, C.c_double]
        L.or_cons_to_prim.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
        L.or_prim_to_cons.argtypes = [P, C.c_double, P]
        L.or_flux_normal.argtypes = [P, C.c_double, P]
        L.or_hllc.argtypes = [P, P, C.c_double, P]
        L.or_exact_star.argtypes = [P, P, C.c_double, C.c_double, C.c_int, P, P, P]
        L.or_exact_sample.argtypes = [P, P, C.c_double, C.c_double, C.c_double, C.c_double, P]
        L.or_riemann_flux.argtypes = [P, P, P, P]
        L.or_oct_stencil.argtypes = [P, P, C.c_int64, P]
        L.or_courant.argtypes = [P, P, P, P]
        L.or_level_update.argtypes = [P, P, C.c_int, P, P, P, C.c_double]
        L.or_octs_update.argtypes = [P, P, C.c_int64, C.c_int64, P, P, P, C.c_double]
        L.or_reflux_restrict.argtypes = [P, P, C.c_int, P, P, C.c_double]
        L.or_step.argtypes = [P, P, P, P, P, C.c_int]
        L.or_init_from_prim.argtypes = [P, P, P, P]
        L.or_prim_of_state.argtypes = [P, P, P, P]
        L.or_box_courant.argtypes = [C.c_int64, P, P, P]
        L.or_box_step.argtypes = [C.c_int64, P, P, P, P, C.c_double]
        L.or_mlp_nparams.restype = C.c_int64
        L.or_mlp_features.argtypes = [P, P, C.c_double, P, P]
        L.or_mlp_forward.argtypes = [P, P, C.c_int64, P, P]
        L.or_mlp_backward.argtypes = [P, P, P, C.c_int64, P, P]
        L.or_adam_step.argtypes = [P, P, P, P, C.c_int64, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int64]
        I = C.c_int
        L.or_courant_levels.argtypes = [P, P, P, P]
        L.or_step_subcycled.argtypes = [P, P, P, P]
        L.or_refine_flags.argtypes = [P, P, C.c_double, I, P]
        L.or_refine_list.argtypes = [P, P, C.c_double, I, P, C.c_int64, C.POINTER(C.c_int64)]
        L.or_remap.argtypes = [P, P, P, P]
        L.or_poisson_apply_A.argtypes = [I, I, I, P, P]
        L.or_poisson_apply_Minv.argtypes = [I, I, I, I, P, P]
        for f in (L.or_cg, L.or_ppcg):
            f.argtypes = [I, I, I, I, P, P, C.c_double, I, P, C.POINTER(C.c_int)]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("riemann", C.c_int32), ("limiter", C.c_int32)]


LIMITER_MINMOD, LIMITER_MC = 0, 1


def params(gamma=1.4, cfl=0.8, rho_floor=1e-10, p_floor=1e-20, riemann=HLLC, limiter=LIMITER_MINMOD):
    return Params(gamma, cfl, rho_floor, p_floor, riemann, limiter)


class Tree:
    """An octree built by the oracle from a list of (level, ix, iy, iz) octs."""

    def __init__(self, lxyz, levelmin, bc=(PERIODIC,) * 6):
        lxyz = np.ascontiguousarray(lxyz, dtype=np.int32).reshape(-1, 4)
        bc = np.ascontiguousarray(bc, dtype=np.int32)
        h = C.c_void_p()
        st = lib().or_tree_build(levelmin, _p(bc), _p(lxyz), lxyz.shape[0], C.byref(h))
        self.status = st
        self._h = h if st == OK else None
        if st != OK:
            return
        n = lib().or_tree_noct(h)
        self.noct = n
        self.ncell = 8 * n
        self.levelmin = levelmin
        self.bc = tuple(int(b) for b in bc)
        a = {k: np.empty(n, np.int32) for k in ("lvl", "ix", "iy", "iz", "father")}
        self.key = np.empty(n, np.uint64)
        self.son = np.empty(8 * n, np.int32)
        self.nbor = np.empty(6 * n, np.int32)
        self.nb27 = np.empty(27 * n, np.int32)
        self.lvl_off = np.empty(MAXLEV + 2, np.int64)
        lib().or_tree_export(h, _p(a["lvl"]), _p(a["ix"]), _p(a["iy"]), _p(a["iz"]), _p(self.key),
                             _p(self.son), _p(a["father"]), _p(self.nbor), _p(self.nb27), _p(self.lvl_off))
        for k, v in a.items():
            setattr(self, k, v)
        self.levelmax = int(self.lvl.max())

    @property
    def ok(self):
        return self.status == OK

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_tree_free(self._h)
            self._h = None

    def lookup(self, l, x, y, z):
        return lib().or_lookup(self._h, l, x, y, z)

    def cell_centres(self):
        """(ncell, 3) cell-centre coordinates and (ncell,) levels, in cell-id order."""
        c = np.arange(8)
        off = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
        base = np.stack([self.ix, self.iy, self.iz], axis=1).astype(np.float64) * 2
        dx = np.ldexp(1.0, -self.lvl.astype(np.int64))
        xyz = (base[:, None, :] + off[None, :, :] + 0.5) * dx[:, None, None]
        lv = np.repeat(self.lvl, 8)
        return xyz.reshape(-1, 3), lv

    def leaf_mask(self):
        return self.son < 0

    # ---- hydro --------------------------------------------------------------
    def init_from_prim(self, w, prm):
        w = _f64(w)
        u = np.empty_like(w)
        lib().or_init_from_prim(self._h, C.byref(prm), _p(w), _p(u))
        return u

    def prim(self, u, prm):
        u = _f64(u)
        w = np.empty_like(u)
        lib().or_prim_of_state(self._h, C.byref(prm), _p(u), _p(w))
        return w

    def courant(self, u, prm):
        u = _f64(u)
        dt = C.c_double()
        lib().or_courant(self._h, C.byref(prm), _p(u), C.byref(dt))
        return dt.value

    def step(self, u, prm, nthreads=0):
        u = _f64(u)
        un = np.empty_like(u)
        dt = C.c_double()
        st = lib().or_step(self._h, C.byref(prm), _p(u), _p(un), C.byref(dt), nthreads)
        return un, dt.value, st

    def step_subcycled(self, u, prm):
        """One coarse step with sub-cycled levels (dt halves per level); returns (u, dt_base, status)."""
        u = _f64(u).copy()
        dt = C.c_double()
        st = lib().or_step_subcycled(self._h, C.byref(prm), _p(u), C.byref(dt))
        return u, dt.value, st

    def courant_levels(self, u, prm):
        u = _f64(u)
        dt = C.c_double()
        lib().or_courant_levels(self._h, C.byref(prm), _p(u), C.byref(dt))
        return dt.value

    def level_update(self, level, u_old, u_new, reg, dt, prm):
        return lib().or_level_update(self._h, C.byref(prm), level, _p(u_old), _p(u_new), _p(reg), dt)

    def reflux_restrict(self, level, reg, u_new, dt, prm):
        return lib().or_reflux_restrict(self._h, C.byref(prm), level, _p(reg) if reg is not None else None,
                                        _p(u_new), dt)

    # ---- refinement (refine_fine) ----------------------------------------------------
    def refine_flags(self, u, mass_thr, lmax):
        u = _f64(u)
        f = np.zeros(self.ncell, np.uint8)
        st = lib().or_refine_flags(self._h, _p(u), mass_thr, lmax, _p(f))
        return f, st

    def refine_list(self, u, mass_thr, lmax):
        """New oct list (level, ix, iy, iz) after refinement by mass (refine.c)."""
        u = _f64(u)
        cap = self.ncell + 1
        out = np.zeros((cap, 4), np.int32)
        n = C.c_int64()
        st = lib().or_refine_list(self._h, _p(u), mass_thr, lmax, _p(out), cap, C.byref(n))
        return out[:n.value].copy(), st

    def remap(self, u, new_tree):
        """State on new_tree: copied where the cell exists here, interpolated otherwise."""
        u = _f64(u)
        un = np.empty((5, new_tree.ncell))
        st = lib().or_remap(self._h, _p(u), new_tree._h, _p(un))
        return un, st

    # ---- global conservation diagnostics ----------------------------------------------
    def conservation_totals(self, u):
        """[2][5]: the sum over the leaf cells of U_v dV (dV = dx_l^3 = 2^-3l) and of
        |U_v| dV, each exactly rounded (math.fsum): the plain definition of the leaf totals
        that the level step (Table 1, godunov_fine with refluxing) conserves, with no
        summation order of its own."""
        u = _f64(u)
        leaf = self.son < 0
        dV = np.ldexp(1.0, -3 * np.repeat(self.lvl, 8).astype(np.int64))[leaf]
        out = np.empty((2, 5))
        for v in range(5):
            x = u[v, leaf] * dV                  # exact: dV is a power of two
            out[0, v] = math.fsum(x.tolist())
            out[1, v] = math.fsum(np.abs(x).tolist())
        return out

    def stencil(self, u, oct_id):
        u = _f64(u)
        s = np.empty(5 * 216)
        st = lib().or_oct_stencil(self._h, _p(u), oct_id, _p(s))
        return s.reshape(5, 6, 6, 6), st


def box_conservation_totals(sizes, u):
    """[nbox][2][5] for a batch of uniform boxes of sizes[b]^3 cells stored one after the
    other: sum over box b's cells of U_v / N^3 and of |U_v| / N^3, as the exactly rounded
    sum (math.fsum) divided by the integer N^3 (one more rounding)."""
    u = _f64(u)
    out = np.empty((len(sizes), 2, 5))
    c0 = 0
    for b, N in enumerate(sizes):
        n = int(N) ** 3
        for v in range(5):
            x = u[v, c0:c0 + n]
            out[b, 0, v] = math.fsum(x.tolist()) / n
            out[b, 1, v] = math.fsum(np.abs(x).tolist()) / n
        c0 += n
    return out


def hilbert_key(bits, x, y, z):
    return lib().or_hilbert_key(bits, x, y, z)


def minmod(a, b):
    return lib().or_minmod(a, b)


def mc(a, b):
    return lib().or_mc(a, b)


def cons_to_prim(U, gamma, rho_floor=1e-10, p_floor=1e-20):
    U = _f64(U); W = np.empty(5)
    lib().or_cons_to_prim(_p(U), gamma, rho_floor, p_floor, _p(W))
    return W


def prim_to_cons(W, gamma):
    W = _f64(W); U = np.empty(5)
    lib().or_prim_to_cons(_p(W), gamma, _p(U))
    return U


def flux_normal(W, gamma):
    W = _f64(W); F = np.empty(5)
    lib().or_flux_normal(_p(W), gamma, _p(F))
    return F


def hllc(WL, WR, gamma):
    WL = _f64(WL); WR = _f64(WR); F = np.empty(5)
    lib().or_hllc(_p(WL), _p(WR), gamma, _p(F))
    return F


def exact_star(WL, WR, gamma, tol=1e-14, maxit=50):
    WL = _f64(WL); WR = _f64(WR)
    ps, us, it = C.c_double(), C.c_double(), C.c_int()
    st = lib().or_exact_star(_p(WL), _p(WR), gamma, tol, maxit, C.byref(ps), C.byref(us), C.byref(it))
    return ps.value, us.value, st, it.value


def exact_sample(WL, WR, gamma, ps, us, S):
    WL = _f64(WL); WR = _f64(WR); W = np.empty(5)
    lib().or_exact_sample(_p(WL), _p(WR), gamma, ps, us, S, _p(W))
    return W


def riemann_flux(WL, WR, prm):
    WL = _f64(WL); WR = _f64(WR); F = np.empty(5)
    st = lib().or_riemann_flux(_p(WL), _p(WR), C.byref(prm), _p(F))
    return F, st


# ---- uniform boxes ----------------------------------------------------------------
def box_courant(N, u, prm):
    u = _f64(u)
    dt = C.c_double()
    lib().or_box_courant(N, C.byref(prm), _p(u), C.byref(dt))
    return dt.value


def box_step(N, bc, u, prm, dt):
    """One step of a uniform N^3 box; state [5][N^3] with cell i + N (j + N k)."""
    u = _f64(u)
    un = np.empty_like(u)
    bc = np.ascontiguousarray(bc, dtype=np.int32)
    st = lib().or_box_step(N, _p(bc), C.byref(prm), _p(u), _p(un), dt)
    return un, st


# ---- surrogate network ---------------------------------------------------------
def mlp_nparams():
    return lib().or_mlp_nparams()


def mlp_features(WL, WR, gamma):
    WL = _f64(WL); WR = _f64(WR); x = np.empty(7); ref = np.empty(3)
    lib().or_mlp_features(_p(WL), _p(WR), gamma, _p(x), _p(ref))
    return x, ref


def mlp_forward(theta, x, keep_act=False):
    theta = _f64(theta); x = _f64(x).reshape(-1, 7)
    n = x.shape[0]
    y = np.empty((n, 2))
    act = np.empty((n, 6 * 64)) if keep_act else None
    lib().or_mlp_forward(_p(theta), _p(x), n, _p(y), _p(act) if keep_act else None)
    return (y, act) if keep_act else y


def mlp_backward(theta, x, dy):
    """Gradient of sum(dy * y) with respect to theta."""
    theta = _f64(theta); x = _f64(x).reshape(-1, 7); dy = _f64(dy).reshape(-1, 2)
    _, act = mlp_forward(theta, x, keep_act=True)
    g = np.zeros(theta.size)
    lib().or_mlp_backward(_p(theta), _p(x), _p(dy), x.shape[0], _p(act), _p(g))
    return g


def adam_step(theta, m, v, grad, lr, beta1, beta2, eps, t):
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = _f64(grad)
    lib().or_adam_step(_p(theta), _p(m), _p(v), _p(grad), theta.size, lr, beta1, beta2, eps, t)


# ---- Poisson solve (Sec. 2.3) ---------------------------------------------------
def poisson_apply_A(shape, x):
    """y = A x, A = 6 I - (sum over in-box face neighbours); shape = (nx, ny, nz),
    vectors indexed i + nx (j + ny k)."""
    nx, ny, nz = shape
    x = _f64(x).ravel()
    y = np.empty_like(x)
    lib().or_poisson_apply_A(nx, ny, nz, _p(x), _p(y))
    return y


def poisson_apply_Minv(shape, r, precond=PRECOND_IP):
    nx, ny, nz = shape
    r = _f64(r).ravel()
    u = np.empty_like(r)
    lib().or_poisson_apply_Minv(nx, ny, nz, precond, _p(r), _p(u))
    return u


def _krylov(fn, shape, b, x0, precond, tol, maxit):
    nx, ny, nz = shape
    b = _f64(b).ravel()
    x = np.zeros_like(b) if x0 is None else _f64(x0).ravel().copy()
    eps = np.full(maxit + 1, np.nan)
    it = C.c_int()
    st = fn(nx, ny, nz, precond, _p(b), _p(x), tol, maxit, _p(eps), C.byref(it))
    return x, eps[:it.value + 1].copy(), it.value, st


def cg(shape, b, x0=None, precond=PRECOND_NONE, tol=1e-4, maxit=1000):
    """Textbook (preconditioned) CG; returns (x, eps history per Eq. 3, iterations, status)."""
    return _krylov(lib().or_cg, shape, b, x0, precond, tol, maxit)


def ppcg(shape, b, x0=None, precond=PRECOND_IP, tol=1e-4, maxit=1000):
    """Preconditioned pipelined CG (Ghysels & Vanroose 2014, Algorithm 4) as adopted in
    Sec. 2.3; returns (x, eps history per Eq. 3, iterations, status)."""
    return _krylov(lib().or_ppcg, shape, b, x0, precond, tol, maxit)
