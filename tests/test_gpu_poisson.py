"""GPU parity of the Poisson solver (PPCG of Sec. 2.3) against the oracle, through the C ABI.

Tolerances.  The kernels sum inner products per thread block, fuse multiply-adds and
evaluate each stencil in its own order; the oracle sums sequentially without fusion.
Replaying the oracle's iteration with a different summation order moved the iterate by
at most 1.3e-12 of max|x| and eps (Eq. 3) by at most 1.2e-14 over 100 iterations on
64^3 and ragged 37x21x13 boxes, so the bounds below (1e-10 of max|x|, 1e-11 absolute on
eps) leave two orders of margin while a wrong coefficient, sign or index is off by
orders of magnitude more.  On the 256^3 box the oracle's own sequential inner products
carry the larger error: recursive summation of n terms is exact to (n-1) u sum|t_i|
(Higham 2002, Sec. 4.2), u = 2^-53, so there eps is compared within 2 n u of itself."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2411_14631_gb300 import build
    build.build()
    from paper_2411_14631_gb300 import abi, poisson
    abi.lib()
    return abi, poisson


def _rhs(shape, seed):
    return np.random.default_rng(seed).standard_normal(int(np.prod(shape)))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda:0")


@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 21, 13), (64, 3, 5), (33, 17, 40)])
def test_operators_match_oracle(oracle, P, shape):
    abi, poisson = P
    x = _rhs(shape, 1)
    for op, ref in ((abi.OP_A, oracle.poisson_apply_A(shape, x)),
                    (abi.OP_MINV, oracle.poisson_apply_Minv(shape, x, oracle.PRECOND_IP))):
        y = poisson.apply(shape, op, _dev(x)).cpu().numpy()
        assert np.allclose(y, ref, rtol=0, atol=1e-14 * np.abs(x).max() * 8)


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("shape,tile_y,seg", [((37, 21, 13), 16, 0), ((37, 21, 13), 8, 4), ((37, 21, 13), 16, 5),
                                              ((64, 64, 64), 16, 0), ((64, 64, 64), 8, 24), ((5, 70, 9), 8, 0)])
def test_fixed_iterations_match_oracle(oracle, P, precond, shape, tile_y, seg):
    """tol = 0: exactly K iterations; iterate and eps history element by element, for
    several tile heights and z segments (ragged tiles, segments that do not divide nz)."""
    abi, poisson = P
    K = 30
    b = _rhs(shape, 2)
    x0 = 0.1 * _rhs(shape, 3)
    xo, eo, ito, sto = oracle.ppcg(shape, b, x0=x0, precond=precond, tol=0.0, maxit=K)
    assert sto == oracle.ENOCONV and ito == K
    s = poisson.PPCG(shape, precond=precond, tol=0.0, max_iter=K, check_every=7, tile_y=tile_y, seg=seg)
    x, e, info = s.solve(_dev(b), _dev(x0))
    assert info.status == abi.ENOCONV and info.iters == K and info.done == 1
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-10 * np.abs(xo).max()
    assert np.abs(e - eo).max() <= 1e-11


@pytest.mark.parametrize("precond", [0, 1])
def test_solve_to_tolerance_matches_oracle(oracle, P, precond):
    shape = (48, 40, 36)
    b = _rhs(shape, 4)
    xo, eo, ito, sto = oracle.ppcg(shape, b, precond=precond, tol=1e-8, maxit=2000)
    assert sto == oracle.OK
    abi, poisson = P
    x, e, info = poisson.PPCG(shape, precond=precond, tol=1e-8, max_iter=2000).solve(_dev(b))
    assert info.status == abi.OK
    assert info.iters == ito
    assert np.abs(e - eo).max() <= 1e-11 and info.eps == pytest.approx(e[-1], abs=0)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-10 * np.abs(xo).max()


def test_deterministic_and_reentrant(P):
    abi, poisson = P
    shape = (40, 33, 29)
    b = _dev(_rhs(shape, 5))
    s = poisson.PPCG(shape, tol=1e-6, max_iter=500)
    x1, e1, i1 = s.solve(b)
    x2, e2, i2 = s.solve(b)
    assert i1.iters == i2.iters and torch.equal(x1, x2) and np.array_equal(e1, e2)


def test_sine_mode_one_iteration(P):
    """A right-hand side in one Dirichlet sine mode is solved by the first step: x = b / lambda."""
    abi, poisson = P
    nx, ny, nz = shape = (24, 20, 18)
    i, j, k = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1), indexing="ij")
    a, bb, c = 3, 2, 5
    v = (np.sin(np.pi * a * i / (nx + 1)) * np.sin(np.pi * bb * j / (ny + 1)) *
         np.sin(np.pi * c * k / (nz + 1))).transpose(2, 1, 0).ravel()
    lam = 6 - 2 * (np.cos(np.pi * a / (nx + 1)) + np.cos(np.pi * bb / (ny + 1)) + np.cos(np.pi * c / (nz + 1)))
    for precond in (0, 1):
        x, e, info = poisson.PPCG(shape, precond=precond, tol=1e-12, max_iter=10).solve(_dev(v))
        assert info.status == abi.OK and info.iters == 1
        assert np.abs(x.cpu().numpy() - v / lam).max() <= 1e-13


def test_edge_cases(oracle, P):
    abi, poisson = P
    # one cell
    x, e, info = poisson.PPCG((1, 1, 1), tol=1e-14, max_iter=4).solve(_dev([3.0]))
    assert info.status == abi.OK and info.iters == 1 and x.item() == pytest.approx(0.5, abs=1e-16)
    # the initial guess already solves the system (integer values: A x is exact in any order)
    shape = (20, 9, 7)
    xd = np.random.default_rng(6).integers(-8, 9, int(np.prod(shape))).astype(np.float64)
    b = oracle.poisson_apply_A(shape, xd)
    x, e, info = poisson.PPCG(shape, tol=1e-6, max_iter=5).solve(_dev(b), _dev(xd))
    assert info.status == abi.OK and info.iters == 0 and e[0] == 0.0 and np.array_equal(x.cpu().numpy(), xd)
    # no iterations allowed
    x, e, info = poisson.PPCG(shape, tol=1e-6, max_iter=0).solve(_dev(b))
    assert info.status == abi.ENOCONV and info.iters == 0 and e[0] == 1.0
    # argument errors come back as statuses
    L = abi.lib()
    prm = abi.PpcgParams(20, 9, 7, 1, 1e-6, 5, 0, 12, 0)
    s = poisson.PPCG(shape, tol=1e-6, max_iter=5)
    import ctypes as C
    assert L.ppcg_start(C.byref(prm), C.c_void_p(s.work.data_ptr()), C.c_void_p(s.work.data_ptr()),
                        C.c_void_p(s.work.data_ptr()), s.nbytes, None, None) == abi.EINVAL
    prm.tile_y = 16
    assert L.ppcg_start(C.byref(prm), C.c_void_p(s.work.data_ptr()), C.c_void_p(s.work.data_ptr()),
                        C.c_void_p(s.work.data_ptr()), s.nbytes - 8, None, None) == abi.ECAPACITY


def test_full_size_plummer_density(oracle, P):
    """The 256^3 study workload (clumpy density, Dirichlet box): ten iterations element by
    element against the oracle, then the full solve to eps = 1e-4 checked by the oracle's
    operators: the true residual of the returned x meets Eq. 3's bound."""
    from paper_2411_14631_gb300 import workloads
    abi, poisson = P
    shape = (256, 256, 256)
    b = workloads.poisson_rhs(256, seed=0)
    K = 10
    xo, eo, ito, sto = oracle.ppcg(shape, b, precond=1, tol=0.0, maxit=K)
    bd = _dev(b)
    x, e, info = poisson.PPCG(shape, tol=0.0, max_iter=K).solve(bd)
    assert info.iters == K
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-10 * np.abs(xo).max()
    n = b.size
    assert np.all(np.abs(e - eo) <= 1e-11 + 2 * n * 2.0 ** -53 * eo)
    x, e, info = poisson.PPCG(shape, tol=1e-4, max_iter=3000).solve(bd)
    assert info.status == abi.OK and e[-1] <= 1e-4 and np.all(e[1:-1] > 1e-4)
    xh = x.cpu().numpy()
    r = b - oracle.poisson_apply_A(shape, xh)
    u = oracle.poisson_apply_Minv(shape, r)
    u0 = oracle.poisson_apply_Minv(shape, b)
    eps_true = np.sqrt((r @ u) / (b @ u0))
    assert eps_true == pytest.approx(e[-1], rel=1e-6)
