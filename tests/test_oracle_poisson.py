"""Pins of the oracle's Poisson solvers (CG and the PPCG of Sec. 2.3) to things other than
themselves: an independently assembled sparse Laplacian, the incomplete-Poisson
preconditioner derived from its definition K K^T, the Dirichlet sine modes (closed-form
eigenpairs of both operators), scipy's conjugate gradient, and a direct solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def _lap(shape):
    """-h^2 Laplacian with homogeneous Dirichlet boundaries, assembled as Kronecker sums of
    1-D second differences (x fastest)."""
    nx, ny, nz = shape

    def d1(n):
        return sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], shape=(n, n))

    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    N = sp.kron(Iz, sp.kron(Iy, d1(nx))) + sp.kron(Iz, sp.kron(d1(ny), Ix)) + sp.kron(d1(nz), sp.kron(Iy, Ix))
    return (6.0 * sp.identity(nx * ny * nz) - N).tocsr(), N.tocsr()


def _ip_minv(shape):
    """The 3-D incomplete-Poisson inverse with constant stencil 13/12 and 1/6 (Sec. 2.3)."""
    _, N = _lap(shape)
    return (13.0 / 12.0 * sp.identity(N.shape[0]) + N / 6.0).tocsr()


def _mode(shape, a, b, c):
    nx, ny, nz = shape
    i, j, k = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1), indexing="ij")
    v = np.sin(np.pi * a * i / (nx + 1)) * np.sin(np.pi * b * j / (ny + 1)) * np.sin(np.pi * c * k / (nz + 1))
    cs = np.cos(np.pi * a / (nx + 1)) + np.cos(np.pi * b / (ny + 1)) + np.cos(np.pi * c / (nz + 1))
    return v.transpose(2, 1, 0).ravel(), cs   # index i + nx (j + ny k)


def test_operator_matches_kronecker_laplacian(oracle):
    rng = np.random.default_rng(1)
    for shape in [(1, 1, 1), (5, 1, 1), (4, 3, 2), (7, 6, 5)]:
        A, _ = _lap(shape)
        x = rng.standard_normal(A.shape[0])
        assert np.allclose(oracle.poisson_apply_A(shape, x), A @ x, rtol=0, atol=1e-13)
        assert np.allclose(oracle.poisson_apply_Minv(shape, x, oracle.PRECOND_IP), _ip_minv(shape) @ x,
                           rtol=0, atol=1e-13)
        assert np.array_equal(oracle.poisson_apply_Minv(shape, x, oracle.PRECOND_NONE), x)


def test_preconditioner_is_incomplete_kkt(oracle):
    """M^-1 = K K^T with K = I - L D^-1 (L the strictly lower part of A, D its diagonal),
    fill-in outside the 7-point pattern dropped: 1/6 on every face neighbour, and
    1 + 3/36 = 13/12 in the centre of each cell whose three lower neighbours exist.
    Cells on a lower face have fewer; the oracle keeps the constant stencil there."""
    shape = (5, 4, 3)
    A, N = _lap(shape)
    Ad = A.toarray()
    L = np.tril(Ad, -1)
    K = np.eye(Ad.shape[0]) - L @ np.diag(1.0 / np.diag(Ad))
    P = K @ K.T
    pattern = (N.toarray() != 0) | np.eye(Ad.shape[0], dtype=bool)
    n = Ad.shape[0]
    Minv = np.stack([oracle.poisson_apply_Minv(shape, np.eye(n)[c]) for c in range(n)], axis=1)
    off = pattern & ~np.eye(n, dtype=bool)
    assert np.allclose(Minv[off], P[off], rtol=0, atol=1e-15)
    assert np.all(Minv[~pattern] == 0.0)
    nx, ny, nz = shape
    for c in range(n):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        if i > 0 and j > 0 and k > 0:
            assert P[c, c] == pytest.approx(13.0 / 12.0, abs=1e-15)
            assert Minv[c, c] == pytest.approx(P[c, c], abs=1e-15)


def test_sine_modes_are_eigenvectors(oracle):
    shape = (6, 5, 4)
    for a, b, c in [(1, 1, 1), (3, 2, 4), (6, 5, 4)]:
        v, cs = _mode(shape, a, b, c)
        assert np.allclose(oracle.poisson_apply_A(shape, v), (6.0 - 2.0 * cs) * v, atol=1e-13)
        assert np.allclose(oracle.poisson_apply_Minv(shape, v), (13.0 / 12.0 + cs / 3.0) * v, atol=1e-13)


@pytest.mark.parametrize("solver", ["cg", "ppcg"])
@pytest.mark.parametrize("precond", [0, 1])
def test_single_and_double_mode_converge_in_one_and_two(oracle, solver, precond):
    """A right-hand side in one eigenvector of A (and of M^-1) is solved by the first step;
    one in two eigenvectors with distinct eigenvalues of M^-1 A by the second."""
    shape = (6, 5, 4)
    f = getattr(oracle, solver)
    v, cs = _mode(shape, 2, 1, 3)
    x, eps, it, st = f(shape, v, precond=precond, tol=1e-12, maxit=10)
    assert st == oracle.OK and it == 1
    assert np.allclose(x, v / (6.0 - 2.0 * cs), rtol=0, atol=1e-14)
    w, _ = _mode(shape, 5, 4, 1)
    x, eps, it, st = f(shape, v + 0.5 * w, precond=precond, tol=1e-12, maxit=10)
    assert st == oracle.OK and it == 2
    assert eps[1] > 1e-3


@pytest.mark.parametrize("precond", [0, 1])
def test_iterates_match_scipy_cg(oracle, precond):
    """Both oracle solvers reproduce scipy's (preconditioned) CG iterates and the Eq. 3
    measure evaluated from true residuals b - A x_k."""
    shape = (12, 10, 8)
    A, _ = _lap(shape)
    Minv = _ip_minv(shape) if precond else sp.identity(A.shape[0]).tocsr()
    rng = np.random.default_rng(7)
    b = rng.standard_normal(A.shape[0])
    xs = []
    spl.cg(A, b, x0=np.zeros_like(b), rtol=0.0, atol=0.0, maxiter=15,
           M=spl.aslinearoperator(Minv), callback=lambda xk: xs.append(xk.copy()))
    r0 = b
    g0 = r0 @ (Minv @ r0)
    eps_ref = [np.sqrt((b - A @ xk) @ (Minv @ (b - A @ xk)) / g0) for xk in xs]
    for solver in (oracle.cg, oracle.ppcg):
        for k in (1, 5, 15):
            x, eps, it, st = solver(shape, b, precond=precond, tol=0.0, maxit=k)
            assert st == oracle.ENOCONV and it == k and eps.size == k + 1 and eps[0] == 1.0
            assert np.allclose(x, xs[k - 1], rtol=0, atol=1e-10 * np.abs(xs[k - 1]).max())
            assert np.allclose(eps[1:], eps_ref[:k], rtol=1e-8, atol=0)


@pytest.mark.parametrize("precond", [0, 1])
def test_converged_solution_matches_direct_solve(oracle, precond):
    shape = (9, 8, 7)
    A, _ = _lap(shape)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(A.shape[0])
    xd = spl.spsolve(A.tocsc(), b)
    x0 = rng.standard_normal(A.shape[0])
    x, eps, it, st = oracle.ppcg(shape, b, x0=x0, precond=precond, tol=1e-12, maxit=500)
    assert st == oracle.OK and eps[-1] <= 1e-12 and np.all(eps[:-1] > 1e-12)
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()


def test_edge_cases(oracle):
    # one cell: A = 6, M^-1 = 13/12, so x = b / 6 after one step
    for solver in (oracle.cg, oracle.ppcg):
        for precond in (0, 1):
            x, eps, it, st = solver((1, 1, 1), [3.0], precond=precond, tol=1e-14, maxit=5)
            assert st == oracle.OK and it == 1 and x[0] == pytest.approx(0.5, abs=1e-16)
    # the initial guess already solves the system
    shape = (4, 4, 4)
    xd = np.random.default_rng(5).standard_normal(64)
    b = oracle.poisson_apply_A(shape, xd)
    for solver in (oracle.cg, oracle.ppcg):
        x, eps, it, st = solver(shape, b, x0=xd, tol=1e-6, maxit=5)
        assert st == oracle.OK and it == 0 and eps[0] == 0.0 and np.array_equal(x, xd)
        x, eps, it, st = solver(shape, np.ones(64), maxit=0)
        assert st == oracle.ENOCONV and it == 0 and eps[0] == 1.0
        _, _, _, st = solver((0, 4, 4), np.ones(1), maxit=3)
        assert st == oracle.EINVAL
        _, _, _, st = solver(shape, np.ones(64), precond=7, maxit=3)
        assert st == oracle.EINVAL


def test_preconditioner_halves_iterations(oracle):
    """Fig. 4 / Sec. 2.3: to eps = 1e-4 the preconditioned solve needs about half the
    iterations of plain CG (1.86x in the paper's run).  For this stencil pair the ratio of
    condition numbers is 12 / (max_c (6-2c)(13/12+c/3) * 12/25) = 3.84 on fine grids, so
    about sqrt(3.84) = 1.96 in iterations."""
    shape = (48, 48, 48)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(int(np.prod(shape)))
    _, e_cg, it_cg, st1 = oracle.cg(shape, b, precond=0, tol=1e-4, maxit=2000)
    _, e_pp, it_pp, st2 = oracle.ppcg(shape, b, precond=1, tol=1e-4, maxit=2000)
    assert st1 == st2 == oracle.OK
    assert 1.5 <= it_cg / it_pp <= 2.3
