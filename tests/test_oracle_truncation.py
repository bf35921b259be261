"""One step of the oracle against the exact solution of the Euler equations.

The data is a smooth simple wave: isentropic gas (p = rho^gamma, gamma = 1.4) whose
backward Riemann invariant u - 2c/(gamma-1) is uniform, so the solution is carried
unchanged along the forward characteristics dx/dt = u + c until they cross (Courant &
Friedrichs; Toro 2009, Sec. 3.1).  Here rho = 1 + 0.1 sin(2 pi x), boosted by a uniform
u0 = 1, on a periodic box; the exact state at x and t comes from solving
x = x0 + (u + c)(x0) t for x0, and cell averages from Gauss-Legendre quadrature.

A second-order scheme's error after one step is O(dx^3) (dt proportional to dx) where
the solution is smooth and monotone; at extrema the MinMod slopes clip and the error is
O(dx^2), so the measure skips cells near them.  A dropped, misplaced or wrongly scaled
term of the MUSCL-Hancock predictor, or a wrong sign of the face states, leaves O(dx^2)
everywhere."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

G, EPS, U0 = 1.4, 0.1, 1.0
C0 = np.sqrt(G)


def _state(x0):
    rho = 1.0 + EPS * np.sin(2 * np.pi * x0)
    c = C0 * rho ** ((G - 1) / 2)
    return rho, U0 + 2.0 / (G - 1) * (c - C0), rho ** G


def _exact(x, t):
    """Newton on f(x0) = x0 + (u + c)(x0) t - x (monotone before the characteristics cross)."""
    x0 = x - (C0 + U0) * t
    for _ in range(50):
        rho = 1.0 + EPS * np.sin(2 * np.pi * x0)
        c = C0 * rho ** ((G - 1) / 2)
        u = U0 + 2.0 / (G - 1) * (c - C0)
        dc = C0 * (G - 1) / 2 * rho ** ((G - 3) / 2) * EPS * 2 * np.pi * np.cos(2 * np.pi * x0)
        x0 = x0 - (x0 + (u + c) * t - x) / (1.0 + t * (2.0 / (G - 1) + 1.0) * dc)
    return _state(x0)


def _cell_avg(x, dx, t):
    """Conserved-variable cell averages (the solution varies in x only)."""
    gx, gw = np.polynomial.legendre.leggauss(5)
    out = 0.0
    for q, wq in zip(gx, gw):
        rho, u, p = _exact(x + 0.5 * dx * q, t)
        z = np.zeros_like(rho)
        out = out + 0.5 * wq * np.stack([rho, rho * u, z, z, p / (G - 1) + 0.5 * rho * u * u])
    return out


def _away_from_extrema(x):
    return np.abs(np.cos(2 * np.pi * x)) > 0.5


def octree_errors(oracle, level):
    """Mean error of rho, rho u, E after one oracle step (its own CFL step) on the
    complete level-l octree."""
    dx = 1.0 / (1 << level)
    t = oracle.Tree(W.uniform_tree(level), level, (oracle.PERIODIC,) * 6)
    xyz, _ = t.cell_centres()
    u0 = _cell_avg(xyz[:, 0], dx, 0.0)
    u1, dt, st = t.step(u0, oracle.params(gamma=G, cfl=0.6))
    assert st == 0
    ue = _cell_avg(xyz[:, 0], dx, dt)
    m = (t.son < 0) & _away_from_extrema(xyz[:, 0])
    return np.array([np.mean(np.abs(u1[v, m] - ue[v, m])) for v in (0, 1, 4)])


def box_errors(oracle, N):
    """The same on a uniform N^3 box (the batch path), at a fixed dt = 0.25 dx."""
    dx = 1.0 / N
    i = np.arange(N ** 3) % N
    x = (i + 0.5) * dx
    u0 = _cell_avg(x, dx, 0.0)
    dt = 0.25 * dx
    u1, st = oracle.box_step(N, np.zeros(6, np.int32), u0, oracle.params(gamma=G, cfl=0.6), dt)
    assert st == 0
    ue = _cell_avg(x, dx, dt)
    m = _away_from_extrema(x)
    return np.array([np.mean(np.abs(u1[v, m] - ue[v, m])) for v in (0, 1, 4)])


def test_exact_solution_is_a_simple_wave():
    # the quadrature and Newton solve: at t = 0 the averages are those of the data, and the
    # backward invariant stays uniform at a later time
    x = np.linspace(0.0, 1.0, 101)
    rho, u, p = _exact(x, 0.3)
    c = np.sqrt(G * p / rho)
    assert np.ptp(u - 2 * c / (G - 1)) < 1e-12
    assert np.max(np.abs(p - rho ** G)) < 1e-12


def test_octree_step_local_error_is_third_order(oracle):
    e5, e6 = octree_errors(oracle, 5), octree_errors(oracle, 6)
    order = np.log2(e5 / e6)
    assert np.all(order > 2.8), (e5, e6, order)


def test_box_step_local_error_is_third_order(oracle):
    e5, e6 = box_errors(oracle, 32), box_errors(oracle, 64)
    order = np.log2(e5 / e6)
    assert np.all(order > 2.8), (e5, e6, order)
