"""Pins of the oracle's sub-cycled step (dt(l+1) = dt(l)/2, coarse first, time-interpolated
ghosts, refluxing over both fine steps): a single level reduces to the single-dt step bit
for bit, uniform flow stays uniform across levels, the leaf totals are conserved, the
time step has its closed form, and a smooth wave crossing refinement bands is as accurate
as with one time step for all levels (and more accurate than the coarse level alone)."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

PER = (0,) * 6


def band_tree(lmin, lfine):
    """Levels 1..lmin complete; finer levels over the band n/4 <= x < 3n/4 (oct units)."""
    levels = {l: W.full_level(l) for l in range(1, lmin + 1)}
    for l in range(lmin + 1, lfine + 1):
        n = 1 << (l - 1)
        g = np.arange(n)
        x, y, z = np.meshgrid(g, g, g, indexing="ij")
        sel = (x >= n // 4) & (x < 3 * n // 4)
        levels[l] = W._pack(x[sel], y[sel], z[sel])
    return W.to_lxyz(W.balance(levels, True))


def _totals(t, u):
    leaf = t.son < 0
    vol = np.ldexp(1.0, -3 * np.repeat(t.lvl, 8).astype(np.int64))[leaf]
    return np.array([np.sum(u[v, leaf] * vol) for v in range(5)])


def _wave(x, t=0.0, eps=0.2, g=1.4):
    Wp = W.uniform_prims(x, 1.0, (1.0, 0.0, 0.0), 1.0 / g)
    Wp[0] = 1 + eps * np.sin(2 * np.pi * (x[:, 0] - t))
    return Wp


def test_single_level_is_the_single_dt_step(oracle):
    t = oracle.Tree(W.uniform_tree(4), 4, PER)
    xyz, _ = t.cell_centres()
    prm = oracle.params(gamma=1.4, cfl=0.6)
    u = t.init_from_prim(_wave(xyz), prm)
    a, da, sa = t.step(u, prm)
    b, db, sb = t.step_subcycled(u, prm)
    assert sa == sb == 0 and da == db and np.array_equal(a, b)


@pytest.mark.parametrize("tree", ["band", "random"])
def test_uniform_flow_stays_uniform(oracle, tree):
    if tree == "band":
        lx, lmin = band_tree(4, 6), 4
    else:
        lx, lmin = W.random_tree(3, 2, seed=7, p_refine=0.3, periodic=True), 3
    t = oracle.Tree(lx, lmin, PER)
    assert t.levelmax >= lmin + 2
    xyz, _ = t.cell_centres()
    prm = oracle.params(gamma=5 / 3, cfl=0.8)
    u = t.init_from_prim(W.uniform_prims(xyz, 1.3, (0.4, -0.7, 0.2), 0.9), prm)
    un = u
    for _ in range(2):
        un, dt, st = t.step_subcycled(un, prm)
        assert st == 0
    for v in range(5):
        scale = np.max(np.abs(u[v])) + 1e-300
        assert np.max(np.abs(un[v] - u[v])) <= 1e-14 * scale, v


def test_conservation(oracle):
    lx = W.random_tree(3, 2, seed=11, p_refine=0.3, periodic=True)
    t = oracle.Tree(lx, 3, PER)
    xyz, _ = t.cell_centres()
    prm = oracle.params(gamma=5 / 3, cfl=0.5)
    rng = np.random.default_rng(3)
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    Wp = np.empty((5, xyz.shape[0]))
    for v in range(5):
        s = sum(np.sin(2 * np.pi * xyz[:, d] + ph[v, d]) for d in range(3))
        Wp[v] = s * (0.3 if v in (0, 4) else 0.5)
    Wp[0] += 1.0
    Wp[4] += 1.5
    u = t.init_from_prim(Wp, prm)
    tot0, scale = _totals(t, u), _totals(t, np.abs(u))
    for _ in range(3):
        u, dt, st = t.step_subcycled(u, prm)
        assert st == 0
    assert np.all(np.abs(_totals(t, u) - tot0) <= 1e-13 * scale)


def test_time_step_closed_form(oracle):
    """Uniform gas: every level allows the same Courant number, so the coarsest level's
    step is C dx_lmin / (3 c + sum |u|) however deep the tree goes."""
    t = oracle.Tree(band_tree(4, 6), 4, PER)
    xyz, _ = t.cell_centres()
    g, rho, p = 5 / 3, 1.3, 0.9
    vel = (0.4, -0.7, 0.2)
    prm = oracle.params(gamma=g, cfl=0.8)
    u = t.init_from_prim(W.uniform_prims(xyz, rho, vel, p), prm)
    c = np.sqrt(g * p / rho)
    expect = 0.8 * (1.0 / 16) / sum(abs(v) + c for v in vel)
    assert t.courant_levels(u, prm) == pytest.approx(expect, rel=1e-14)
    assert t.courant(u, prm) == pytest.approx(expect / 4, rel=1e-14)


def _wave_error(oracle, lx, lmin, subcycle, tf=0.1):
    t = oracle.Tree(lx, lmin, PER)
    xyz, lv = t.cell_centres()
    prm = oracle.params(gamma=1.4, cfl=0.6)
    u = t.init_from_prim(_wave(xyz), prm)
    tt = 0.0
    while tt < tf:
        u, dt, st = (t.step_subcycled if subcycle else t.step)(u, prm)
        assert st == 0
        tt += dt
    leaf = t.son < 0
    w = t.prim(u, prm)
    dx = np.ldexp(1.0, -lv)
    exact = 1 + 0.2 * np.sin(2 * np.pi * (xyz[:, 0] - tt)) * np.sinc(dx)
    vol = dx ** 3
    return np.sum(np.abs(w[0, leaf] - exact[leaf]) * vol[leaf]) / 0.2


def test_wave_through_refinement_bands(oracle):
    lx = band_tree(4, 5)
    e_sub = _wave_error(oracle, lx, 4, True)
    e_one = _wave_error(oracle, lx, 4, False)
    e_coarse = _wave_error(oracle, W.uniform_tree(4), 4, False)
    assert e_sub <= 1.1 * e_one, (e_sub, e_one)
    assert e_sub <= 0.8 * e_coarse, (e_sub, e_coarse)
