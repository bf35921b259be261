"""Pins of the monotonized central slope limiter (van Leer 1977) of the reconstruction:
its closed forms, and that it is less dissipative than MinMod where it should be (the
Sod tube and a smooth wave are closer to their exact solutions)."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

OUT, PER = (1,) * 6, (0,) * 6


@pytest.mark.parametrize("a,b,expect", [(1.0, 2.0, 1.5), (1.0, 4.0, 2.0), (4.0, 1.0, 2.0), (1.0, 1.0, 1.0),
                                        (-1.0, -0.1, -0.2), (1.0, -1.0, 0.0), (0.0, 3.0, 0.0), (-2.0, -2.5, -2.25)])
def test_mc_closed_forms(oracle, a, b, expect):
    assert oracle.mc(a, b) == expect
    assert oracle.mc(b, a) == expect
    assert oracle.mc(-a, -b) == -expect


def test_mc_between_minmod_and_twice_minmod(oracle):
    rng = np.random.default_rng(1)
    for a, b in rng.normal(size=(200, 2)):
        m, c = oracle.minmod(a, b), oracle.mc(a, b)
        if a * b > 0:
            assert abs(m) <= abs(c) <= 2 * abs(m) + 1e-15 and np.sign(c) == np.sign(a)
        else:
            assert c == 0.0


def _sod_l1(oracle, limiter, level=5, nsteps=20):
    t = oracle.Tree(W.uniform_tree(level), level, OUT)
    xyz, _ = t.cell_centres()
    prm = oracle.params(gamma=1.4, cfl=0.8, limiter=limiter)
    u = t.init_from_prim(W.sod_prims(xyz, 0), prm)
    tf = 0.0
    for _ in range(nsteps):
        u, dt, st = t.step(u, prm)
        assert st == 0
        tf += dt
    WL = np.array([1.0, 0, 0, 0, 1.0]); WR = np.array([0.125, 0, 0, 0, 0.1])
    ps, us, _, _ = oracle.exact_star(WL, WR, 1.4)
    leaf = t.son < 0
    n = 1 << level
    xs = np.sort(np.unique(xyz[leaf, 0]))
    q = (np.arange(64) + 0.5) / 64 - 0.5
    ex = np.array([np.mean([oracle.exact_sample(WL, WR, 1.4, ps, us, (x + qq / n - 0.5) / tf)[0] for qq in q])
                   for x in xs])
    w = t.prim(u, prm)
    rho = np.array([w[0, leaf][xyz[leaf, 0] == x][0] for x in xs])
    return np.mean(np.abs(rho - ex)) / np.mean(ex)


def test_mc_sharper_on_sod(oracle):
    e_mm = _sod_l1(oracle, oracle.LIMITER_MINMOD)
    e_mc = _sod_l1(oracle, oracle.LIMITER_MC)
    assert e_mc < 0.9 * e_mm, (e_mc, e_mm)


def _wave_err(oracle, limiter, level):
    t = oracle.Tree(W.uniform_tree(level), level, PER)
    xyz, lv = t.cell_centres()
    prm = oracle.params(gamma=1.4, cfl=0.6, limiter=limiter)

    def prims(x, tt=0.0):
        Wp = W.uniform_prims(x, 1.0, (1.0, 0.0, 0.0), 1.0 / 1.4)
        Wp[0] = 1 + 0.2 * np.sin(2 * np.pi * (x[:, 0] - tt))
        return Wp

    u = t.init_from_prim(prims(xyz), prm)
    tt = 0.0
    while tt < 0.1:
        u, dt, st = t.step(u, prm)
        tt += dt
    leaf = t.son < 0
    w = t.prim(u, prm)
    exact = 1 + 0.2 * np.sin(2 * np.pi * (xyz[:, 0] - tt)) * np.sinc(1.0 / (1 << level))
    return np.mean(np.abs(w[0, leaf] - exact[leaf])) / 0.2


def test_mc_smooth_wave(oracle):
    e4 = _wave_err(oracle, oracle.LIMITER_MC, 4)
    e5 = _wave_err(oracle, oracle.LIMITER_MC, 5)
    assert np.log2(e4 / e5) > 1.7, (e4, e5)
    assert e5 < _wave_err(oracle, oracle.LIMITER_MINMOD, 5)
