"""Pins of the oracle's refinement step (refine_fine, Table 1): the new oct set against an
independent set-based construction (the mass criterion, then the 2:1 closure of
``workloads.balance``), limiting cases, conservation of the leaf totals, exact copies
of surviving cells, and linear fields reproduced by the interpolation of new cells."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W


def _tree(oracle, lxyz, levelmin, periodic=True):
    bc = (oracle.PERIODIC if periodic else oracle.OUTFLOW,) * 6
    t = oracle.Tree(lxyz, levelmin, bc)
    assert t.ok
    return t


def _state(t, rho):
    u = np.zeros((5, t.ncell))
    u[0] = rho
    u[1] = 0.3 * rho
    u[4] = 2.0 + rho
    return u


def _set(lxyz):
    return {tuple(int(v) for v in r) for r in np.asarray(lxyz)}


def _brute(t, u, thr, lmax, periodic):
    """Children of every cell that passes the mass test, levels 1..levelmin complete,
    then the 2:1 closure."""
    xyz, lv = t.cell_centres()
    dx = np.ldexp(1.0, -lv)
    flag = (lv >= t.levelmin) & (lv < lmax) & (u[0] * dx ** 3 > thr)
    levels = {l: W.full_level(l) for l in range(1, t.levelmin + 1)}
    X = np.floor(xyz / dx[:, None]).astype(np.int64)
    for l in range(t.levelmin, lmax):
        sel = flag & (lv == l)
        if sel.any():
            kids = W._pack(X[sel, 0], X[sel, 1], X[sel, 2])
            levels[l + 1] = np.unique(np.concatenate([levels.get(l + 1, np.empty(0, np.int64)), kids]))
    return _set(W.to_lxyz(W.balance(levels, periodic)))


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_new_octs_match_set_construction(oracle, periodic, seed):
    lx = W.random_tree(3, 2, seed, p_refine=0.3, periodic=periodic)
    t = _tree(oracle, lx, 3, periodic)
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.normal(0.0, 1.0, t.ncell))
    xyz, lv = t.cell_centres()
    thr = np.quantile(rho * np.ldexp(1.0, -3 * lv), 0.8)
    u = _state(t, rho)
    for lmax in (4, 5, 6):
        new, st = t.refine_list(u, thr, lmax)
        assert st == oracle.OK
        assert len(new) == len(_set(new))
        assert _set(new) == _brute(t, u, thr, lmax, periodic)
        t2 = oracle.Tree(new, 3, t.bc)
        assert t2.ok, "refined tree must satisfy the 2:1 rule"
        assert t2.levelmax <= lmax


def test_limiting_cases(oracle):
    lx = W.random_tree(3, 2, 7, p_refine=0.4)
    t = _tree(oracle, lx, 3)
    # everything light: back to the complete base levels
    new, st = t.refine_list(_state(t, np.full(t.ncell, 1e-3)), 1.0, 8)
    assert st == oracle.OK and _set(new) == _set(W.uniform_tree(3))
    # everything heavy: every existing cell below lmax is refined, one level per call
    new, st = t.refine_list(_state(t, np.full(t.ncell, 1e6)), 1e-9, 8)
    xyz, lv = t.cell_centres()
    assert st == oracle.OK and len(new) == 1 + t.ncell
    new, st = t.refine_list(_state(t, np.full(t.ncell, 1e6)), 1e-9, 4)
    assert _set(new) == _set(W.uniform_tree(4))
    # bad arguments
    _, st = t.refine_list(_state(t, np.ones(t.ncell)), 1.0, 2)
    assert st == oracle.EINVAL


@pytest.mark.parametrize("periodic", [True, False])
def test_remap_conserves_and_copies(oracle, periodic):
    lx = W.random_tree(3, 2, 11, p_refine=0.35, periodic=periodic)
    t = _tree(oracle, lx, 3, periodic)
    rng = np.random.default_rng(5)
    u = np.stack([np.exp(rng.normal(0, 0.5, t.ncell)), rng.normal(0, 1, t.ncell), rng.normal(0, 1, t.ncell),
                  rng.normal(0, 1, t.ncell), 3 + rng.random(t.ncell)])
    # restricted state (refined cells hold the mean of their children), as after a step
    for l in range(t.levelmax - 1, 0, -1):
        for cell in range(t.lvl_off[l] * 8, t.lvl_off[l + 1] * 8):
            s = t.son[cell]
            if s >= 0:
                u[:, cell] = u[:, 8 * s:8 * s + 8].mean(axis=1)
    xyz, lv = t.cell_centres()
    thr = np.quantile(u[0] * np.ldexp(1.0, -3 * lv), 0.75)
    new, st = t.refine_list(u, thr, 6)
    t2 = oracle.Tree(new, 3, t.bc)
    un, st = t.remap(u, t2)
    assert st == oracle.OK

    def totals(tree, uu):
        xyz_, lv_ = tree.cell_centres()
        leaf = tree.son < 0
        vol = np.ldexp(1.0, -3 * lv_)
        return np.array([np.sum(uu[v, leaf] * vol[leaf]) for v in range(5)]), \
            np.array([np.sum(np.abs(uu[v, leaf]) * vol[leaf]) for v in range(5)])

    a, sa = totals(t, u)
    b, _ = totals(t2, un)
    assert np.all(np.abs(a - b) <= 1e-14 * sa)
    # surviving cells keep their state bit for bit
    old = {(int(l), *(int(c) for c in np.floor(x / np.ldexp(1.0, -l)))): i for i, (x, l) in enumerate(zip(xyz, lv))}
    xyz2, lv2 = t2.cell_centres()
    kept = 0
    for j, (x, l) in enumerate(zip(xyz2, lv2)):
        key = (int(l), *(int(c) for c in np.floor(x / np.ldexp(1.0, -l))))
        if key in old:
            assert np.array_equal(un[:, j], u[:, old[key]])
            kept += 1
    assert 0 < kept < t2.ncell


def test_new_cells_reproduce_linear_field(oracle):
    """Refining interior cells of a linear density field: both one-sided differences
    agree, so MinMod keeps the slope and each child gets the field's value at its own
    centre."""
    t = _tree(oracle, W.uniform_tree(3), 3)
    xyz, lv = t.cell_centres()
    rho = 2.0 + 0.5 * xyz[:, 0] - 0.25 * xyz[:, 1] + 0.125 * xyz[:, 2]
    u = _state(t, rho)
    # the criterion sees a heavy interior block of level-3 cells (centres 0.3125..0.6875)
    heavy = (np.abs(xyz - 0.5) < 0.2).all(axis=1) & (lv == 3)
    flag_u = u.copy()
    flag_u[0] = np.where(heavy, 100.0 * rho, rho)
    new, st = t.refine_list(flag_u, 0.2, 4)
    assert st == oracle.OK and len(new) == 1 + 8 + 64 + 64
    t2 = oracle.Tree(new, 3, t.bc)
    un, st = t.remap(u, t2)
    assert st == oracle.OK
    xyz2, lv2 = t2.cell_centres()
    fine = lv2 == 4
    expect = 2.0 + 0.5 * xyz2[:, 0] - 0.25 * xyz2[:, 1] + 0.125 * xyz2[:, 2]
    assert fine.sum() == 512
    assert np.allclose(un[0, fine], expect[fine], rtol=0, atol=1e-14)
