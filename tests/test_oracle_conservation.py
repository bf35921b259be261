"""Pins for the oracle's leaf totals (the global conservation diagnostics): closed forms
that a wrong volume weight, a refined cell counted as a leaf, a dropped cell or a
dropped variable would each break."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W


@pytest.fixture(scope="module")
def amr_tree(oracle):
    return oracle.Tree(W.random_tree(3, 3, 41, p_refine=0.35, periodic=True), 3, (0,) * 6)


def test_uniform_state_totals_are_the_state(oracle, amr_tree):
    """The leaves tile the unit box, so a uniform U has totals U (exactly: every U dV is a
    dyadic product and the sums are exactly rounded); |U| for the absolute totals."""
    t = amr_tree
    assert t.levelmax >= 5
    U = np.array([1.25, -0.5, 0.75, -3.0, 7.5])
    u = np.repeat(U[:, None], t.ncell, axis=1)
    tot = t.conservation_totals(u)
    assert np.array_equal(tot[0], U)
    assert np.array_equal(tot[1], np.abs(U))


def test_linear_field_integrates_exactly(oracle, amr_tree):
    """U = x (and y, z, x + y + z) at the cell centres integrates to 1/2 (3/2): the
    midpoint rule is exact for linear fields on every cell of any size, so the volume
    weights must be the cells' own."""
    t = amr_tree
    xyz, _ = t.cell_centres()
    u = np.stack([xyz[:, 0], xyz[:, 1], xyz[:, 2], xyz.sum(axis=1), 1.0 - xyz[:, 0]])
    tot = t.conservation_totals(u)
    assert np.array_equal(tot[0], [0.5, 0.5, 0.5, 1.5, 0.5])


def test_refined_cells_do_not_count(oracle, amr_tree):
    """Values in refined cells (whose children are the leaves) do not enter the totals."""
    t = amr_tree
    rng = np.random.default_rng(3)
    u = rng.standard_normal((5, t.ncell))
    ref = t.son >= 0
    assert ref.sum() > 0
    a = t.conservation_totals(u)
    u[:, ref] = 1e30
    b = t.conservation_totals(u)
    assert np.array_equal(a, b)


def test_single_leaf_weight(oracle, amr_tree):
    """One non-zero leaf cell at level l gives totals U 2^-3l: the weight of each level."""
    t = amr_tree
    leaf = np.nonzero(t.son < 0)[0]
    lv = np.repeat(t.lvl, 8)
    levels = [l for l in range(t.levelmin, t.levelmax + 1) if np.any(lv[leaf] == l)]
    assert len(levels) >= 3
    for l in levels:
        c = leaf[lv[leaf] == l][0]
        u = np.zeros((5, t.ncell))
        u[:, c] = [1.0, 2.0, -3.0, 4.0, 5.0]
        tot = t.conservation_totals(u)
        assert np.array_equal(tot[0], np.array([1.0, 2.0, -3.0, 4.0, 5.0]) * 2.0 ** (-3 * l)), l


def test_box_totals(oracle):
    """Uniform boxes of N^3 cells: a uniform U gives U (to one rounding of the division
    by N^3); a single cell of value N^3 gives 1 in its own box and 0 in the others."""
    sizes = [12, 16, 20]
    n = [s ** 3 for s in sizes]
    U = np.array([1.1, -0.3, 0.2, 0.0, 2.5])
    u = np.repeat(U[:, None], sum(n), axis=1)
    tot = oracle.box_conservation_totals(sizes, u)
    for b in range(3):
        assert np.allclose(tot[b, 0], U, rtol=2e-16, atol=0)
        assert np.allclose(tot[b, 1], np.abs(U), rtol=2e-16, atol=0)
    u = np.zeros((5, sum(n)))
    u[:, n[0] + 5] = n[1]
    tot = oracle.box_conservation_totals(sizes, u)
    assert np.array_equal(tot[1, 0], np.ones(5)) and np.all(tot[0] == 0) and np.all(tot[2] == 0)
