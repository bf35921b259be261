"""The seeded input generators (no GPU): each workload has the statistics and structure
that its recipe states, so that the CUDA path and the oracle are fed what the benchmark
claims."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W


def _shell_power(d):
    n = d.shape[0]
    p = np.abs(np.fft.fftn(d)) ** 2
    k1 = np.fft.fftfreq(n) * n
    k = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2)
    kb = np.rint(k).astype(int)
    return np.bincount(kb.ravel(), p.ravel()) / np.maximum(np.bincount(kb.ravel()), 1)


def test_grf_unit_variance_seeded_and_k_minus_4():
    d = W.grf(32, 7)
    assert abs(d.mean()) < 1e-12 and abs(d.std() - 1.0) < 1e-12
    assert np.array_equal(d, W.grf(32, 7)) and not np.array_equal(d, W.grf(32, 8))
    ps = _shell_power(d)
    k = np.arange(2, 13)
    slope = np.polyfit(np.log(k), np.log(ps[k]), 1)[0]
    assert abs(slope + 4.0) < 0.3, slope
    assert ps[0] < 1e-20                              # the k = 0 mode is removed


def test_turbulent_box_lognormal_density_and_mach_2():
    rho, v = W.turbulent_fields(4)
    assert rho.shape == (16, 16, 16) and v.shape == (3, 16, 16, 16)
    lr = np.log(rho)
    # rho = exp(sigma delta - sigma^2/2) with delta of zero mean and unit variance, sigma = 1
    assert abs(lr.mean() + 0.5) < 1e-12 and abs(lr.std() - 1.0) < 1e-12
    assert abs(np.sqrt(np.mean(np.sum(v * v, axis=0))) - 2.0) < 1e-12
    # three independent velocity fields: different seeds, nearly uncorrelated
    c = np.corrcoef(v.reshape(3, -1))
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 0.3)


def test_sod_states():
    xyz = np.array([[0.25, 0.5, 0.5], [0.75, 0.1, 0.9]])
    Wp = W.sod_prims(xyz)
    assert np.array_equal(Wp[:, 0], [1.0, 0.0, 0.0, 0.0, 1.0])
    assert np.array_equal(Wp[:, 1], [0.125, 0.0, 0.0, 0.0, 0.1])


def test_cell_centres_of_a_complete_level():
    lx = W.uniform_tree(3)
    xyz = W.cell_centres(lx[lx[:, 0] == 3])
    assert xyz.shape == (8 * 64, 3)
    g = np.sort(np.unique(np.round(xyz * 8 - 0.5, 12)))
    assert np.array_equal(g, np.arange(8))            # every level-3 cell centre, once per axis value
    assert len(np.unique(xyz, axis=0)) == 512


def test_sedov_batch_sizes():
    s = W.sedov_batch_sizes()
    assert s.shape == (48,) and np.array_equal(s, W.sedov_batch_sizes())
    assert set(np.unique(s)) <= set(range(32, 193, 16))
    assert len(np.unique(s)) >= 8                    # the draw spans the range


def test_box_layout_is_a_permutation():
    for N in (16, 48):
        p = W.box_batch_to_lex(N)
        assert np.array_equal(np.sort(p), np.arange(N ** 3))


def test_sedov_energy_in_one_cell():
    lx = W.uniform_tree(4)
    xyz = W.cell_centres(lx[lx[:, 0] == 4])
    Wp = W.sedov_prims(xyz, 4)
    hot = Wp[4] > 1e-5
    assert hot.sum() == 1
    # E = p / (gamma - 1) times the cell volume is the blast energy
    assert abs((Wp[4][hot][0] - 1e-5) / 0.4 / 16 ** 3 - 1.0) < 1e-12
    assert np.all(np.floor(xyz[hot] * 16) == 8)


@pytest.fixture(scope="module")
def plummer_small():
    return W.plummer_tree(base=4, lmax=7, nclump=8, seed=3)


def test_plummer_tree_balanced_and_complete_base(oracle, plummer_small):
    lx, _ = plummer_small
    assert oracle.Tree(lx, 4).ok                      # the oracle's geometric build accepts it (2:1)
    for l in range(1, 5):
        assert (lx[:, 0] == l).sum() == 8 ** (l - 1)  # levels 1-4 complete
    assert lx[:, 0].max() <= 7


def test_plummer_refinement_rule(plummer_small):
    """Every existing level-l cell (base <= l < lmax) whose centre density exceeds
    8^(l - base) is refined; balancing may refine more, never less."""
    lx, centres = plummer_small
    octs = {l: set(map(tuple, lx[lx[:, 0] == l][:, 1:4])) for l in range(1, 8)}
    for l in range(4, 7):
        cells = W.cell_centres(lx[lx[:, 0] == l])
        rho = W.plummer_density(cells, centres)
        ijk = np.floor(cells * (1 << l)).astype(int)
        need = ijk[rho > 8.0 ** (l - 4)]
        assert len(need) > 0 or l > 4
        for c in need:
            assert tuple(c) in octs[l + 1], (l, c)   # a refined level-l cell is a level-(l+1) oct
