"""Pins for the oracle's uniform-box step: for power-of-two boxes it equals the octree
oracle bit for bit; a Sedov blast in a non-power-of-two box has the self-similar radius;
a periodic box conserves mass, momentum and energy."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W


def _lex_of_tree(t, level):
    """Map level-`level` cells of an oracle tree to lexicographic indices."""
    n = 1 << level
    o0, o1 = int(t.lvl_off[level]), int(t.lvl_off[level + 1])
    c = np.arange(8)
    i = (2 * t.ix[o0:o1, None] + (c & 1)).ravel()
    j = (2 * t.iy[o0:o1, None] + ((c >> 1) & 1)).ravel()
    k = (2 * t.iz[o0:o1, None] + ((c >> 2) & 1)).ravel()
    return np.arange(8 * o0, 8 * o1), i + n * (j + n * k)


@pytest.mark.parametrize("bc,riemann", [((1,) * 6, 0), ((0,) * 6, 0), ((1,) * 6, 1)])
def test_box_step_equals_octree_step(oracle, bc, riemann):
    level, N = 4, 16
    t = oracle.Tree(W.uniform_tree(level), level, bc)
    xyz, _ = t.cell_centres()
    rng = np.random.default_rng(2)
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    Wp = np.empty((5, xyz.shape[0]))
    for v in range(5):
        Wp[v] = 0.3 * sum(np.sin(2 * np.pi * xyz[:, d] + ph[v, d]) for d in range(3))
    Wp[0] += 1.0; Wp[4] += 1.5
    prm = oracle.params(gamma=1.4, cfl=0.6, riemann=riemann)
    u = t.init_from_prim(Wp, prm)
    cells, lex = _lex_of_tree(t, level)
    ub = np.empty((5, N ** 3))
    ub[:, lex] = u[:, cells]
    dt_t = t.courant(u, prm)
    dt_b = oracle.box_courant(N, ub, prm)
    assert dt_t == dt_b
    un_t, dt2, st = t.step(u, prm)
    un_b, st_b = oracle.box_step(N, bc, ub, prm, dt_b)
    assert st == st_b == 0
    assert np.array_equal(un_b[:, lex], un_t[:, cells])


def test_box_sedov_radius_non_power_of_two(oracle):
    N = 48
    prm = oracle.params(gamma=1.4, cfl=0.8)
    u = np.empty((5, N ** 3))
    Wl = W.sedov_box_prims_lex(N)
    # conserved variables of the lexicographic Sedov data (v = 0)
    u[0] = Wl[0]; u[1:4] = 0.0; u[4] = Wl[4] / 0.4
    centre = (N // 2 + 0.5) / N
    tt, R = 0.0, 0.0
    while R < 0.3:
        dt = oracle.box_courant(N, u, prm)
        u, st = oracle.box_step(N, (1,) * 6, u, prm, dt)
        assert st == 0
        tt += dt
        R = 0.851 ** -0.2 * (tt * tt) ** 0.2
    i = np.arange(N ** 3)
    x = np.stack([i % N, (i // N) % N, i // (N * N)], axis=1)
    r = np.linalg.norm((x + 0.5) / N - centre, axis=1)
    bins = np.arange(0, 0.5, 1.0 / N)
    idx = np.digitize(r, bins)
    prof = np.array([u[0][idx == b].mean() if np.any(idx == b) else 0 for b in range(1, bins.size)])
    R_num = 0.5 * (bins[np.argmax(prof)] + bins[np.argmax(prof) + 1])
    assert abs(R_num - R) <= max(2.0 / N, 0.05 * R), (R_num, R)


def test_box_conservation_periodic(oracle):
    N = 24
    rng = np.random.default_rng(8)
    i = np.arange(N ** 3)
    x = np.stack([i % N, (i // N) % N, i // (N * N)], axis=1) / N
    u = np.empty((5, N ** 3))
    u[0] = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    u[1] = 0.2 * u[0]; u[2] = -0.1 * u[0]; u[3] = 0.3 * np.sin(2 * np.pi * x[:, 2])
    u[4] = 2.0 + 0.1 * np.cos(2 * np.pi * x[:, 2])
    prm = oracle.params(gamma=5 / 3, cfl=0.5)
    tot0 = u.sum(axis=1)
    for _ in range(4):
        u, st = oracle.box_step(N, (0,) * 6, u, prm, oracle.box_courant(N, u, prm))
    assert np.all(np.abs(u.sum(axis=1) - tot0) <= 1e-13 * 4 * np.abs(u).sum(axis=1))
