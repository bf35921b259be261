"""Pins for the oracle's octree: the Hilbert key is a hierarchical Hilbert curve, and the
son / father / nbor / nb27 tables agree with a brute-force dictionary search on small
random balanced octrees."""
import itertools

import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W


@pytest.mark.parametrize("bits", [1, 2, 3, 4, 5])
def test_hilbert_bijection_and_adjacency(oracle, bits):
    n = 1 << bits
    inv = {}
    for x, y, z in itertools.product(range(n), repeat=3):
        k = oracle.hilbert_key(bits, x, y, z)
        assert 0 <= k < n ** 3 and k not in inv
        inv[k] = (x, y, z)
    assert len(inv) == n ** 3
    for k in range(n ** 3 - 1):
        a, b = np.array(inv[k]), np.array(inv[k + 1])
        assert np.abs(a - b).sum() == 1          # consecutive cells share a face
    assert inv[0] == (0, 0, 0)


@pytest.mark.parametrize("bits", [2, 3, 4, 6])
def test_hilbert_prefix_property(oracle, bits):
    rng = np.random.default_rng(bits)
    n = 1 << bits
    for x, y, z in rng.integers(0, n, (300, 3)):
        k = oracle.hilbert_key(bits, int(x), int(y), int(z))
        kp = oracle.hilbert_key(bits - 1, int(x) >> 1, int(y) >> 1, int(z) >> 1)
        assert k >> 3 == kp


def _brute_tables(t):
    """Recompute the tables with a dict of (level, ix, iy, iz) -> oct id."""
    ids = {(int(l), int(x), int(y), int(z)): i for i, (l, x, y, z) in enumerate(zip(t.lvl, t.ix, t.iy, t.iz))}
    n = t.noct
    son = np.full(8 * n, -1, np.int64); father = np.full(n, -1, np.int64)
    nbor = np.full(6 * n, -1, np.int64); nb27 = np.zeros(27 * n, np.int64)

    def cell(l, X, Y, Z):
        o = ids.get((l, X >> 1, Y >> 1, Z >> 1))
        return None if o is None else o * 8 + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1)

    def wrap(l, P):
        m = 1 << l
        out = []
        for a, c in enumerate(P):
            if 0 <= c < m:
                out.append(c)
            elif t.bc[2 * a + (1 if c >= m else 0)] == 0:
                out.append(c % m)
            else:
                return None
        return out

    for (l, x, y, z), o in ids.items():
        for c in range(8):
            s = ids.get((l + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1)))
            son[8 * o + c] = -1 if s is None else s
        if l == 1:
            nb27[27 * o:27 * o + 27] = -(2 ** 31)
            nb27[27 * o + 13] = o
            continue
        father[o] = cell(l - 1, x, y, z)
        for k in range(6):
            P = [x, y, z]; P[k // 2] += 1 if k & 1 else -1
            P = wrap(l - 1, P)
            nbor[6 * o + k] = -1 if P is None else cell(l - 1, *P)
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
            P = wrap(l - 1, [x + dx, y + dy, z + dz])
            if P is None:
                nb27[27 * o + k] = -(2 ** 31); continue
            s = ids.get((l, *P))
            nb27[27 * o + k] = s if s is not None else -1 - cell(l - 1, *P)
    return son, father, nbor, nb27


@pytest.mark.parametrize("seed", range(12))
def test_tables_match_brute_force(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    base = int(rng.integers(2, 4)); extra = int(rng.integers(1, 4))
    periodic = bool(seed % 2)
    lx = W.random_tree(base, extra, seed, p_refine=0.25, periodic=periodic)
    bc = (0,) * 6 if periodic else (1,) * 6
    t = oracle.Tree(lx, base, bc)
    assert t.ok, t.status
    # numbering: by level, then Hilbert key
    order = np.lexsort((t.key, t.lvl))
    assert np.array_equal(order, np.arange(t.noct))
    for i in range(0, t.noct, max(1, t.noct // 50)):
        assert t.key[i] == oracle.hilbert_key(int(t.lvl[i]) - 1, int(t.ix[i]), int(t.iy[i]), int(t.iz[i]))
    son, father, nbor, nb27 = _brute_tables(t)
    assert np.array_equal(t.son, son)
    assert np.array_equal(t.father, father)
    assert np.array_equal(t.nbor, nbor)
    assert np.array_equal(t.nb27, nb27)
    assert t.lvl_off[base] == sum(8 ** (l - 1) for l in range(1, base))


def test_unbalanced_tree_rejected(oracle):
    # level 3 complete, one level-4 oct, and a level-5 oct two father cells away from
    # any level-4 oct: its father's neighbours are missing at level 4
    levels = {l: W.full_level(l) for l in range(1, 4)}
    levels[4] = W._pack(np.array([0]), np.array([0]), np.array([0]))
    levels[5] = W._pack(np.array([1]), np.array([1]), np.array([1]))
    t = oracle.Tree(W.to_lxyz(levels), 3)
    assert t.status == oracle.EUNBALANCED


def test_invalid_inputs_rejected(oracle):
    lx = W.uniform_tree(3)
    assert oracle.Tree(lx[:-1], 3).status == oracle.EINVAL          # level 3 incomplete
    dup = np.concatenate([lx, lx[-1:]])
    assert oracle.Tree(dup, 3).status == oracle.EINVAL              # duplicate oct
    bad = lx.copy(); bad[-1, 1] = 99
    assert oracle.Tree(bad, 3).status == oracle.EINVAL              # coordinate out of range
    assert oracle.Tree(lx, 3, (0, 1, 0, 0, 0, 0)).status == oracle.EINVAL   # half-periodic axis
