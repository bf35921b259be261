"""GPU parity of refinement between steps (refine_fine): amr_refine, amr_build_octree_device
and amr_remap_state against the oracle's refine_list and remap.

Tables of the refined tree: bit-exact.  Remapped state: copies bit-exact, interpolated
cells within 1e-12 of the oracle per field (the kernels may contract multiply-adds).
Leaf totals of the five conserved variables are unchanged to rounding."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_14631_gb300 import build
    build.build()
    from paper_2411_14631_gb300 import hydro
    return hydro


def _restricted_state(t, seed):
    rng = np.random.default_rng(seed)
    u = np.stack([np.exp(rng.normal(0, 0.7, t.ncell)), rng.normal(0, 1, t.ncell), rng.normal(0, 1, t.ncell),
                  rng.normal(0, 1, t.ncell), 3 + rng.random(t.ncell)])
    for l in range(t.levelmax - 1, 0, -1):
        for cell in range(t.lvl_off[l] * 8, t.lvl_off[l + 1] * 8):
            s = t.son[cell]
            if s >= 0:
                u[:, cell] = u[:, 8 * s:8 * s + 8].mean(axis=1)
    return u


def _check_tree(g, t):
    tab = {k: v.cpu().numpy() for k, v in g.tables().items()}
    for k in ("lvl", "ix", "iy", "iz", "son", "father", "nbor", "nb27"):
        assert np.array_equal(tab[k], getattr(t, k)), k
    assert np.array_equal(tab["key"].view(np.uint64), t.key)


def _leaf_totals(son, lvl_cell, u):
    leaf = son < 0
    vol = np.ldexp(1.0, -3 * lvl_cell[leaf].astype(np.int64))
    return np.array([np.sum(u[v, leaf] * vol) for v in range(5)]), \
        np.array([np.sum(np.abs(u[v, leaf]) * vol) for v in range(5)])


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_refine_matches_oracle(oracle, H, periodic, seed):
    import torch
    bc = (0,) * 6 if periodic else (1,) * 6
    lx = W.random_tree(3, 2, seed, p_refine=0.3, periodic=periodic)
    t = oracle.Tree(lx, 3, bc)
    g = H.Octree(lx, 3, bc)
    u = _restricted_state(t, seed)
    xyz, lv = t.cell_centres()
    thr = float(np.quantile(u[0] * np.ldexp(1.0, -3 * lv), 0.75))
    for lmax in (4, 6):
        new_o, st = t.refine_list(u, thr, lmax)
        assert st == oracle.OK
        t2 = oracle.Tree(new_o, 3, bc)
        assert t2.ok
        un_o, st = t.remap(u, t2)
        assert st == oracle.OK
        g2, un_g = g.refine(torch.tensor(u, device="cuda"), thr, lmax)
        assert g2.noct == t2.noct and g2.levelmax == t2.levelmax
        _check_tree(g2, t2)
        un_g = un_g.cpu().numpy()
        err = np.array([np.max(np.abs(un_g[v] - un_o[v])) / np.max(np.abs(un_o[v])) for v in range(5)])
        assert np.all(err <= 1e-12), err
        a, sa = _leaf_totals(t.son, np.repeat(t.lvl, 8), u)
        b, _ = _leaf_totals(t2.son, np.repeat(t2.lvl, 8), un_g)
        assert np.all(np.abs(a - b) <= 1e-13 * sa)


def test_refine_limits_and_errors(oracle, H):
    import ctypes as C
    import torch
    from paper_2411_14631_gb300 import abi
    lx = W.random_tree(3, 2, 9, p_refine=0.4)
    g = H.Octree(lx, 3, (0,) * 6)
    # light everywhere: back to the complete base levels; heavy: one more level everywhere
    u = torch.zeros((5, g.ncell), dtype=torch.float64, device="cuda")
    u[0] = 1e-3
    u[4] = 1.0
    g2, _ = g.refine(u, 1.0, 8)
    assert g2.noct == 1 + 8 + 64 and g2.levelmax == 3
    u[0] = 1e6
    g3, u3 = g.refine(u, 1e-9, 8)
    assert g3.noct == 1 + g.ncell
    assert torch.all(u3[0] == 1e6)               # a uniform state stays uniform
    # argument errors come back as statuses, before any launch
    L = abi.lib()
    rp = abi.RefineParams(1.0, 2, 0)             # levelmax below levelmin
    cnt = (C.c_int64 * (abi.MAXLEV + 1))()
    n = C.c_int64()
    assert L.amr_refine(C.byref(g.t), C.byref(rp), C.c_void_p(u.data_ptr()), C.c_void_p(u.data_ptr()), 1 << 30,
                        C.c_void_p(u.data_ptr()), g.ncell + 1, cnt, C.byref(n), None) == abi.EINVAL
    rp.levelmax = 6
    assert L.amr_refine(C.byref(g.t), C.byref(rp), C.c_void_p(u.data_ptr()), C.c_void_p(u.data_ptr()), 1 << 30,
                        C.c_void_p(u.data_ptr()), g.ncell, cnt, C.byref(n), None) == abi.ECAPACITY
    # a device list whose level counts disagree with the list is rejected
    geom = abi.AmrGeom(3, (C.c_int32 * 6)(*(0,) * 6))
    lxd = torch.tensor(W.uniform_tree(3), dtype=torch.int32, device="cuda")
    good = (C.c_int64 * (abi.MAXLEV + 1))(*([0, 1, 8, 64] + [0] * (abi.MAXLEV - 3)))
    bad = (C.c_int64 * (abi.MAXLEV + 1))(*([0, 1, 8, 63, 1] + [0] * (abi.MAXLEV - 4)))
    tb, wb = C.c_size_t(), C.c_size_t()
    assert L.amr_build_octree_device_query(C.byref(geom), good, C.byref(tb), C.byref(wb)) == abi.OK
    mem = torch.empty(tb.value + (1 << 20), dtype=torch.uint8, device="cuda")
    ws = torch.empty(wb.value + (1 << 20), dtype=torch.uint8, device="cuda")
    out = abi.AmrTree()
    assert L.amr_build_octree_device(C.byref(geom), C.c_void_p(lxd.data_ptr()), bad, C.c_void_p(mem.data_ptr()),
                                     mem.numel(), C.c_void_p(ws.data_ptr()), ws.numel(), C.byref(out),
                                     None) == abi.EINVAL
    assert L.amr_build_octree_device(C.byref(geom), C.c_void_p(lxd.data_ptr()), good, C.c_void_p(mem.data_ptr()),
                                     mem.numel(), C.c_void_p(ws.data_ptr()), ws.numel(), C.byref(out),
                                     None) == abi.OK
    assert out.noct == 73


def test_refine_plummer_full_size(oracle, H):
    """The Plummer-clump AMR mesh (levels 7-12, 2.7 M octs) after ten FP32 steps, refined
    by the rule it was built with (rho dx^3 > dx_7^3): the new tree and state against the
    oracle, and the leaf totals."""
    import torch
    from paper_2411_14631_gb300 import abi
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx, centres = W.plummer_tree()
    g = H.Octree(lx, 7, (0,) * 6)
    w0 = W.plummer_prims(cell_centres_of(g), centres)
    sim = H.Simulation(g, H.Params(5.0 / 3.0, cfl=0.8, precision=abi.PREC_FP32), w0=w0)
    for _ in range(10):
        sim.step()
    u = sim.u.clone()
    thr = 2.0 ** -21
    g2, un_g = g.refine(u, thr, 12)
    uh = u.cpu().numpy()
    t = oracle.Tree(lx, 7, (0,) * 6)
    assert t.noct == g.noct
    new_o, st = t.refine_list(uh, thr, 12)
    assert st == oracle.OK
    t2 = oracle.Tree(new_o, 7, (0,) * 6)
    _check_tree(g2, t2)
    un_o, st = t.remap(uh, t2)
    un_g = un_g.cpu().numpy()
    err = np.array([np.max(np.abs(un_g[v] - un_o[v])) / np.max(np.abs(un_o[v])) for v in range(5)])
    assert np.all(err <= 1e-12), err
    a, sa = _leaf_totals(t.son, np.repeat(t.lvl, 8), uh)
    b, _ = _leaf_totals(t2.son, np.repeat(t2.lvl, 8), un_g)
    assert np.all(np.abs(a - b) <= 1e-13 * sa)
    assert g2.noct != g.noct                      # the mesh moved with the gas
