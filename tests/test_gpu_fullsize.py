"""Full-size parity: one step of the benchmark workloads in the launch configuration
bench.py times (all levels in one launch), compared with the oracle cell by cell.

* Turbulent periodic box 256^3 (16.8 M cells, levels 1-8).
* Plummer-clump AMR mesh, base level 7 refined to level 12 (2.7 M octs, 1.9e7 leaves).

FP64 path: per field max|gpu - oracle| / max|oracle| <= 1e-12 over every cell, and the
same time step.  FP32 path: relative L1 of each conserved field within 1e-4, that is the
FP32 unit round-off (6e-8) times the cancellation |F| / |F_left - F_right| of a cell's
flux difference, up to about 1e3 in these workloads (momenta start at zero next to
1e4 density contrasts)."""
import os

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


def _one_step_parity(oracle, H, lx, levelmin, bc, w_of_xyz, gamma):
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    t = oracle.Tree(lx, levelmin, bc)
    assert t.ok
    g = H.Octree(lx, levelmin, bc)
    xyz, _ = t.cell_centres()
    assert np.array_equal(cell_centres_of(g), xyz)          # same cell order on both sides
    w0 = w_of_xyz(xyz)
    prm_o = oracle.params(gamma=gamma, cfl=0.8)
    u0 = t.init_from_prim(w0, prm_o)
    u1, dt_o, st = t.step(u0, prm_o)
    assert st == 0
    out = {}
    for precision in (0, 1):
        prm = H.Params(gamma, cfl=0.8, precision=precision)
        sim = H.Simulation(g, prm, w0=w0)
        dt_g = float(sim.dt.item())
        sim.step()
        torch.cuda.synchronize()
        ug = sim.u.cpu().numpy()
        out[precision] = (ug, dt_g)
        assert prm.read_status()[0] == 0
    ug, dt_g = out[0]
    assert abs(dt_g - dt_o) <= 1e-14 * dt_o
    for v in range(5):
        err = np.max(np.abs(ug[v] - u1[v])) / np.max(np.abs(u1[v]))
        assert err <= 1e-12, (v, err)
    ug32, dt32 = out[1]
    assert dt32 <= dt_o and dt32 >= dt_o * (1 - 1e-4)
    leaf = t.son < 0
    for v in range(5):
        l1 = np.abs(ug32[v, leaf] - u1[v, leaf]).sum() / (np.abs(u1[v, leaf]).sum() + 1e-300)
        assert l1 <= 1e-4, (v, l1)


def test_turbulent_box_256_one_step(oracle, H):
    lx = W.uniform_tree(8)
    rho, v = W.turbulent_fields(8)
    _one_step_parity(oracle, H, lx, 8, (0,) * 6, lambda xyz: W.grid_prims(xyz, 8, rho, v), 5.0 / 3.0)


def test_plummer_amr_one_step(oracle, H):
    lx, centres = W.plummer_tree()
    _one_step_parity(oracle, H, lx, 7, (0,) * 6, lambda xyz: W.plummer_prims(xyz, centres), 5.0 / 3.0)
