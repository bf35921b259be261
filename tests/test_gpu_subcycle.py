"""GPU parity of the sub-cycled step (hydro_step_subcycled) with the oracle's
or_step_subcycled: FP64 fields within 1e-12 per field (max norm, relative), the coarsest
level's step within 1e-14; uniform flow, conservation, graph replay and the reduction
to hydro_step on one level."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

pytestmark = pytest.mark.gpu
PER, OUT = (0,) * 6, (1,) * 6


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_14631_gb300 import build
    build.build()
    from paper_2411_14631_gb300 import hydro
    return hydro


def _smooth(xyz, seed):
    rng = np.random.default_rng(seed)
    Wp = np.empty((5, xyz.shape[0]))
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    for v in range(5):
        s = sum(np.sin(2 * np.pi * xyz[:, d] + ph[v, d]) for d in range(3))
        Wp[v] = s * (0.3 if v in (0, 4) else 0.5)
    Wp[0] += 1.0
    Wp[4] += 1.5
    return Wp


def _relerr(a, b):
    return np.array([np.max(np.abs(a[v] - b[v])) / max(np.max(np.abs(b[v])), 1e-300) for v in range(5)])


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("seed", [1, 2])
def test_subcycled_matches_oracle(oracle, H, periodic, seed):
    bc = PER if periodic else OUT
    lx = W.random_tree(3, 3, seed, p_refine=0.3, periodic=periodic)
    t = oracle.Tree(lx, 3, bc)
    assert t.levelmax >= 5
    g = H.Octree(lx, 3, bc)
    xyz, _ = t.cell_centres()
    w0 = _smooth(xyz, seed)
    prm_o = oracle.params(gamma=5 / 3, cfl=0.6)
    u_o = t.init_from_prim(w0, prm_o)
    sim = H.SubcycledSimulation(g, H.Params(5 / 3, cfl=0.6), w0=w0)
    for _ in range(2):
        u_o, dt_o, st = t.step_subcycled(u_o, prm_o)
        assert st == 0
        sim.step()
        assert sim.dt.item() == pytest.approx(dt_o, rel=1e-14)
    err = _relerr(sim.u.cpu().numpy(), u_o)
    assert np.all(err <= 1e-12), err


def test_single_level_equals_hydro_step(H):
    import torch
    g = H.Octree(W.uniform_tree(5), 5, PER)
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    w0 = _smooth(cell_centres_of(g), 4)
    prm = H.Params(1.4, cfl=0.7)
    a = H.SubcycledSimulation(g, prm, w0=w0)
    b = H.Simulation(g, prm, w0=w0)
    for _ in range(3):
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert torch.equal(a.u, b.u)


def test_uniform_flow_conservation_and_graph(H):
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx = W.random_tree(3, 3, 5, p_refine=0.3, periodic=True)
    g = H.Octree(lx, 3, PER)
    xyz = cell_centres_of(g)
    prm = H.Params(5 / 3, cfl=0.8)
    sim = H.SubcycledSimulation(g, prm, w0=W.uniform_prims(xyz, 1.3, (0.4, -0.7, 0.2), 0.9))
    u0 = sim.u.clone()
    for _ in range(2):
        sim.step()
    for v in range(5):
        scale = torch.max(torch.abs(u0[v])).item()
        assert torch.max(torch.abs(sim.u[v] - u0[v])).item() <= 1e-14 * scale
    # conservation of the leaf totals, and graph replays equal to eager steps
    tab = g.tables()
    leaf = (tab["son"] < 0).cpu().numpy()
    vol = np.ldexp(1.0, -3 * np.repeat(tab["lvl"].cpu().numpy(), 8).astype(np.int64))[leaf]
    w0 = _smooth(xyz, 9)
    e = H.SubcycledSimulation(g, prm, w0=w0)
    r = H.SubcycledSimulation(g, prm, w0=w0).use_graph()
    e.step()                                  # use_graph made one eager step
    ue = e.u.cpu().numpy()
    tot0 = np.array([np.sum(ue[v, leaf] * vol) for v in range(5)])
    scale = np.array([np.sum(np.abs(ue[v, leaf]) * vol) for v in range(5)])
    for _ in range(3):
        e.step()
        r.step()
    torch.cuda.synchronize()
    assert torch.equal(e.u, r.u)
    ue = e.u.cpu().numpy()
    tot = np.array([np.sum(ue[v, leaf] * vol) for v in range(5)])
    assert np.all(np.abs(tot - tot0) <= 1e-13 * scale)


def test_fp32_path_close_to_oracle(oracle, H):
    from paper_2411_14631_gb300 import abi
    lx = W.random_tree(3, 2, 3, p_refine=0.35, periodic=True)
    t = oracle.Tree(lx, 3, PER)
    g = H.Octree(lx, 3, PER)
    xyz, _ = t.cell_centres()
    w0 = _smooth(xyz, 6)
    prm_o = oracle.params(gamma=5 / 3, cfl=0.6)
    u_o = t.init_from_prim(w0, prm_o)
    sim = H.SubcycledSimulation(g, H.Params(5 / 3, cfl=0.6, precision=abi.PREC_FP32), w0=w0)
    u_o, _, _ = t.step_subcycled(u_o, prm_o)
    sim.step()
    u = sim.u.cpu().numpy()
    l1 = np.abs(u[0] - u_o[0]).sum() / np.abs(u_o[0]).sum()
    assert l1 <= 1e-5, l1


def test_plummer_full_size_one_step(oracle, H):
    """The Plummer-clump mesh (levels 7-12): one coarse step is 32 steps of level 12; FP64
    against the oracle on every cell."""
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx, centres = W.plummer_tree()
    g = H.Octree(lx, 7, PER)
    w0 = W.plummer_prims(cell_centres_of(g), centres)
    t = oracle.Tree(lx, 7, PER)
    prm_o = oracle.params(gamma=5 / 3, cfl=0.8)
    u_o = t.init_from_prim(w0, prm_o)
    sim = H.SubcycledSimulation(g, H.Params(5 / 3, cfl=0.8), w0=w0)
    u_o, dt_o, st = t.step_subcycled(u_o, prm_o)
    assert st == 0
    sim.step()
    assert sim.dt.item() == pytest.approx(dt_o, rel=1e-14)
    err = _relerr(sim.u.cpu().numpy(), u_o)
    assert np.all(err <= 1e-12), err
