"""The restriction of the complete levels deferred out of hydro_step
(hydro_params.defer_restriction) and run by hydro_restrict_complete: through the C ABI
on one stream, and overlapped with the next step on a second stream
(Simulation(overlap=True), eagerly and from CUDA graphs), the states of every level --
the deferred coarse levels included -- and the time steps are bit for bit those of the
plain step, on a uniform box and on AMR trees, in both precisions."""
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


def _fields(xyz, seed):
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    w = np.empty((5, xyz.shape[0]))
    for v in range(5):
        w[v] = sum(np.sin(2 * np.pi * xyz[:, d] + ph[v, d]) for d in range(3)) * (0.3 if v in (0, 4) else 0.5)
    w[0] += 1.0
    w[4] += 1.5
    return w


def _tree(H, kind, seed):
    if kind == "uniform":
        return H.Octree(W.uniform_tree(6), 2, (0,) * 6)
    lx = W.random_tree(4, 2, seed, p_refine=0.3, periodic=True)
    return H.Octree(lx, 4, (0,) * 6)


@pytest.mark.parametrize("kind,precision,seed", [("uniform", 1, 1), ("uniform", 0, 2), ("amr", 1, 3), ("amr", 0, 4)])
def test_deferred_restriction_is_bitwise_the_step(H, kind, precision, seed):
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    g = _tree(H, kind, seed)
    assert int(g.t.grid_level) >= 4                    # there are complete levels to restrict
    w0 = _fields(cell_centres_of(g), seed)
    prm = H.Params(5 / 3, cfl=0.6, precision=precision)
    ref = H.Simulation(g, prm, w0=w0)
    # C ABI on one stream: the deferred step, then the restriction
    prm_d = H.Params(5 / 3, cfl=0.6, precision=precision, defer_restriction=True)
    a = H.Simulation(g, prm_d, w0=w0)
    # overlapped with the next step on a second stream, eagerly and from graphs (use_graph
    # takes one eager step)
    b = H.Simulation(g, prm, w0=w0, overlap=True)
    c = H.Simulation(g, prm, w0=w0, overlap=True).use_graph()
    assert b.overlap and c.overlap and c.nsteps == 1
    for _ in range(5):
        ref.step()
        a.step()
        H.hydro_restrict_complete(g, a.u)
        b.step()
    for _ in range(4):
        c.step()
    b.join()
    c.join()
    torch.cuda.synchronize()
    for s_ in (a, b, c):
        assert s_.nsteps == 5
        assert torch.equal(s_.u, ref.u) and torch.equal(s_.dt, ref.dt)
    assert prm.read_status()[0] == 0 and prm_d.read_status()[0] == 0


def test_restrict_complete_arguments(H):
    from paper_2411_14631_gb300 import abi
    g = _tree(H, "uniform", 0)
    assert abi.lib().hydro_restrict_complete(None, None, None) == abi.EINVAL
    import ctypes
    assert abi.lib().hydro_restrict_complete(ctypes.byref(g.t), None, None) == abi.EINVAL


def test_restrict_complete_is_a_no_op_on_box_batches(H):
    import torch
    g = H.Octree.boxes([16, 32], (1,) * 6)
    assert g.n_inst == 2
    u = torch.randn((5, g.ncell), dtype=torch.float64, device="cuda")
    before = u.clone()
    H.hydro_restrict_complete(g, u)
    torch.cuda.synchronize()
    assert torch.equal(u, before)

