"""hydro_step's reflux + restriction pass through the C ABI: the levels below the deepest
complete one are restricted three per launch (one CTA per subtree); the step is bit for
bit the per-level reflux_level calls on AMR trees (periodic and outflow, both precisions,
deepest complete level 2 to 6), eagerly and replayed from a CUDA graph."""
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


@pytest.mark.parametrize("seed,periodic,precision,base", [(81, True, 0, 3), (82, False, 1, 4), (83, True, 1, 5),
                                                         (84, False, 0, 6), (85, True, 1, 2)])
def test_step_reflux_equals_per_level(H, seed, periodic, precision, base):
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx = W.random_tree(base, 2 if base < 6 else 1, seed, p_refine=0.3, periodic=periodic)
    g = H.Octree(lx, max(base, 2), (0,) * 6 if periodic else (1,) * 6)
    assert g.levelmax > base
    w0 = _fields(cell_centres_of(g), seed)
    prm = H.Params(5 / 3, cfl=0.6, precision=precision)
    a = H.Simulation(g, prm, w0=w0)
    b = H.Simulation(g, prm, w0=w0)
    for _ in range(3):
        a.step()                                   # hydro_step
        b.dt_next.fill_(1e300)
        H.hydro_godunov_level(g, -1, prm, b.u, b.u_new, b.reg, b.dt, b.dt_next)
        for l in range(g.levelmax - 1, 0, -1):
            H.reflux_level(g, l, prm, b.reg, b.u_new, b.dt, b.dt_next)
        b.u, b.u_new = b.u_new, b.u
        b.dt, b.dt_next = b.dt_next, b.dt
    torch.cuda.synchronize()
    assert torch.equal(a.u, b.u) and torch.equal(a.dt, b.dt)
    assert prm.read_status()[0] == 0
    c = H.Simulation(g, prm, w0=w0).use_graph()
    for _ in range(2):
        c.step()
    torch.cuda.synchronize()
    assert torch.equal(c.u, a.u) and torch.equal(c.dt, a.dt)
