"""hydro_step_static_scratch: the step for callers that cannot allocate device memory
when they step (real-time loops that forbid allocation after start-up, hosts whose
device memory belongs to another framework's pool).

It keeps the flux register in a fixed array inside the library instead of a caller
buffer.  Checked here through the C ABI against hydro_step with a caller-allocated
register, on two calls in a row, within the FP64 parity tolerance of the other tests
(the two run the same kernels on the same inputs, so the states are also bitwise
equal); on a tree whose register has a ghost-children part; and the size limit is
enforced.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-12


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
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    Wp = np.empty((5, xyz.shape[0]))
    for v in range(5):
        Wp[v] = 0.3 * sum(np.sin(2 * np.pi * xyz[:, d] + ph[v, d]) for d in range(3))
    Wp[0] += 1.0
    Wp[4] += 1.5
    return Wp


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_step_matches_hydro_step(H, precision):
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    # a tree with ghost fathers, so that the ghost-children part at the end of the array
    # (the second term of the capacity check) is written and read
    for seed in range(77, 97):
        lx = W.random_tree(3, 3, seed, p_refine=0.3, periodic=False)
        tree = H.Octree(lx, 3, (1,) * 6)
        if tree.t.n_ghost > 0:
            break
    assert tree.t.n_ghost > 0
    assert tree.levelmax >= 5 and 0 < tree.noct - tree.t.reg_base <= 131072
    prm = H.Params(5 / 3, cfl=0.6, precision=precision)
    w0 = _smooth(cell_centres_of(tree), 1)
    ref = H.Simulation(tree, prm, w0=w0)
    u_a, u_b = ref.u.clone(), torch.empty_like(ref.u)
    dt_a, dt_b = ref.dt.clone(), torch.empty_like(ref.dt)
    for call in range(2):
        ref.step()
        H.hydro_step_static_scratch(tree, prm, u_a, u_b, dt_a, dt_b)
        torch.cuda.synchronize()
        for v in range(5):
            scale = torch.max(torch.abs(ref.u[v])).item()
            assert torch.max(torch.abs(u_b[v] - ref.u[v])).item() <= FP64_TOL * scale, (call, v)
        assert torch.equal(u_b, ref.u), call
        assert abs(dt_b.item() - ref.dt.item()) <= 1e-14 * ref.dt.item()
        u_a, u_b = u_b, u_a
        dt_a, dt_b = dt_b, dt_a
    assert prm.read_status()[0] == 0


def test_static_scratch_rejects_large_trees(H):
    import torch
    from paper_2411_14631_gb300 import abi
    lx = W.uniform_tree(8)                          # 2.4 M octs, all above level 2
    tree = H.Octree(lx, 2, (0,) * 6)
    assert tree.noct - tree.t.reg_base > 131072
    prm = H.Params(1.4)
    u = torch.ones((5, tree.ncell), dtype=torch.float64, device="cuda")
    u_new = torch.empty_like(u)
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.AmrError) as e:
        H.hydro_step_static_scratch(tree, prm, u, u_new, dt)
    assert e.value.status == abi.ECAPACITY
