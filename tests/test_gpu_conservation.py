"""hydro_conservation (GPU FP64 leaf totals) through the C ABI: the same bits for every
launch shape, within 1e-14 (relative to the sum of |U| dV) of the oracle's exactly
rounded sums on AMR trees, a 128^3 box and a batch of uneven boxes; and conservation of
mass and energy by the FP64 and FP32 steps measured with it."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-14


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_14631_gb300 import build
    build.build()
    from paper_2411_14631_gb300 import hydro
    return hydro


def _check(gpu, ref):
    gpu = np.asarray(gpu).reshape(ref.shape)
    scale = ref[..., 1, :]
    assert np.all(np.abs(gpu[..., 0, :] - ref[..., 0, :]) <= TOL * scale), (gpu, ref)
    assert np.all(np.abs(gpu[..., 1, :] - ref[..., 1, :]) <= TOL * scale), (gpu, ref)


@pytest.mark.parametrize("seed", [41, 42])
def test_totals_match_oracle_and_launch_shape(oracle, H, seed):
    import torch
    lx = W.random_tree(3, 3, seed, p_refine=0.35, periodic=True)
    t = oracle.Tree(lx, 3, (0,) * 6)
    g = H.Octree(lx, 3, (0,) * 6)
    rng = np.random.default_rng(seed)
    # state in the device tree's cell order (same (level, Hilbert) order as the oracle's)
    u = rng.standard_normal((5, t.ncell)) * np.array([[1.0], [3.0], [3.0], [3.0], [10.0]])
    u[0] = np.abs(u[0]) + 0.1
    ud = torch.tensor(u, device="cuda")
    ref = t.conservation_totals(u)
    outs = [H.hydro_conservation(g, ud, blocks=b).cpu().numpy() for b in (0, 1, 3, 1000)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    _check(outs[0][0], ref)


def test_totals_128_box(oracle, H):
    import torch
    lx = W.uniform_tree(7)
    t = oracle.Tree(lx, 7, (0,) * 6)
    g = H.Octree(lx, 7, (0,) * 6)
    rho, v = W.turbulent_fields(7)
    xyz, _ = t.cell_centres()
    prm = oracle.params(gamma=5 / 3)
    u = t.init_from_prim(W.grid_prims(xyz, 7, rho, v), prm)
    ref = t.conservation_totals(u)
    ud = torch.tensor(u, device="cuda")
    a = H.hydro_conservation(g, ud).cpu().numpy()
    b = H.hydro_conservation(g, ud, blocks=57).cpu().numpy()
    assert np.array_equal(a, b)
    _check(a[0], ref)


def test_box_batch_totals(oracle, H):
    import torch
    sizes = np.array([16, 12, 32, 4, 20], dtype=np.int32)
    g = H.Octree.boxes(sizes)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((5, int(np.sum(sizes.astype(np.int64) ** 3))))
    # batch mode stores each box's octs lexicographically with the cells of an oct together
    ud = torch.tensor(u, device="cuda")
    outs = [H.hydro_conservation(g, ud, blocks=b).cpu().numpy() for b in (0, 2)]
    assert np.array_equal(outs[0], outs[1])
    # the totals do not depend on the order of the cells inside a box
    ref = oracle.box_conservation_totals(sizes, u)
    _check(outs[0], ref)


def test_argument_errors(H):
    import torch
    from paper_2411_14631_gb300 import abi
    import ctypes as C
    g = H.Octree(W.uniform_tree(3), 3, (0,) * 6)
    u = torch.zeros((5, g.ncell), dtype=torch.float64, device="cuda")
    tot = torch.zeros((1, 2, 5), dtype=torch.float64, device="cuda")
    nb = int(abi.lib().hydro_conservation_work_bytes(C.byref(g.t)))
    work = torch.zeros(nb + 512, dtype=torch.uint8, device="cuda")
    L = abi.lib()
    P = lambda x: C.c_void_p(x)
    assert L.hydro_conservation(C.byref(g.t), P(u.data_ptr()), P(tot.data_ptr()), P(work.data_ptr()), nb - 8, 0,
                                None) == abi.ECAPACITY
    assert L.hydro_conservation(C.byref(g.t), P(u.data_ptr()), P(tot.data_ptr()), P(work.data_ptr() + 8), nb, 0,
                                None) == abi.EINVAL
    assert L.hydro_conservation(C.byref(g.t), P(u.data_ptr()), P(tot.data_ptr()), P(work.data_ptr()), nb, -1,
                                None) == abi.EINVAL
    assert L.hydro_conservation(C.byref(g.t), P(u.data_ptr()), P(tot.data_ptr()), P(work.data_ptr()), nb, 0,
                                None) == abi.OK


@pytest.mark.parametrize("precision", [0, 1])
def test_step_conserves_measured_on_gpu(H, precision):
    """Ten steps on a periodic AMR tree keep the leaf totals of mass, momentum and energy
    to rounding, as measured by hydro_conservation: FP64 round-off in the FP64 path; in
    the FP32 path a cell's six face fluxes are summed in FP32 before the FP64 update, so
    the totals keep FP32 round-off of the increments (the bound of the other
    conservation test, 1e-9 after ten steps)."""
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx = W.random_tree(3, 2, 17, p_refine=0.3, periodic=True)
    g = H.Octree(lx, 3, (0,) * 6)
    xyz = cell_centres_of(g)
    w = np.empty((5, xyz.shape[0]))
    w[0] = 1.0 + 0.3 * np.sin(2 * np.pi * xyz[:, 0]) * np.cos(2 * np.pi * xyz[:, 1])
    w[1] = 0.4 * np.sin(2 * np.pi * xyz[:, 2])
    w[2] = -0.3 * np.cos(2 * np.pi * xyz[:, 0])
    w[3] = 0.2
    w[4] = 1.0 + 0.2 * np.sin(2 * np.pi * xyz[:, 1])
    sim = H.Simulation(g, H.Params(5 / 3, cfl=0.6, precision=precision), w0=w)
    t0 = H.hydro_conservation(g, sim.u).cpu().numpy()[0]
    for _ in range(10):
        sim.step()
    t1 = H.hydro_conservation(g, sim.u).cpu().numpy()[0]
    scale = np.maximum(t0[1], t1[1])
    tol = 1e-13 * 10 if precision == 0 else 1e-9
    assert np.all(np.abs(t1[0] - t0[0]) <= tol * scale), (t0, t1)
    assert sim.prm.read_status()[0] == 0
