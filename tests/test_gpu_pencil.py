"""The column-per-thread z-column kernel (16 x 16-cell footprints, FP32 path) through the
C ABI: for every segment length, ragged ones included, it gives the tile kernel's states
and time steps bit for bit (the tile kernel is the one checked against the oracle), and
the 8 x 8 slab kernel's too -- on complete levels (periodic and outflow, HLLC and exact
solver), on the deepest complete level of AMR trees, on batches of uneven boxes, and on
the 256^3 benchmark box in the benchmark's launch configuration."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

pytestmark = pytest.mark.gpu
OUT, PER = (1,) * 6, (0,) * 6


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
    w[4, ::97] += 3.0                        # pressure spikes: shocks and rarefactions
    return w


def _run(H, tree, w0, steps=3, **kw):
    import torch
    sim = H.Simulation(tree, H.Params(5 / 3, cfl=0.6, precision=1, **kw), w0=w0)
    for _ in range(steps):
        sim.step()
    torch.cuda.synchronize()
    st, _ = sim.prm.read_status()
    return sim.u.cpu().numpy(), sim.dt.cpu().numpy(), st


@pytest.mark.parametrize("level,bc,riemann", [(4, OUT, 0), (5, PER, 0), (5, OUT, 1), (6, PER, 0), (6, OUT, 0)])
def test_pencil_equals_tiles_every_segment(H, level, bc, riemann):
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    g = H.Octree(W.uniform_tree(level), level, bc)
    w0 = _fields(cell_centres_of(g), 50 + level)
    ref_u, ref_dt, st = _run(H, g, w0, riemann=riemann, tiles_only=True)
    assert st == 0
    slab = _run(H, g, w0, riemann=riemann, col_kernel=1)
    assert np.array_equal(slab[0], ref_u) and np.array_equal(slab[1], ref_dt)
    n = 1 << level
    for seg in sorted({0, 2, 6, 10, 16, 22, n}):
        u, dt, st = _run(H, g, w0, riemann=riemann, col_kernel=2, col_seg=seg)
        assert st == 0
        assert np.array_equal(u, ref_u), seg
        assert np.array_equal(dt, ref_dt), seg


@pytest.mark.parametrize("seed,periodic,base", [(70, True, 4), (71, False, 4), (73, True, 5)])
def test_pencil_with_refinement_equals_tiles(H, seed, periodic, base):
    """The deepest complete level of an AMR tree (faces next to refined cells skipped,
    refined cells left to the restriction, fused restriction of the level's fathers)."""
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx = W.random_tree(base, 2, seed, p_refine=0.3, periodic=periodic)
    bc = PER if periodic else OUT
    g = H.Octree(lx, base, bc)
    assert g.t.grid_level == base and g.levelmax >= base + 1
    w0 = _fields(cell_centres_of(g), seed)
    ref_u, ref_dt, _ = _run(H, g, w0, tiles_only=True)
    for seg in (0, 4, 14):
        u, dt, st = _run(H, g, w0, col_kernel=2, col_seg=seg)
        assert st == 0
        assert np.array_equal(u, ref_u), seg
        assert np.array_equal(dt, ref_dt), seg


@pytest.mark.parametrize("bc", [OUT, PER])
def test_pencil_box_batch_equals_tiles(H, bc):
    """Boxes that are multiples of 16 cells, one launch, a time step per box."""
    import torch
    sizes = np.array([32, 16, 48, 16], dtype=np.int32)
    tree = H.Octree.boxes(sizes, bc)
    assert tree.t.col_work > 0
    rng = np.random.default_rng(5)
    w0 = np.empty((5, tree.ncell))
    w0[0] = 1.0 + 0.3 * rng.random(tree.ncell)
    w0[1:4] = 0.4 * rng.standard_normal((3, tree.ncell))
    w0[4] = 1.0 + rng.random(tree.ncell)
    res = {}
    for name, kw in (("tiles", dict(tiles_only=True)), ("slab", dict(col_kernel=1)), ("pencil", dict(col_kernel=2))):
        sim = H.Simulation(tree, H.Params(1.4, cfl=0.6, precision=1, **kw), w0=w0)
        for _ in range(3):
            sim.step()
        torch.cuda.synchronize()
        res[name] = (sim.u.cpu().numpy(), sim.dt.cpu().numpy())
    for name in ("slab", "pencil"):
        assert np.array_equal(res[name][0], res["tiles"][0]), name
        assert np.array_equal(res[name][1], res["tiles"][1]), name


def test_pencil_full_size_benchmark_box(H):
    """The 256^3 turbulent box, one step in the benchmark's launch configuration (the
    library's default segment), against the tile kernel bit for bit."""
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    g = H.Octree(W.uniform_tree(8), 8, PER)
    rho, v = W.turbulent_fields(8)
    w0 = W.grid_prims(cell_centres_of(g), 8, rho, v)
    out = []
    for kw in (dict(tiles_only=True), dict()):
        sim = H.Simulation(g, H.Params(5 / 3, cfl=0.8, precision=1, **kw), w0=w0)
        sim.step()
        torch.cuda.synchronize()
        out.append((sim.u, sim.dt.clone(), sim.prm.read_status()[0]))
        del sim
    assert out[0][2] == 0 and out[1][2] == 0
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])


def test_long_segments_on_a_128_box(H):
    """The autotuner's longest segments on a 128^3 box (level 7): the pencil kernel with 96
    (ragged: 96 + 32) and 128 cells, the slab kernel with 64 and 128, each bitwise the
    default pencil launch, over two steps."""
    import torch
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    g = H.Octree(W.uniform_tree(7), 7, PER)
    w0 = _fields(cell_centres_of(g), 77)
    ref = _run(H, g, w0, steps=2)
    assert ref[2] == 0
    for kw in (dict(col_kernel=2, col_seg=96), dict(col_kernel=2, col_seg=128), dict(col_kernel=1, col_seg=64),
               dict(col_kernel=1, col_seg=128)):
        u, dt, st = _run(H, g, w0, steps=2, **kw)
        assert st == 0, kw
        assert np.array_equal(u, ref[0]) and np.array_equal(dt, ref[1]), kw
