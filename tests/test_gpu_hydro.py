"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer tables: bit-exact.  FP64 fields: per field max|gpu - oracle| / max|oracle|
<= 1e-12 (the tolerance stated for the FP64 GPU path; the kernels may contract
multiply-adds, the oracle does not).  FP32 path: L1 distance from the FP64 oracle
bounded (reconstruction and Riemann solve in FP32, state accumulation in FP64)."""
import numpy as np
import pytest

from paper_2411_14631_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
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


def _smooth_random(xyz, seed, amp=0.3):
    rng = np.random.default_rng(seed)
    Wp = np.empty((5, xyz.shape[0]))
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    for v in range(5):
        s = sum(np.sin(2 * np.pi * xyz[:, d] + ph[v, d]) for d in range(3))
        Wp[v] = s * (amp if v in (0, 4) else 0.5)
    Wp[0] = 1.0 + Wp[0]
    Wp[4] = 1.5 + Wp[4]
    return Wp


def _pair(oracle, H, lx, levelmin, bc, prims, gamma, cfl=0.8, riemann=0, precision=0, tile=0, limiter=0):
    import torch
    t = oracle.Tree(lx, levelmin, bc)
    assert t.ok
    g = H.Octree(lx, levelmin, bc)
    xyz, _ = t.cell_centres()
    w0 = prims(xyz)
    prm_o = oracle.params(gamma=gamma, cfl=cfl, riemann=riemann, limiter=limiter)
    prm_g = H.Params(gamma, cfl=cfl, riemann=riemann, precision=precision, tile=tile, limiter=limiter)
    u_o = t.init_from_prim(w0, prm_o)
    sim = H.Simulation(g, prm_g, w0=w0)
    torch.cuda.synchronize()
    return t, g, prm_o, prm_g, u_o, sim


def _relerr(a, b):
    return np.array([np.max(np.abs(a[v] - b[v])) / max(np.max(np.abs(b[v])), 1e-300) for v in range(5)])


@pytest.mark.parametrize("seed", range(6))
def test_octree_tables_bit_exact(oracle, H, seed):
    rng = np.random.default_rng(200 + seed)
    base = int(rng.integers(2, 4)); extra = int(rng.integers(1, 4))
    periodic = bool(seed % 2)
    lx = W.random_tree(base, extra, seed, p_refine=0.25, periodic=periodic)
    rng.shuffle(lx)                       # input order must not matter
    bc = PER if periodic else OUT
    t = oracle.Tree(lx, base, bc)
    g = H.Octree(lx, base, bc)
    tab = {k: v.cpu().numpy() for k, v in g.tables().items()}
    for k in ("lvl", "ix", "iy", "iz", "son", "father", "nbor", "nb27"):
        assert np.array_equal(tab[k], getattr(t, k)), k
    assert np.array_equal(tab["key"].view(np.uint64), t.key)
    assert np.array_equal(g.lvl_off[:22], t.lvl_off[:22])
    refm = (t.son.reshape(-1, 8) >= 0) @ (1 << np.arange(8))
    assert np.array_equal(tab["refmask"], refm.astype(np.uint8))


def test_octree_errors(oracle, H):
    from paper_2411_14631_gb300 import abi
    levels = {l: W.full_level(l) for l in range(1, 4)}
    levels[4] = W._pack(np.array([0]), np.array([0]), np.array([0]))
    levels[5] = W._pack(np.array([1]), np.array([1]), np.array([1]))
    with pytest.raises(abi.AmrError) as e:
        H.Octree(W.to_lxyz(levels), 3)
    assert e.value.status == abi.EUNBALANCED
    lx = W.uniform_tree(3)
    with pytest.raises(abi.AmrError) as e:
        H.Octree(np.concatenate([lx, lx[-1:]]), 3)
    assert e.value.status == abi.EINVAL
    with pytest.raises(abi.AmrError) as e:
        H.Octree(lx[:-1], 3)
    assert e.value.status == abi.EINVAL


def _run_both(t, prm_o, u_o, sim, nsteps):
    import torch
    dts = []
    for _ in range(nsteps):
        dt_g = float(sim.dt.item())
        u_o, dt_o, st = t.step(u_o, prm_o)
        assert st == 0
        dts.append((dt_o, dt_g))
        sim.step()
    torch.cuda.synchronize()
    return u_o, sim.u.cpu().numpy(), dts


def test_sod_32cubed_fp64_parity(oracle, H):
    """Sod shock tube, 32^3 at level 5 (4096 octs), outflow, HLLC, CFL 0.8, 20 steps."""
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, W.uniform_tree(5), 5, OUT, lambda x: W.sod_prims(x), 1.4)
    u_o, u_g, dts = _run_both(t, prm_o, u_o, sim, 20)
    for dt_o, dt_g in dts:
        assert abs(dt_o - dt_g) <= 1e-14 * dt_o
    assert np.all(_relerr(u_g, u_o) <= FP64_TOL), _relerr(u_g, u_o)
    assert prm_g.read_status()[0] == 0


@pytest.mark.parametrize("seed,periodic", [(0, True), (1, False), (2, True), (3, False)])
def test_amr_fp64_parity(oracle, H, seed, periodic):
    """Random balanced AMR trees (up to 3 levels of refinement): ghost interpolation,
    flux register, refluxing and restriction against the oracle."""
    lx = W.random_tree(3, 3, 50 + seed, p_refine=0.3, periodic=periodic)
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, PER if periodic else OUT,
                                        lambda x: _smooth_random(x, seed), 5 / 3, cfl=0.6)
    assert t.levelmax >= 5
    u_o, u_g, dts = _run_both(t, prm_o, u_o, sim, 4)
    for dt_o, dt_g in dts:
        assert abs(dt_o - dt_g) <= 1e-14 * dt_o
    err = _relerr(u_g, u_o)
    assert np.all(err <= FP64_TOL), err


@pytest.mark.parametrize("seed,periodic", [(0, True), (1, False)])
def test_mc_limiter_fp64_parity(oracle, H, seed, periodic):
    """The monotonized central limiter (tile kernel on every level), FP64 against the oracle
    on random AMR trees; a uniform 16^3 box exercises the level the z-column kernel would
    take with MinMod."""
    lx = W.random_tree(3, 3, 60 + seed, p_refine=0.3, periodic=periodic)
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, PER if periodic else OUT,
                                        lambda x: _smooth_random(x, seed), 5 / 3, cfl=0.6, limiter=1)
    u_o, u_g, dts = _run_both(t, prm_o, u_o, sim, 4)
    for dt_o, dt_g in dts:
        assert abs(dt_o - dt_g) <= 1e-14 * dt_o
    assert np.all(_relerr(u_g, u_o) <= FP64_TOL), _relerr(u_g, u_o)
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, W.uniform_tree(4), 4, OUT, lambda x: W.sod_prims(x), 1.4,
                                        limiter=1)
    u_o, u_g, _ = _run_both(t, prm_o, u_o, sim, 10)
    assert np.all(_relerr(u_g, u_o) <= FP64_TOL), _relerr(u_g, u_o)


def test_exact_riemann_fp64_parity(oracle, H):
    lx = W.random_tree(3, 2, 7, p_refine=0.3, periodic=False)
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, OUT, lambda x: W.sod_prims(x, 1), 1.4, riemann=1)
    u_o, u_g, _ = _run_both(t, prm_o, u_o, sim, 5)
    err = _relerr(u_g, u_o)
    assert np.all(err <= FP64_TOL), err


def test_single_level_calls_match_step(oracle, H):
    """hydro_godunov_level per level + reflux_level per level == hydro_step (the two
    reflux names are one entry point: each is used on every other level)."""
    import torch
    lx = W.random_tree(3, 2, 9, p_refine=0.3, periodic=True)
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, PER, lambda x: _smooth_random(x, 5), 5 / 3)
    u_new = torch.empty_like(sim.u)
    reg = torch.zeros_like(sim.reg)
    for l in range(g.levelmin, g.levelmax + 1):
        H.hydro_godunov_level(g, l, prm_g, sim.u, u_new, reg, sim.dt)
    for l in range(g.levelmax - 1, 0, -1):
        (H.reflux_level if l % 2 else H.hydro_reflux_level)(g, l, prm_g, reg, u_new, sim.dt)
    sim.step()
    assert torch.equal(u_new, sim.u)


def _l1(t, a, b):
    leaf = t.son < 0
    vol = np.ldexp(1.0, -3 * np.repeat(t.lvl, 8).astype(np.int64))[leaf]
    return np.array([np.sum(np.abs(a[v, leaf] - b[v, leaf]) * vol) / np.sum(np.abs(b[v, leaf]) * vol + 1e-300)
                     for v in range(5)])


@pytest.mark.parametrize("tile", [1, 2])
def test_fp32_path_close_to_oracle(oracle, H, tile):
    """FP32 reconstruction + Riemann with FP64 accumulation stays within FP32 round-off
    growth of the FP64 oracle on a smooth AMR flow."""
    lx = W.random_tree(3, 2, 21, p_refine=0.3, periodic=True)
    t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, PER, lambda x: _smooth_random(x, 8), 5 / 3,
                                        cfl=0.6, precision=1, tile=tile)
    import torch
    u_o2 = u_o.copy()
    for _ in range(5):
        sim.step()
    torch.cuda.synchronize()
    for _ in range(5):
        u_o2, _, _ = t.step(u_o2, prm_o)
    l1 = _l1(t, sim.u.cpu().numpy(), u_o2)
    assert np.all(l1[[0, 4]] < 1e-5), l1


def test_fp32_tile_depth_invariance(oracle, H):
    """The tile a cell is updated in does not change its arithmetic: depth-1 and depth-2
    tiles give bitwise identical states."""
    import torch
    lx = W.random_tree(3, 2, 31, p_refine=0.4, periodic=False)
    res = []
    for tile in (1, 2):
        t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, OUT, lambda x: _smooth_random(x, 2), 5 / 3,
                                            precision=1, tile=tile)
        for _ in range(3):
            sim.step()
        torch.cuda.synchronize()
        res.append(sim.u.cpu().numpy())
    assert np.array_equal(res[0], res[1])


def test_conservation_fp64_and_fp32(oracle, H):
    import torch
    lx = W.random_tree(3, 2, 41, p_refine=0.3, periodic=True)
    for precision in (0, 1):
        t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, lx, 3, PER, lambda x: _smooth_random(x, 3), 5 / 3,
                                            cfl=0.5, precision=precision)
        leaf = t.son < 0
        vol = np.ldexp(1.0, -3 * np.repeat(t.lvl, 8).astype(np.int64))[leaf]
        tot = lambda u: np.array([np.sum(u[v, leaf] * vol) for v in range(5)])
        scale = tot(np.abs(u_o))
        t0 = tot(sim.u.cpu().numpy())
        for _ in range(5):
            sim.step()
        torch.cuda.synchronize()
        drift = np.abs(tot(sim.u.cpu().numpy()) - t0) / scale
        limit = 5e-13 if precision == 0 else 1e-9
        assert np.all(drift < limit), (precision, drift)


def test_uniform_flow_preserved(oracle, H):
    import torch
    for precision in (0, 1):
        t, g, prm_o, prm_g, u_o, sim = _pair(oracle, H, W.uniform_tree(4), 4, PER,
                                            lambda x: W.uniform_prims(x, 1.3, (0.4, -0.7, 0.2), 0.9), 5 / 3,
                                            precision=precision)
        u0 = sim.u.clone()
        for _ in range(3):
            sim.step()
        torch.cuda.synchronize()
        assert torch.equal(sim.u, u0)


def test_cuda_graph_replay_matches_eager(oracle, H):
    import torch
    lx = W.random_tree(3, 2, 61, p_refine=0.3, periodic=True)
    g = H.Octree(lx, 3, PER)
    t = oracle.Tree(lx, 3, PER)
    xyz, _ = t.cell_centres()
    w0 = _smooth_random(xyz, 12)
    for precision in (0, 1):
        a = H.Simulation(g, H.Params(5 / 3, precision=precision), w0=w0)
        b = H.Simulation(g, H.Params(5 / 3, precision=precision), w0=w0).use_graph()
        for _ in range(5):
            a.step()
        for _ in range(4):
            b.step()
        torch.cuda.synchronize()
        assert torch.equal(a.u, b.u) and torch.equal(a.dt, b.dt)


def test_autotuner_picks_a_candidate(oracle, H, tmp_path, monkeypatch):
    from paper_2411_14631_gb300 import autotune
    monkeypatch.setenv("AMRHYDRO_TUNE_CACHE", str(tmp_path / "tune.json"))
    lx = W.uniform_tree(5)
    g = H.Octree(lx, 5, OUT)
    t = oracle.Tree(lx, 5, OUT)
    xyz, _ = t.cell_centres()
    best, ms = autotune.tune(g, 1.4, W.sod_prims(xyz), steps=2)
    names = set(ms)
    # a complete 32^3 level: pencil and slab z-column candidates, no tile levels
    assert any(n.startswith("pencil/") for n in names) and any(n.startswith("slab/") for n in names)
    assert best["col_kernel"] in (1, 2) and best["tile"] == 0
    assert min(ms.values()) == ms[autotune._name(best)]
    best2, ms2 = autotune.tune(g, 1.4, W.sod_prims(xyz), steps=2)   # cached
    assert best2 == best and ms2 == ms


@pytest.mark.parametrize("level,precision,riemann,bc", [(5, 0, 0, OUT), (5, 1, 0, PER), (6, 1, 0, OUT),
                                                        (6, 0, 1, PER), (5, 1, 1, OUT)])
def test_column_kernel_equals_tiles(oracle, H, level, precision, riemann, bc):
    """A complete finest level is updated by the z-column kernel; the tile kernel
    (tiles_only) gives the same states and time steps bit for bit."""
    import torch
    lx = W.uniform_tree(level)
    g = H.Octree(lx, level, bc)
    assert g.t.grid_level == level
    t = oracle.Tree(lx, level, bc)
    xyz, _ = t.cell_centres()
    w0 = _smooth_random(xyz, 40 + level)
    w0[4, :: 97] += 3.0                    # a few pressure spikes: shocks and rarefactions
    res = []
    for tiles_only in (False, True):
        sim = H.Simulation(g, H.Params(5 / 3, cfl=0.6, precision=precision, riemann=riemann,
                                       tiles_only=tiles_only), w0=w0)
        for _ in range(3):
            sim.step()
        torch.cuda.synchronize()
        res.append((sim.u.cpu().numpy(), sim.dt.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("seed,periodic,precision", [(70, True, 0), (71, False, 1), (72, True, 1)])
def test_column_kernel_with_refinement_equals_tiles(oracle, H, seed, periodic, precision):
    """The deepest complete level of an AMR tree runs on the z-column kernel (faces next to
    refined cells skipped, refined cells left to the restriction); it matches the tile
    kernel bit for bit, states and time steps."""
    import torch
    lx = W.random_tree(4, 2, seed, p_refine=0.3, periodic=periodic)
    bc = PER if periodic else OUT
    g = H.Octree(lx, 4, bc)
    assert g.t.grid_level == 4 and g.levelmax >= 5
    t = oracle.Tree(lx, 4, bc)
    xyz, _ = t.cell_centres()
    w0 = _smooth_random(xyz, seed)
    res = []
    for tiles_only in (False, True):
        sim = H.Simulation(g, H.Params(5 / 3, cfl=0.6, precision=precision, tiles_only=tiles_only), w0=w0)
        for _ in range(3):
            sim.step()
        torch.cuda.synchronize()
        res.append((sim.u.cpu().numpy(), sim.dt.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
