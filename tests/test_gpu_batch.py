"""Batch mode on the GPU: many independent uniform boxes of uneven size updated in one
launch, each with its own CFL time step, against the oracle's uniform-box step.
FP64: per-box dt within 1e-14, states within 1e-12 (per field, max norm, relative)."""
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


def _box_fields(N, seed):
    """Smooth flow plus a pressure spike, lexicographic (primitive variables)."""
    i = np.arange(N ** 3)
    x = np.stack([i % N, (i // N) % N, i // (N * N)], axis=1) / N
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, (5, 3))
    Wp = np.empty((5, N ** 3))
    for v in range(5):
        Wp[v] = 0.3 * sum(np.sin(2 * np.pi * x[:, d] + ph[v, d]) for d in range(3))
    Wp[0] += 1.0
    Wp[4] += 1.5
    Wp[4, (N // 2) * (1 + N + N * N)] += 20.0
    return Wp


def _cons_lex(oracle, Wl, gamma):
    U = np.empty_like(Wl)
    for c in range(Wl.shape[1]):
        U[:, c] = oracle.prim_to_cons(Wl[:, c], gamma)
    return U


@pytest.mark.parametrize("bc", [(1,) * 6, (0,) * 6])
def test_batch_fp64_matches_oracle_per_box(oracle, H, bc):
    import torch
    sizes = np.array([16, 24, 12, 20], dtype=np.int32)
    gamma = 1.4
    tree = H.Octree.boxes(sizes, bc)
    assert tree.n_inst == 4 and tree.ncell == int((sizes.astype(np.int64) ** 3).sum())
    fields = {int(N): _box_fields(int(N), 10 + k) for k, N in enumerate(sizes)}
    w0 = W.batch_prims(sizes, lambda N: fields[N])
    prm = H.Params(gamma, cfl=0.6)
    sim = H.Simulation(tree, prm, w0=w0)
    prm_o = oracle.params(gamma=gamma, cfl=0.6)
    u_o = {int(N): _cons_lex(oracle, fields[int(N)], gamma) for N in sizes}
    for step in range(3):
        dts = sim.dt.cpu().numpy()
        for b, N in enumerate(sizes):
            N = int(N)
            dt_o = oracle.box_courant(N, u_o[N], prm_o)
            assert abs(dts[b] - dt_o) <= 1e-14 * dt_o, (step, b)
            u_o[N], st = oracle.box_step(N, bc, u_o[N], prm_o, dt_o)
            assert st == 0
        sim.step()
    torch.cuda.synchronize()
    ug = sim.u.cpu().numpy()
    for b, N in enumerate(sizes):
        N = int(N)
        seg = ug[:, tree.cell_off[b]:tree.cell_off[b + 1]]
        ref = np.empty_like(seg)
        ref[:, :] = u_o[N][:, W.box_batch_to_lex(N)]
        for v in range(5):
            err = np.max(np.abs(seg[v] - ref[v])) / np.max(np.abs(ref[v]))
            assert err <= 1e-12, (b, v, err)


def test_batch_tile_depth_invariance_and_fp32(oracle, H):
    import torch
    sizes = np.array([16, 24, 32, 8], dtype=np.int32)      # all multiples of 8: depth 2 available
    tree = H.Octree.boxes(sizes, (1,) * 6)
    fields = {int(N): _box_fields(int(N), 30 + k) for k, N in enumerate(sizes)}
    w0 = W.batch_prims(sizes, lambda N: fields[N])
    res = []
    for tile in (1, 2):
        sim = H.Simulation(tree, H.Params(5 / 3, cfl=0.6, precision=1, tile=tile), w0=w0)
        for _ in range(4):
            sim.step()
        torch.cuda.synchronize()
        res.append(sim.u.cpu().numpy())
    assert np.array_equal(res[0], res[1])
    sim64 = H.Simulation(tree, H.Params(5 / 3, cfl=0.6), w0=w0)
    for _ in range(4):
        sim64.step()
    u64 = sim64.u.cpu().numpy()
    l1 = np.abs(res[0][0] - u64[0]).sum() / np.abs(u64[0]).sum()
    assert l1 < 1e-5, l1


def test_batch_rejects_bad_sizes(H):
    from paper_2411_14631_gb300 import abi
    with pytest.raises(abi.AmrError):
        H.Octree.boxes(np.array([16, 18], dtype=np.int32))


@pytest.mark.parametrize("bc", [(1,) * 6, (0,) * 6])
def test_batch_column_kernel(oracle, H, bc):
    """Boxes that are all multiples of 16 cells run on the z-column kernel: FP64 against
    the box oracle, and bitwise equal to the tile kernel (tiles_only) in FP64 and FP32."""
    import torch
    sizes = np.array([16, 32, 48, 16], dtype=np.int32)
    tree = H.Octree.boxes(sizes, bc)
    assert tree.t.col_work > 0
    fields = {int(N): _box_fields(int(N), 50 + k) for k, N in enumerate(sizes)}
    w0 = W.batch_prims(sizes, lambda N: fields[N])
    res = {}
    for precision in (0, 1):
        for tiles_only in (False, True):
            sim = H.Simulation(tree, H.Params(1.4, cfl=0.6, precision=precision, tiles_only=tiles_only), w0=w0)
            for _ in range(3):
                sim.step()
            torch.cuda.synchronize()
            res[(precision, tiles_only)] = (sim.u.cpu().numpy(), sim.dt.cpu().numpy())
    for precision in (0, 1):
        assert np.array_equal(res[(precision, False)][0], res[(precision, True)][0])
        assert np.array_equal(res[(precision, False)][1], res[(precision, True)][1])
    prm_o = oracle.params(gamma=1.4, cfl=0.6)
    ug = res[(0, False)][0]
    for b, N in enumerate(sizes):
        N = int(N)
        U = _cons_lex(oracle, fields[N], 1.4)
        for _ in range(3):
            U, st = oracle.box_step(N, bc, U, prm_o, oracle.box_courant(N, U, prm_o))
        seg = ug[:, tree.cell_off[b]:tree.cell_off[b + 1]]
        ref = U[:, W.box_batch_to_lex(N)]
        for v in range(5):
            assert np.max(np.abs(seg[v] - ref[v])) <= 1e-12 * np.max(np.abs(ref[v])), (b, v)
