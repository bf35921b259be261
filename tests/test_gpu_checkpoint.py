"""Checkpoint / resume through the host (save_checkpoint, load_checkpoint): a run saved
after some steps and resumed from the file continues bit for bit like the run that was
not interrupted, on an AMR tree (both precisions) and on a batch of boxes; a file whose
state does not fit the rebuilt tree, or of another version, is refused."""
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


def _interrupted_equals_straight(H, tree, prm, w0, before, after, path):
    import torch
    straight = H.Simulation(tree, prm, w0=w0)
    for _ in range(before + after):
        straight.step()
    first = H.Simulation(tree, prm, w0=w0)
    for _ in range(before):
        first.step()
    H.save_checkpoint(path, first)
    resumed = H.load_checkpoint(path, prm)
    assert resumed.nsteps == before and resumed.tree.ncell == tree.ncell
    for _ in range(after):
        resumed.step()
    torch.cuda.synchronize()
    assert torch.equal(resumed.u, straight.u)
    assert torch.equal(resumed.dt, straight.dt)
    assert prm.read_status()[0] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_amr_bit_for_bit(H, tmp_path, precision):
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    lx = W.random_tree(3, 2, 77, p_refine=0.3, periodic=False)
    tree = H.Octree(lx, 3, (1,) * 6)
    w0 = W.sod_prims(cell_centres_of(tree))
    prm = H.Params(1.4, cfl=0.8, precision=precision)
    _interrupted_equals_straight(H, tree, prm, w0, 3, 4, tmp_path / "amr.npz")


def test_resume_batch_bit_for_bit(H, tmp_path):
    sizes = np.array([16, 32, 20], dtype=np.int32)
    tree = H.Octree.boxes(sizes, (1,) * 6)
    w0 = W.batch_prims(sizes, lambda N: W.sedov_box_prims_lex(int(N)))
    prm = H.Params(1.4, cfl=0.8, precision=1)
    _interrupted_equals_straight(H, tree, prm, w0, 2, 3, tmp_path / "boxes.npz")


def test_refuses_mismatched_files(H, tmp_path):
    lx = W.random_tree(2, 1, 5, p_refine=0.3)
    tree = H.Octree(lx, 2)
    prm = H.Params(5 / 3)
    sim = H.Simulation(tree, prm, w0=W.uniform_prims(W.cell_centres(lx)))
    path = tmp_path / "run.npz"
    H.save_checkpoint(path, sim)
    with np.load(path) as z:
        rec = dict(z)
    bad = dict(rec, u=rec["u"][:, :-8])
    np.savez(tmp_path / "short.npz", **bad)
    with pytest.raises(ValueError):
        H.load_checkpoint(tmp_path / "short.npz", prm)
    np.savez(tmp_path / "version.npz", **dict(rec, version=np.int32(99)))
    with pytest.raises(ValueError):
        H.load_checkpoint(tmp_path / "version.npz", prm)
