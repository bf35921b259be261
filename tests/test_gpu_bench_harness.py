"""The benchmark's timing helpers give the states of the runs they time: bench.time_path
makes its steps on a side stream, which must first wait for the initial state made on
the current stream.  After the same number of steps the FP32 and FP64 paths, each on its
own CFL steps (the FP32 candidate is 2^-16 smaller), differ by FP32 round-off and that
small shift in time; a run that started before its initial state was ready, or that
compared states of different step counts, differs by a whole step (about 1e-2 here)."""
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


def test_time_path_runs_on_the_initial_state(H):
    import torch
    import bench
    from paper_2411_14631_gb300 import abi
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    level = 6
    lx = W.uniform_tree(level)
    rho, v = W.turbulent_fields(level)
    tree = H.Octree(lx, level, (abi.BC_PERIODIC,) * 6)
    w0 = W.grid_prims(cell_centres_of(tree), level, rho, v)
    stream = torch.cuda.Stream()
    out = {}
    for prec in (abi.PREC_FP32, abi.PREC_FP64):
        prm = H.Params(5.0 / 3.0, cfl=0.8, precision=prec)
        _, _, sim, _ = bench.time_path(H, tree, prm, w0, 3, 2, stream, "p%d" % prec)
        torch.cuda.synchronize()
        out[prec] = sim
    # the same five steps from the initial state, made on the current stream
    ref = H.Simulation(tree, H.Params(5.0 / 3.0, cfl=0.8, precision=abi.PREC_FP64), w0=w0)
    for _ in range(5):
        ref.step()
    torch.cuda.synchronize()
    assert torch.equal(out[abi.PREC_FP64].u, ref.u)
    u32, u64 = out[abi.PREC_FP32].u, out[abi.PREC_FP64].u
    l1 = (torch.abs(u32[0] - u64[0]).sum() / torch.abs(u64[0]).sum()).item()
    assert l1 < 1e-4, l1
