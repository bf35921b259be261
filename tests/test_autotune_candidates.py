"""The autotuner's candidate launch shapes (host logic, no GPU): which z-column kernels
and segments apply to a mesh, for each precision and Riemann solver."""
from types import SimpleNamespace

from paper_2411_14631_gb300 import abi, autotune


def _tree(grid_level=8, n_inst=0, col_work=0):
    return SimpleNamespace(t=SimpleNamespace(grid_level=grid_level, n_inst=n_inst, col_work=col_work))


def _shapes(c):
    return sorted((d["col_kernel"], d["col_seg"]) for d in c)


def test_fp32_256_box_has_pencil_and_slab_segments():
    c = autotune.column_candidates(_tree(8), abi.PREC_FP32, abi.RIEMANN_HLLC)
    pencil = [s for k, s in _shapes(c) if k == 2]
    slab = [s for k, s in _shapes(c) if k == 1]
    assert pencil == [0, 16, 24, 32, 38, 44, 52, 64, 96, 128]
    assert slab == [0, 16, 32, 64, 128]
    assert len(c) == 15


def test_segments_never_exceed_the_level():
    c = autotune.column_candidates(_tree(5), abi.PREC_FP32, abi.RIEMANN_HLLC)   # 32 cells per axis
    assert _shapes(c) == [(1, 0), (1, 16), (1, 32), (2, 0), (2, 16), (2, 24), (2, 32)]


def test_slab_segments_divide_the_level():
    # the pencil kernel's segments may leave a ragged last segment; the slab kernel's must divide n
    c = autotune.column_candidates(_tree(7), abi.PREC_FP32, abi.RIEMANN_HLLC)
    for k, s in _shapes(c):
        if k == 1 and s:
            assert 128 % s == 0


def test_fp64_has_the_slab_kernel_only():
    c = autotune.column_candidates(_tree(8), abi.PREC_FP64, abi.RIEMANN_HLLC)
    assert {k for k, _ in _shapes(c)} == {1}


def test_exact_solver_keeps_both_kernels_in_fp32():
    c = autotune.column_candidates(_tree(8), abi.PREC_FP32, abi.RIEMANN_EXACT)
    assert {k for k, _ in _shapes(c)} == {1, 2}


def test_surrogate_has_one_default_shape():
    for rs in (abi.RIEMANN_MLP, abi.RIEMANN_MLP_SEEDED):
        assert autotune.column_candidates(_tree(8), abi.PREC_FP32, rs) == [dict(col_kernel=0, col_seg=0)]


def test_box_batches_use_the_fixed_segment():
    c = autotune.column_candidates(_tree(0, n_inst=48, col_work=4096), abi.PREC_FP32, abi.RIEMANN_HLLC)
    assert _shapes(c) == [(1, 0), (2, 0)]
    c = autotune.column_candidates(_tree(0, n_inst=3, col_work=0), abi.PREC_FP32, abi.RIEMANN_HLLC)
    assert c == [dict(col_kernel=0, col_seg=0)]      # no box fits the column kernels: tiles only


def test_coarse_meshes_have_no_column_kernel():
    assert autotune.column_candidates(_tree(2), abi.PREC_FP32, abi.RIEMANN_HLLC) == [dict(col_kernel=0, col_seg=0)]
