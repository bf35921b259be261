"""Argument errors of the C ABI come back at once, before the library touches a stream or
device memory: the calls below return AMR_EINVAL (or AMR_OK for an empty no-op) on a
machine without a GPU, where any CUDA call would fail with a CUDA error instead.  Device
pointers here are fake addresses that the rejected calls never use, so the test runs
only where no GPU is visible."""
import ctypes as C

import pytest
import torch

from paper_2411_14631_gb300 import abi

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="fake device pointers: no-GPU check only")



@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2411_14631_gb300 import build
    return build.build()                      # rebuilt if a source is newer than the library


FAKE = C.c_void_p(1 << 20)          # 16-byte aligned, never dereferenced by a rejected call
FAKE2 = C.c_void_p((1 << 20) + 4096)


def _tree(noct=8, levelmin=2, levelmax=4, n_inst=0, grid_level=2):
    t = abi.AmrTree()
    t.noct, t.levelmin, t.levelmax, t.n_inst, t.grid_level = noct, levelmin, levelmax, n_inst, grid_level
    return t


def _params(**kw):
    p = abi.HydroParams(1.4, 0.8, 1e-10, 1e-20, abi.RIEMANN_HLLC, abi.PREC_FP64, 0, 0, None, 0.0,
                        abi.LIMITER_MINMOD, None, None, 0, 0, 0, 0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_step_rejects_before_resetting_dt_next():
    L = abi.lib()
    p = _params()
    # an invalid tree, a bad parameter, a missing flux register: AMR_EINVAL, and the
    # d_dt_next reset (a CUDA call, which fails here) is not reached
    assert L.hydro_step(None, C.byref(p), FAKE, FAKE, FAKE, FAKE, FAKE2, None) == abi.EINVAL
    assert L.hydro_step(C.byref(_tree(noct=0)), C.byref(p), FAKE, FAKE, FAKE, FAKE, FAKE2, None) == abi.EINVAL
    assert L.hydro_step(C.byref(_tree()), C.byref(_params(gamma=1.0)), FAKE, FAKE, FAKE, FAKE, FAKE2,
                        None) == abi.EINVAL
    assert L.hydro_step(C.byref(_tree()), C.byref(p), FAKE, FAKE, None, FAKE, FAKE2, None) == abi.EINVAL
    surrogate64 = _params(riemann=abi.RIEMANN_MLP)            # the surrogate needs FP32 and weights
    assert L.hydro_step(C.byref(_tree()), C.byref(surrogate64), FAKE, FAKE, FAKE, FAKE, FAKE2,
                        None) == abi.EINVAL


@pytest.mark.parametrize("bad", [dict(gamma=1.0), dict(cfl=0.0), dict(rho_floor=0.0), dict(p_floor=-1.0),
                                 dict(riemann=9), dict(precision=3), dict(tile=3), dict(limiter=5),
                                 dict(col_kernel=3), dict(col_seg=7)])
def test_update_rejects_bad_parameters(bad):
    L = abi.lib()
    t = _tree()
    assert L.hydro_godunov_level(C.byref(t), -1, C.byref(_params(**bad)), FAKE, FAKE, FAKE, FAKE, None,
                                 None) == abi.EINVAL
    assert L.hydro_courant(C.byref(t), C.byref(_params(**bad)), FAKE, FAKE, None) == abi.EINVAL


def test_update_and_reflux_reject_levels_and_buffers():
    L = abi.lib()
    t, p = _tree(), _params()
    for level in (0, 1, 5):                                   # outside levelmin .. levelmax
        assert L.hydro_godunov_level(C.byref(t), level, C.byref(p), FAKE, FAKE, FAKE, FAKE, None,
                                     None) == abi.EINVAL
    assert L.hydro_godunov_level(C.byref(t), -1, C.byref(p), None, FAKE, FAKE, FAKE, None, None) == abi.EINVAL
    for level in (0, 4):                                      # outside 1 .. levelmax-1
        assert L.hydro_reflux_level(C.byref(t), level, C.byref(p), FAKE, FAKE, FAKE, None, None) == abi.EINVAL
    assert L.hydro_reflux_level(C.byref(t), 2, C.byref(p), None, FAKE, FAKE, None, None) == abi.EINVAL
    assert L.hydro_courant(None, C.byref(p), FAKE, FAKE, None) == abi.EINVAL


def test_restrict_complete_no_ops_and_errors():
    L = abi.lib()
    assert L.hydro_restrict_complete(None, FAKE, None) == abi.EINVAL
    assert L.hydro_restrict_complete(C.byref(_tree()), None, None) == abi.EINVAL
    assert L.hydro_restrict_complete(C.byref(_tree(n_inst=3)), FAKE, None) == abi.OK        # batch: nothing
    assert L.hydro_restrict_complete(C.byref(_tree(grid_level=2)), FAKE, None) == abi.OK    # no level below g-1


def test_subcycled_and_harvest_reject():
    L = abi.lib()
    t, p = _tree(), _params()
    assert L.hydro_step_subcycled(C.byref(t), C.byref(p), FAKE, FAKE, FAKE, FAKE, FAKE2, None) == abi.EINVAL
    assert L.hydro_harvest_faces(C.byref(t), C.byref(p), FAKE, FAKE, FAKE, 10, 0, FAKE2, None) == abi.EINVAL
    assert L.hydro_harvest_faces(C.byref(_tree(n_inst=2)), C.byref(p), FAKE, FAKE, FAKE, 10, 1, FAKE2,
                                 None) == abi.EINVAL


def test_conversions_and_status():
    L = abi.lib()
    assert L.hydro_state_to_fp32(FAKE, FAKE2, -1, None) == abi.EINVAL
    assert L.hydro_state_to_fp32(None, None, 0, None) == abi.OK
    assert L.hydro_state_from_fp32(None, FAKE, 5, None) == abi.EINVAL
    assert L.amr_get_status(None, None, None) == abi.EINVAL


def test_tensor_core_surrogate_rejects():
    L = abi.lib()
    assert L.mlp_forward_tc(None, FAKE, FAKE2, 10, None, None) == abi.EINVAL
    assert L.mlp_forward_tc(FAKE, FAKE, FAKE2, -1, None, None) == abi.EINVAL
    assert L.mlp_forward_tc(FAKE, None, None, 0, None, None) == abi.OK                     # no samples
    assert L.mlp_forward_tc(FAKE, None, FAKE2, 10, None, None) == abi.EINVAL
    assert L.mlp_forward_tc(FAKE, C.c_void_p((1 << 20) + 4), FAKE2, 10, None, None) == abi.EINVAL   # x: 16 B
    assert L.mlp_forward_tc(FAKE, FAKE, C.c_void_p((1 << 20) + 4), 10, None, None) == abi.EINVAL   # y: 8 B
    n = C.c_int64()
    assert L.mlp_tanh_rate(None, C.byref(n), None) == abi.EINVAL
