"""Host-side parameter handling of the Python binding (no GPU: the status word and
counters live in host memory here)."""
import pytest

from paper_2411_14631_gb300 import abi, hydro as H


def test_params_fill_the_c_struct():
    p = H.Params(5 / 3, cfl=0.5, precision=abi.PREC_FP32, tile=1, device="cpu", col_kernel=2, col_seg=38,
                 defer_restriction=True)
    c = p.c
    assert (c.gamma, c.cfl, c.precision, c.tile, c.col_kernel, c.col_seg, c.defer_restriction) == \
        (5 / 3, 0.5, abi.PREC_FP32, 1, 2, 38, 1)
    assert c.d_status == p.status.data_ptr() and c.d_counters == p.counters.data_ptr()
    assert c.reserved == 0


def test_with_fields_copies_and_shares_the_status():
    p = H.Params(1.4, device="cpu")
    q = p.with_fields(defer_restriction=1, col_seg=64)
    assert (q.c.defer_restriction, q.c.col_seg) == (1, 64)
    assert (p.c.defer_restriction, p.c.col_seg) == (0, 0)          # the original is unchanged
    assert q.status is p.status and q.counters is p.counters
    assert q.c.d_status == p.c.d_status
    q.c.cfl = 0.1
    assert p.c.cfl == 0.8


def test_with_fields_rejects_unknown_names():
    p = H.Params(1.4, device="cpu")
    with pytest.raises(TypeError, match="defer_restrction"):
        p.with_fields(defer_restrction=1)
