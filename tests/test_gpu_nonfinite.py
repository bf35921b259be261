"""Non-finite and out-of-range states in both precision paths (through the C ABI).

The FP32 path reads the FP64 state through an integer FP64 -> FP32 conversion and adds
its FP32 increments back through an FP32 -> FP64 one.  Those conversions are checked
here against the IEEE conversions (numpy on the host), special values included; then
NaN, +Inf and 1e300 are written into a few cells of the host-side initial state and
both paths must report AMR_ENONPHYSICAL after one step.
"""
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


FLT_MAX = float(np.finfo(np.float32).max)


def _fp64_inputs():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(200_000) * np.exp(rng.uniform(-110, 110, 200_000))
    half_ulp_max = FLT_MAX + 2.0 ** 103           # exact tie between FLT_MAX and 2^128
    one = np.float64(1.0)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 2.0 ** 128, -2.0 ** 128,
               np.nextafter(2.0 ** 128, 0), -np.nextafter(2.0 ** 128, 0), FLT_MAX, -FLT_MAX,
               half_ulp_max, np.nextafter(half_ulp_max, 0), np.nextafter(half_ulp_max, np.inf),
               2.0 ** -126, -2.0 ** -126, np.nextafter(2.0 ** -126, 0), 1e-40, -1e-40, 5e-324,
               1e300, -1e300, 1e39, -1e39, float(one + 2.0 ** -24), float(one + 3 * 2.0 ** -24),
               float(-(one + 2.0 ** -24)), float(one + 2.0 ** -24 + 2.0 ** -52), 1.0, -1.0]
    # exact ties at random magnitudes: the 29 dropped bits are 1 followed by zeros
    ties = rng.standard_normal(2000) * np.exp(rng.uniform(-80, 80, 2000))
    tb = ties.view(np.uint64)
    tb &= ~np.uint64((1 << 29) - 1)
    tb |= np.uint64(1 << 28)
    return np.concatenate([x, np.array(special), tb.view(np.float64)])


def test_fp64_to_fp32_conversion_against_ieee(H):
    """hydro_state_to_fp32 equals IEEE round-to-nearest-even (numpy's float32 cast) on
    every finite value of the FP32 normal range except exact ties, which round away from
    zero; below 2^-126 it gives a signed zero; |x| >= 2^128, +-Inf and NaN give a
    non-finite float of the same sign."""
    import torch
    x = _fp64_inputs()
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty(x.size, dtype=torch.float32, device="cuda")
    H.hydro_state_to_fp32(xd, yd)
    y = yd.cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        ref = x.astype(np.float32)
    ax = np.abs(x)
    bits = x.view(np.uint64)
    tie = (bits & np.uint64((1 << 29) - 1)) == np.uint64(1 << 28)
    over = np.isnan(x) | (ax >= 2.0 ** 128)
    under = ~over & (ax < 2.0 ** -126)
    normal = ~over & ~under
    # non-finite class, sign kept (a NaN carries no sign to compare)
    assert np.all(~np.isfinite(y[over]))
    s = over & ~np.isnan(y)
    assert np.all(np.signbit(y[s]) == np.signbit(x[s]))
    # flush to a signed zero below the normal range
    assert np.all(y[under] == 0) and np.all(np.signbit(y[under]) == np.signbit(x[under]))
    # IEEE away from ties (Inf where the rounding passes FLT_MAX)
    m = normal & ~tie
    assert np.array_equal(y[m], ref[m])
    # ties: the neighbour of larger magnitude (away from zero)
    t = normal & tie
    assert t.sum() >= 1000
    up = np.abs(y[t].astype(np.float64))
    lo = np.abs(ref[t].astype(np.float64))
    assert np.all(up >= ax[t]) and np.all(np.signbit(y[t]) == np.signbit(x[t]))
    assert np.all((up == lo) | (np.nextafter(lo.astype(np.float32), np.float32(np.inf)) == up.astype(np.float32)))
    # the specials by name
    named = {np.inf: np.inf, -np.inf: -np.inf, FLT_MAX: FLT_MAX, 1.0: 1.0}
    for k, v in named.items():
        i = int(np.nonzero(x == k)[0][0])
        assert y[i] == np.float32(v), (k, y[i])
    assert np.isinf(y[int(np.nonzero(x == FLT_MAX + 2.0 ** 103)[0][0])])


def test_fp32_to_fp64_conversion_against_ieee(H):
    """hydro_state_from_fp32 is exact on normal floats and +-Inf, keeps NaN, and gives a
    signed zero for zero and FP32 denormals."""
    import torch
    rng = np.random.default_rng(12)
    f = (rng.standard_normal(200_000) * np.exp(rng.uniform(-85, 85, 200_000))).astype(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, FLT_MAX, -FLT_MAX, 1e-40, -1e-40, 2.0 ** -126,
                        np.float32(2.0 ** -126) * np.float32(0.5), 1.0], dtype=np.float32)
    f = np.concatenate([f, special])
    fd = torch.tensor(f, device="cuda")
    xd = torch.empty(f.size, dtype=torch.float64, device="cuda")
    H.hydro_state_from_fp32(fd, xd)
    x = xd.cpu().numpy()
    nan = np.isnan(f)
    assert np.all(np.isnan(x[nan]))
    den = ~nan & (f != 0) & (np.abs(f) < 2.0 ** -126)
    assert den.sum() >= 2
    assert np.all(x[den] == 0) and np.all(np.signbit(x[den]) == np.signbit(f[den]))
    rest = ~nan & ~den
    assert np.array_equal(x[rest], f[rest].astype(np.float64))
    assert np.all(np.signbit(x[rest]) == np.signbit(f[rest]))


def test_conversion_argument_errors(H):
    import ctypes as C
    from paper_2411_14631_gb300 import abi
    L = abi.lib()
    assert L.hydro_state_to_fp32(None, None, -1, None) == abi.EINVAL
    assert L.hydro_state_to_fp32(None, None, 5, None) == abi.EINVAL
    assert L.hydro_state_from_fp32(None, None, 0, None) == abi.OK


def _smooth(xyz):
    w = np.empty((5, xyz.shape[0]))
    w[0] = 1.0 + 0.2 * np.sin(2 * np.pi * xyz[:, 0])
    w[1] = 0.3 * np.cos(2 * np.pi * xyz[:, 1])
    w[2] = 0.1
    w[3] = -0.2 * np.sin(2 * np.pi * xyz[:, 2])
    w[4] = 1.0 + 0.1 * np.cos(2 * np.pi * xyz[:, 0])
    return w


@pytest.fixture(scope="module")
def trees(H):
    # a complete level-5 box (z-column kernel) and a random AMR tree (tile kernel above
    # its complete level)
    return {"uniform": H.Octree(W.uniform_tree(5), 5, (0,) * 6),
            "amr": H.Octree(W.random_tree(3, 2, 31, p_refine=0.3, periodic=True), 3, (0,) * 6)}


def _leaf_cells(tree, n, seed):
    son = tree.tables()["son"].cpu().numpy()
    leaf = np.nonzero(son < 0)[0]
    return np.random.default_rng(seed).choice(leaf, n, replace=False)


@pytest.mark.parametrize("kind", ["uniform", "amr"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tiles_only", [False, True])
@pytest.mark.parametrize("bad", ["nan", "inf", "1e300"])
def test_nonfinite_cell_is_reported(H, trees, kind, precision, tiles_only, bad):
    """A NaN, +Inf or 1e300 written into the momentum of a few leaf cells of the host-side
    state is reported as AMR_ENONPHYSICAL after one step by both precision paths and by
    both update kernels; the same run without it reports nothing."""
    import torch
    from paper_2411_14631_gb300 import abi
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    tree = trees[kind]
    prm = H.Params(1.4, cfl=0.5, precision=precision, tiles_only=tiles_only)
    w0 = _smooth(cell_centres_of(tree))
    clean = H.Simulation(tree, prm, w0=w0)
    clean.step()
    assert prm.read_status()[0] == 0
    sim = H.Simulation(tree, prm, w0=w0)
    u = sim.u.cpu().numpy()
    val = {"nan": np.nan, "inf": np.inf, "1e300": 1e300}[bad]
    cells = _leaf_cells(tree, 3, 5)
    u[1, cells] = val
    sim.u.copy_(torch.as_tensor(u))
    sim.step()
    st, _ = prm.read_status()
    assert st == abi.ENONPHYSICAL, (kind, precision, tiles_only, bad, st)
