"""The surrogate network on the tcgen05 tensor cores (mlp_forward_tc) through the C ABI:
against the mma.sync path (the same BF16 activations up to the order of the FP32
accumulation) and the oracle's FP64 network (the BF16 tolerance of the other forward
test), on ragged batches of one tile, several tiles and more tiles than resident CTAs, with
non-finite values in the unused input slot; and no wait runs out."""
import numpy as np
import pytest

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


def _theta(seed):
    """Seeded parameters with non-zero biases (the initial network has zero biases)."""
    rng = np.random.default_rng(seed)
    th = []
    for sh in [(64, 7), (64,), (64, 64), (64,), (64, 64), (64,), (2, 64), (2,)]:
        std = 1.0 / np.sqrt(sh[1]) if len(sh) == 2 else 0.3
        th.append(rng.normal(0.0, std, int(np.prod(sh))))
    return np.concatenate(th).astype(np.float32)


def _x8(x7):
    x = np.zeros((x7.shape[0], 8), np.float32)
    x[:, :7] = x7
    return x


@pytest.mark.parametrize("n", [5, 128, 1000, 200_000, 1_000_003])
def test_forward_tc_matches_mma_sync_and_oracle(oracle, H, n):
    import torch
    sur = H.Surrogate(theta=_theta(1))
    th = sur.theta.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(n)
    x7 = rng.normal(0, 1, (n, 7))
    x7[:, 6] = rng.uniform(1.1, 1.7, n)
    x8 = _x8(x7)
    xd = torch.as_tensor(x8).cuda()
    y_sync = sur.forward(xd).cpu().numpy()
    x8[::3, 7] = np.nan                        # the unused slot is ignored by both paths
    xd = torch.as_tensor(x8).cuda()
    y_tc = torch.full((n, 2), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.mlp_forward_tc(sur.packed, xd, y_tc, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    y_tc = y_tc.cpu().numpy()
    assert np.all(np.isfinite(y_tc))
    scale = max(np.abs(y_sync).max(), 1e-6)
    assert np.abs(y_tc - y_sync).max() <= 1e-2 * scale, np.abs(y_tc - y_sync).max() / scale
    m = min(n, 2000)
    y_o = oracle.mlp_forward(th, x7[:m])
    so = np.abs(y_o).max()
    assert np.abs(y_tc[:m] - y_o).max() <= 3e-2 * so, np.abs(y_tc[:m] - y_o).max() / so


def test_forward_tc_argument_errors(H):
    import torch
    from paper_2411_14631_gb300 import abi
    assert abi.lib().mlp_forward_tc(None, None, None, 3, None, None) == abi.EINVAL
    sur = H.Surrogate(seed=1)
    xb = torch.zeros(8 * 4 + 4, dtype=torch.float32, device="cuda")
    y = torch.zeros((3, 2), dtype=torch.float32, device="cuda")
    # an input not on a 16-byte boundary is refused before any launch
    assert abi.lib().mlp_forward_tc(sur.packed.data_ptr(), xb.data_ptr() + 4, y.data_ptr(), 3, None,
                                    None) == abi.EINVAL


def test_tanh_rate_probe(H):
    # the MUFU tanh throughput the inference kernel is bounded by: a power-of-two number
    # of results per SM clock between 4 and 64 on any Blackwell part
    r = H.mlp_tanh_rate()
    assert 4.0 <= r <= 64.0, r


def test_forward_tc_empty_and_single_sample(oracle, H):
    import torch
    sur = H.Surrogate(theta=_theta(2))
    # no samples: nothing is launched, the output is not touched
    x0 = torch.zeros((0, 8), dtype=torch.float32, device="cuda")
    y0 = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    H.mlp_forward_tc(sur.packed, x0, y0)
    # one sample: a tile of one row, the other 127 rows never written
    rng = np.random.default_rng(3)
    x7 = rng.normal(0, 1, (1, 7))
    x7[:, 6] = 1.4
    xd = torch.as_tensor(_x8(x7)).cuda()
    y = torch.full((4, 2), 7.0, dtype=torch.float32, device="cuda")     # one row used, three guards
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.mlp_forward_tc(sur.packed, xd, y[:1], status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    yc = y.cpu().numpy()
    assert np.all(yc[1:] == 7.0)
    y_o = oracle.mlp_forward(sur.theta.cpu().numpy().astype(np.float64), x7)
    assert np.abs(yc[:1] - y_o).max() <= 3e-2 * max(np.abs(y_o).max(), 1e-6)
