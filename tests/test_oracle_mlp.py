"""Pins for the oracle's surrogate network: central finite differences against the
analytic backward pass, closed forms of the forward pass, Adam's first step, and the
invariance of the features under the Euler equations' scaling symmetries."""
import numpy as np


def _theta(oracle, seed, scale=0.3):
    return np.random.default_rng(seed).normal(0, scale, oracle.mlp_nparams())


def test_nparams(oracle):
    assert oracle.mlp_nparams() == 7 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 2 + 2


def test_forward_closed_forms(oracle):
    n = oracle.mlp_nparams()
    th = np.zeros(n)
    th[-2:] = [0.7, -1.3]                       # output bias only
    x = np.random.default_rng(0).normal(size=(5, 7))
    assert np.array_equal(oracle.mlp_forward(th, x), np.tile([0.7, -1.3], (5, 1)))
    # one path: x0 -> h1[0] -> h2[0] -> h3[0] -> y0, all weights 1, biases 0
    th = np.zeros(n)
    o = 0
    th[o + 0] = 1.0; o += 7 * 64 + 64
    th[o + 0] = 1.0; o += 64 * 64 + 64
    th[o + 0] = 1.0; o += 64 * 64 + 64
    th[o + 0] = 1.0
    silu = lambda z: z / (1 + np.exp(-z))
    for x0 in (-2.0, 0.3, 1.7):
        y = oracle.mlp_forward(th, np.array([[x0, 0, 0, 0, 0, 0, 0]]))
        assert abs(y[0, 0] - silu(silu(silu(x0)))) <= 1e-15 and y[0, 1] == 0.0


def test_backward_matches_finite_differences(oracle):
    th = _theta(oracle, 1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 7)); dy = rng.normal(size=(4, 2))
    g = oracle.mlp_backward(th, x, dy)
    f = lambda t: np.sum(oracle.mlp_forward(t, x) * dy)
    idx = np.concatenate([rng.choice(th.size, 200, replace=False), np.arange(th.size - 130, th.size)])
    h = 1e-6
    for i in idx:
        tp = th.copy(); tp[i] += h
        tm = th.copy(); tm[i] -= h
        fd = (f(tp) - f(tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step(oracle):
    """After one step from zero moments, m_hat = g and v_hat = g^2: the update is
    lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    th = rng.normal(size=50); g = rng.normal(size=50)
    m = np.zeros(50); v = np.zeros(50)
    th0 = th.copy()
    oracle.adam_step(th, m, v, g, 1e-3, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(th, th0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_features_invariant_under_scaling(oracle):
    """Riemann problems related by a density scale a, a pressure scale b and a Galilean
    shift share their normalised features (and, by similarity, their normalised
    solution)."""
    rng = np.random.default_rng(4)
    g = 1.4
    for _ in range(10):
        WL = np.array([rng.uniform(0.1, 3), rng.normal(), 0, 0, rng.uniform(0.1, 3)])
        WR = np.array([rng.uniform(0.1, 3), rng.normal(), 0, 0, rng.uniform(0.1, 3)])
        a, b, s = rng.uniform(0.2, 5), rng.uniform(0.2, 5), rng.normal()
        k = np.sqrt(b / a)
        WL2 = np.array([a * WL[0], k * WL[1] + s, 0, 0, b * WL[4]])
        WR2 = np.array([a * WR[0], k * WR[1] + s, 0, 0, b * WR[4]])
        x1, r1 = oracle.mlp_features(WL, WR, g)
        x2, r2 = oracle.mlp_features(WL2, WR2, g)
        assert np.allclose(x1, x2, atol=1e-12)
        ps1, us1, _, _ = oracle.exact_star(WL, WR, g)
        ps2, us2, _, _ = oracle.exact_star(WL2, WR2, g)
        assert abs(np.log(ps1 / r1[0]) - np.log(ps2 / r2[0])) <= 1e-10
        assert abs((us1 - r1[1]) / r1[2] - (us2 - r2[1]) / r2[2]) <= 1e-10


def test_features_worked_examples(oracle):
    """The normalisation written out by hand for two problems: rho_ref = rho_L,
    p_ref = max(p_L, p_R), c_ref = sqrt(p_ref / rho_ref), u_bar = (u_L + u_R) / 2."""
    # Sod's states: rho_ref = 1, p_ref = 1, c_ref = 1, u_bar = 0
    x, ref = oracle.mlp_features(np.array([1.0, 0, 0, 0, 1.0]), np.array([0.125, 0, 0, 0, 0.1]), 1.4)
    assert np.allclose(x, [0, 0, 0, np.log(0.125), 0, np.log(0.1), 1.4], rtol=0, atol=1e-15)
    assert np.allclose(ref, [1.0, 0.0, 1.0], rtol=0, atol=1e-15)
    # a collision with the higher pressure on the right: rho_ref = 4, p_ref = 4,
    # c_ref = 1, u_bar = 0.5
    x, ref = oracle.mlp_features(np.array([4.0, 2.5, 0, 0, 1.0]), np.array([1.0, -1.5, 0, 0, 4.0]), 5 / 3)
    assert np.allclose(x, [0, 2.0, np.log(0.25), np.log(0.25), -2.0, 0, 5 / 3], rtol=0, atol=1e-15)
    assert np.allclose(ref, [4.0, 0.5, 1.0], rtol=0, atol=1e-15)
