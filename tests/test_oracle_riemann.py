"""Pins for the oracle's single-state pieces: MinMod, conversions, HLLC, exact solver.

Pins come from outside the oracle: Toro's tabulated exact solutions (Table 4.2), the
two-rarefaction closed form (Toro Eq. 4.46), Rankine-Hugoniot and Riemann-invariant
relations, symmetry, and special cases with obvious answers.
"""
import os

import numpy as np
import pytest

G = 1.4
GOLD = os.path.join(os.path.dirname(__file__), "golden", "toro_riemann_tests.txt")


def toro_cases():
    rows = np.loadtxt(GOLD)
    return [tuple(r) for r in rows]


def test_minmod_truth_table(oracle):
    mm = oracle.minmod
    assert mm(1.0, 2.0) == 1.0 and mm(2.0, 1.0) == 1.0
    assert mm(-1.0, -3.0) == -1.0 and mm(-3.0, -0.5) == -0.5
    assert mm(1.0, -1.0) == 0.0 and mm(-2.0, 5.0) == 0.0
    assert mm(0.0, 5.0) == 0.0 and mm(5.0, 0.0) == 0.0 and mm(0.0, 0.0) == 0.0
    assert mm(2.0, 2.0) == 2.0


def test_prim_cons_roundtrip(oracle):
    rng = np.random.default_rng(0)
    for _ in range(50):
        W = np.array([rng.uniform(0.1, 10), *rng.normal(0, 2, 3), rng.uniform(0.1, 10)])
        U = oracle.prim_to_cons(W, G)
        # E by hand for one known case as well
        W2 = oracle.cons_to_prim(U, G)
        assert np.allclose(W2, W, rtol=1e-13, atol=1e-13)
    U = oracle.prim_to_cons(np.array([2.0, 1.0, 0.0, 0.0, 0.4]), G)
    assert np.allclose(U, [2.0, 2.0, 0.0, 0.0, 0.4 / 0.4 + 1.0])


def test_floors(oracle):
    W = oracle.cons_to_prim(np.array([1e-20, 0.0, 0.0, 0.0, -1.0]), G, 1e-10, 1e-20)
    assert W[0] == 1e-10 and W[4] == 1e-20


@pytest.mark.parametrize("case", toro_cases())
def test_exact_star_matches_toro_table(oracle, case):
    _, rL, uL, pL, rR, uR, pR, ps_t, us_t, rsl_t, rsr_t = case
    WL = np.array([rL, uL, 0, 0, pL]); WR = np.array([rR, uR, 0, 0, pR])
    ps, us, st, it = oracle.exact_star(WL, WR, G)
    assert st == oracle.OK
    # the table prints 6 significant figures
    assert abs(ps - ps_t) <= 6e-6 * abs(ps_t) + 5e-6
    assert abs(us - us_t) <= 6e-6 * abs(us_t) + 5e-6
    eps = 1e-9 * max(1.0, abs(us))
    rsl = oracle.exact_sample(WL, WR, G, ps, us, us - eps)[0]
    rsr = oracle.exact_sample(WL, WR, G, ps, us, us + eps)[0]
    assert abs(rsl - rsl_t) <= 6e-6 * rsl_t + 5e-6
    assert abs(rsr - rsr_t) <= 6e-6 * rsr_t + 5e-6


def test_exact_two_rarefaction_closed_form(oracle):
    """When both waves are rarefactions the exact p* has a closed form (Toro Eq. 4.46)."""
    rng = np.random.default_rng(1)
    z = (G - 1) / (2 * G)
    n = 0
    while n < 40:
        rL, rR = rng.uniform(0.1, 5, 2); pL, pR = rng.uniform(0.1, 5, 2)
        uL, uR = -rng.uniform(0, 1.5), rng.uniform(0, 1.5)
        cL, cR = np.sqrt(G * pL / rL), np.sqrt(G * pR / rR)
        ps_trrs = ((cL + cR - 0.5 * (G - 1) * (uR - uL)) / (cL / pL ** z + cR / pR ** z)) ** (1 / z)
        if not (ps_trrs < min(pL, pR)):
            continue
        WL = np.array([rL, uL, 0, 0, pL]); WR = np.array([rR, uR, 0, 0, pR])
        ps, us, st, _ = oracle.exact_star(WL, WR, G)
        assert st == oracle.OK
        assert abs(ps - ps_trrs) <= 1e-12 * ps_trrs
        # u* from the left rarefaction's Riemann invariant u + 2c/(g-1)
        us_inv = uL + 2 * cL / (G - 1) * (1 - (ps / pL) ** z)
        assert abs(us - us_inv) <= 1e-11 * (1 + abs(us))
        n += 1


def test_exact_identical_states(oracle):
    W = np.array([1.3, 0.7, -0.2, 0.4, 2.1])
    ps, us, st, _ = oracle.exact_star(W, W, G)
    assert st == oracle.OK
    assert abs(ps - W[4]) <= 1e-14 * W[4] and abs(us - W[1]) <= 1e-14
    W0 = oracle.exact_sample(W, W, G, ps, us, 0.0)
    assert np.allclose(W0, W, rtol=1e-13, atol=1e-14)


def test_exact_mirror_symmetry(oracle):
    rng = np.random.default_rng(2)
    for _ in range(30):
        WL = np.array([rng.uniform(0.1, 5), rng.normal(), 0, 0, rng.uniform(0.1, 5)])
        WR = np.array([rng.uniform(0.1, 5), rng.normal(), 0, 0, rng.uniform(0.1, 5)])
        ps, us, st, _ = oracle.exact_star(WL, WR, G)
        mL = WR.copy(); mL[1] = -WR[1]
        mR = WL.copy(); mR[1] = -WL[1]
        ps2, us2, st2, _ = oracle.exact_star(mL, mR, G)
        if st != oracle.OK:
            assert st2 == st
            continue
        assert abs(ps - ps2) <= 1e-12 * ps and abs(us + us2) <= 1e-12 * (1 + abs(us))


def test_exact_rankine_hugoniot_and_isentrope(oracle):
    """Shock side: mass and momentum flux are continuous in the shock frame; rarefaction
    side: the star density lies on the isentrope p/rho^g of the initial state."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        WL = np.array([rng.uniform(0.2, 3), rng.normal(0, 1), 0, 0, rng.uniform(0.2, 3)])
        WR = np.array([rng.uniform(0.2, 3), rng.normal(0, 1), 0, 0, rng.uniform(0.2, 3)])
        ps, us, st, _ = oracle.exact_star(WL, WR, G)
        if st != oracle.OK:
            continue
        for side, W in ((0, WL), (1, WR)):
            eps = 1e-9 * (1 + abs(us))
            rs = oracle.exact_sample(WL, WR, G, ps, us, us - eps if side == 0 else us + eps)[0]
            r, u, p = W[0], W[1], W[4]
            if ps > p:
                # shock speed from mass conservation, then momentum must balance
                S = (rs * us - r * u) / (rs - r)
                mom_l = r * u * (u - S) + p
                mom_r = rs * us * (us - S) + ps
                assert abs(mom_l - mom_r) <= 1e-9 * (abs(mom_l) + abs(ps))
            else:
                assert abs(ps / rs ** G - p / r ** G) <= 1e-11 * p / r ** G


def test_exact_vacuum_detected(oracle):
    WL = np.array([1.0, -10.0, 0, 0, 0.4]); WR = np.array([1.0, 10.0, 0, 0, 0.4])
    _, _, st, _ = oracle.exact_star(WL, WR, G)
    assert st == oracle.ENONPHYSICAL


def _phys_flux(W):
    r, u, v, w, p = W
    E = p / (G - 1) + 0.5 * r * (u * u + v * v + w * w)
    return np.array([r * u, r * u * u + p, r * u * v, r * u * w, u * (E + p)])


def test_hllc_consistency_and_supersonic(oracle):
    rng = np.random.default_rng(4)
    for _ in range(30):
        W = np.array([rng.uniform(0.1, 5), *rng.normal(0, 1, 3), rng.uniform(0.1, 5)])
        assert np.allclose(oracle.hllc(W, W, G), _phys_flux(W), rtol=1e-13, atol=1e-13)
        assert np.allclose(oracle.flux_normal(W, G), _phys_flux(W), rtol=1e-14, atol=1e-14)
    # supersonic to the right: upwind (left) flux
    WL = np.array([1.0, 5.0, 0.3, 0.1, 1.0]); WR = np.array([0.5, 4.0, 0.0, 0.0, 0.5])
    assert np.array_equal(oracle.hllc(WL, WR, G), oracle.flux_normal(WL, G))


def test_hllc_resolves_stationary_contact(oracle):
    WL = np.array([1.0, 0.0, 0.3, -0.2, 1.0]); WR = np.array([0.1, 0.0, -0.5, 0.7, 1.0])
    F = oracle.hllc(WL, WR, G)
    assert np.allclose(F, [0.0, 1.0, 0.0, 0.0, 0.0], atol=1e-15)


def test_hllc_close_to_exact_for_weak_waves(oracle):
    """For small jumps the approximate and exact Godunov fluxes agree to second order."""
    prm = oracle.params(gamma=G, riemann=oracle.EXACT)
    rng = np.random.default_rng(5)
    for eps in (1e-2, 1e-3):
        errs = []
        for _ in range(20):
            W = np.array([1.0, 0.3, 0.1, 0.0, 1.0])
            d = rng.normal(0, 1, 5); d[2:4] = 0
            WL, WR = W, W + eps * d
            Fe, _ = oracle.riemann_flux(WL, WR, prm)
            errs.append(np.max(np.abs(oracle.hllc(WL, WR, G) - Fe)))
        assert max(errs) < 50 * eps * eps


def test_exact_flux_falls_back_on_vacuum(oracle):
    prm = oracle.params(gamma=G, riemann=oracle.EXACT)
    WL = np.array([1.0, -10.0, 0, 0, 0.4]); WR = np.array([1.0, 10.0, 0, 0, 0.4])
    F, st = oracle.riemann_flux(WL, WR, prm)
    assert st == oracle.ENONPHYSICAL and np.array_equal(F, oracle.hllc(WL, WR, G))


def _mirror(W):
    return np.array([W[0], -W[1], W[2], W[3], W[4]])


def test_hllc_mirror_symmetry(oracle):
    """Reflecting the problem (x -> -x: the states swap sides and the normal velocity
    changes sign) reflects the flux: mass, transverse-momentum and energy fluxes change
    sign, the normal-momentum flux does not.  The reflection maps every branch of HLLC
    onto its partner (left star <-> right star, left <-> right supersonic), so each
    branch is checked against the other."""
    rng = np.random.default_rng(6)
    branches = set()
    for _ in range(400):
        WL = np.array([rng.uniform(0.1, 5), rng.normal(0, 3), *rng.normal(0, 1, 2), rng.uniform(0.1, 5)])
        WR = np.array([rng.uniform(0.1, 5), rng.normal(0, 3), *rng.normal(0, 1, 2), rng.uniform(0.1, 5)])
        F = oracle.hllc(WL, WR, G)
        Fm = oracle.hllc(_mirror(WR), _mirror(WL), G)
        assert np.allclose(Fm, F * np.array([-1, 1, -1, -1, -1]), rtol=1e-12, atol=1e-12), (WL, WR)
        cL, cR = np.sqrt(G * WL[4] / WL[0]), np.sqrt(G * WR[4] / WR[0])
        SL, SR = min(WL[1] - cL, WR[1] - cR), max(WL[1] + cL, WR[1] + cR)
        branches.add("L" if SL >= 0 else "R" if SR <= 0 else "star")
    assert branches == {"L", "R", "star"}
