"""Pins for the generalised-cost oracle (oracle/cross.py, Sec. IV-D), CPU only.

The oracle's substitution is checked against a dense KKT solve of the
generalised quadratic program, whose cost writes the cross term
(H x - r)^T M (u - s) and the offset 1/2 (u - s)^T U (u - s) out term by term
(tests/kkt.py), so a wrong sign, a dropped term or a transposed operand in
F~, c~, X~ or in the control post-transform changes x*, u*, S, v or K.  Each
planted mistake in a copy of the oracle must fail these pins.
"""
import os
import types

import numpy as np
import pytest

import kkt
from conftest import rel_fro
from paper_2104_03186_gb300 import inputs

CROSS_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         "oracle", "cross.py")


def _cases():
    """(problem, cross terms) pairs: time-varying and time-invariant M, p < n,
    p > n, p = m (a transposed M^T fits the shapes), M only, s only."""
    out = []
    p = inputs.random_problem(3, 2, 2, T=6, seed=3)
    out.append((p, inputs.cross_terms(p, seed=1)))
    p = inputs.random_problem(4, 2, 3, T=7, seed=4, pT=2)
    out.append((p, inputs.cross_terms(p, seed=2, scale=0.8)))
    p = inputs.random_problem(3, 1, 5, T=5, seed=5, time_varying=False)
    out.append((p, inputs.cross_terms(p, seed=3, time_varying=False)))
    p = inputs.random_problem(2, 2, 2, T=4, seed=6)
    out.append((p, inputs.CrossTerms(M=inputs.cross_terms(p, seed=4).M, s=None)))
    p = inputs.random_problem(3, 2, 3, T=5, seed=7, with_c=False)
    out.append((p, inputs.CrossTerms(M=None, s=inputs.cross_terms(p, seed=5).s)))
    return out


def _pins_hold(cross) -> bool:
    """Every pin below, compactly; False as soon as one fails."""
    try:
        for prob, ct in _cases():
            o = cross.riccati_cross(prob, ct.M, ct.s)
            u, x, cost = kkt.solve_from(prob, 0, prob.x0, ct.M, ct.s)
            if rel_fro(o["u"], u) > 1e-10 or rel_fro(o["x"], x) > 1e-10:
                return False
            if abs(kkt.total_cost(prob, o["u"], ct.M, ct.s) - cost) > 1e-9 * max(1, abs(cost)):
                return False
            for k in (0, prob.T - 1):
                S, v, K, _ = kkt.value_function(prob, k, ct.M, ct.s)
                if (np.abs(o["S"][k] - S).max() > 1e-8 or np.abs(o["v"][k] - v).max() > 1e-8
                        or np.abs(o["K"][k] - K).max() > 1e-8):
                    return False
        return True
    except (ArithmeticError, np.linalg.LinAlgError, ValueError):
        return False


def test_cross_pins_hold(orc):
    from oracle import cross

    assert _pins_hold(cross)


@pytest.mark.parametrize("idx", range(5))
def test_cross_trajectory_matches_generalised_kkt(orc, idx):
    from oracle import cross

    prob, ct = _cases()[idx]
    o = cross.riccati_cross(prob, ct.M, ct.s)
    u, x, _ = kkt.solve_from(prob, 0, prob.x0, ct.M, ct.s)
    assert rel_fro(o["x"], x) < 1e-11
    assert rel_fro(o["u"], u) < 1e-11


@pytest.mark.parametrize("idx", range(5))
def test_cross_value_function_and_gain_match_kkt(orc, idx):
    """S_k, v_k and the gain of the original control law u_k(x) = -K_k x + d_k,
    read off the brute-force tail problems."""
    from oracle import cross

    prob, ct = _cases()[idx]
    o = cross.riccati_cross(prob, ct.M, ct.s)
    for k in range(prob.T):
        S, v, K, _ = kkt.value_function(prob, k, ct.M, ct.s)
        np.testing.assert_allclose(o["S"][k], S, atol=1e-8)
        np.testing.assert_allclose(o["v"][k], v, atol=1e-8)
        np.testing.assert_allclose(o["K"][k], K, atol=1e-8)


@pytest.mark.parametrize("seed", range(3))
def test_cross_perturbed_controls_cost_more(orc, seed):
    """Optimality under the generalised cost: J(u* + eps d) - J(u*) grows as
    eps^2 with a positive curvature, and never drops below J(u*)."""
    from oracle import cross

    prob = inputs.random_problem(4, 2, 3, T=8, seed=40 + seed)
    ct = inputs.cross_terms(prob, seed=seed, scale=0.7)
    o = cross.riccati_cross(prob, ct.M, ct.s)
    J0 = kkt.total_cost(prob, o["u"], ct.M, ct.s)
    d = np.random.default_rng(seed).standard_normal(o["u"].shape)
    g = [kkt.total_cost(prob, o["u"] + e * d, ct.M, ct.s) - J0 for e in (1e-2, 2e-2)]
    assert g[0] > 0 and g[1] > 0
    assert abs(g[1] / g[0] - 4.0) < 1e-4


def test_cross_without_cross_terms_is_the_plain_problem(orc):
    """M = 0, s = 0 leaves eq. LQT_problem: the plain sequential oracle."""
    from oracle import cross

    prob = inputs.random_problem(4, 2, 3, T=9, seed=8)
    o = cross.riccati_cross(prob, None, None)
    ref = orc.riccati(prob)
    for f in ("S", "v", "K", "x", "u"):
        assert rel_fro(o[f], ref[f]) < 1e-14


def test_cross_zero_horizon(orc):
    from oracle import cross

    prob = inputs.random_problem(3, 2, 2, T=1, seed=9)
    ct = inputs.cross_terms(prob, seed=9)
    prob.T = 0
    for f in ("F", "c", "L", "U", "H", "r", "X"):
        setattr(prob, f, getattr(prob, f)[:0])
    o = cross.riccati_cross(prob, ct.M[:0], ct.s[:0])
    S, v, _, _ = kkt.value_function(prob, 0)
    np.testing.assert_allclose(o["S"][0], S, atol=1e-10)
    np.testing.assert_allclose(o["v"][0], v, atol=1e-10)
    assert o["K"].shape == (0, 2, 3) and o["u"].shape == (0, 2)


CROSS_MUTATIONS = {
    "W_uses_M_not_transposed": ("np.linalg.solve(U, np.swapaxes(Mk, 1, 2))",
                                "np.linalg.solve(U, Mk)"),
    "F_tilde_sign": ("Ft = F - L @ WH", "Ft = F + L @ WH"),
    "c_tilde_drops_Ls": ('np.einsum("kij,kj->ki", W, r) + sk)', 'np.einsum("kij,kj->ki", W, r))'),
    "c_tilde_sign_of_r_term": ('np.einsum("kij,kj->ki", W, r) + sk)',
                               '-np.einsum("kij,kj->ki", W, r) + sk)'),
    "X_tilde_sign": ("Xt = X - Mk @ W", "Xt = X + Mk @ W"),
    "u_drops_offset": ('np.einsum("kij,kj->ki", W, e) + sk', 'np.einsum("kij,kj->ki", W, e)'),
    "u_error_sign_of_r": ('o["x"][:T]) - r', 'o["x"][:T]) + r'),
    "K_without_WH": ('K = o["K"] + WH', 'K = o["K"]'),
}


@pytest.mark.parametrize("name", sorted(CROSS_MUTATIONS))
def test_cross_pins_catch_planted_mistake(orc, name):
    before, after = CROSS_MUTATIONS[name]
    src = open(CROSS_SRC).read()
    assert src.count(before) == 1, "mutation anchor must be unique: " + name
    mod = types.ModuleType("oracle._cross_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(before, after), "cross_mutant.py", "exec"), mod.__dict__)
    assert not _pins_hold(mod), name
