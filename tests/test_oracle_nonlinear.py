"""Pins for the iterated nonlinear LQT oracle (oracle/nonlinear.py,
Sec. IV-D and Sec. VI-E), CPU only.

* The unicycle Jacobians against central differences of f.
* A linear model: one linearise-and-solve pass is the LQT solution, and later
  passes leave it unchanged.
* The converged unicycle trajectory: it satisfies the true nonlinear dynamics,
  and the gradient of the nonlinear cost J(u) = cost(rollout_f(u)), taken by
  central differences through the model alone, vanishes there.
* Planted mistakes in a copy of the oracle fail these pins.
"""
import os
import types

import numpy as np
import pytest

from conftest import rel_fro
from paper_2104_03186_gb300 import inputs

NL_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "oracle", "nonlinear.py")


class LinearModel:
    """f(x, u) = F x + c + L u with one (F, c, L) for every step."""

    def __init__(self, F, c, L):
        self.F, self.c, self.L = F, c, L
        self.n, self.m = L.shape

    def f(self, x, u):
        return x @ self.F.T + self.c + u @ self.L.T

    def jacobians(self, x, u):
        K = x.shape[0]
        return (np.broadcast_to(self.F, (K,) + self.F.shape).copy(),
                np.broadcast_to(self.L, (K,) + self.L.shape).copy())


def _nonlinear_cost(prob, x, u):
    """Cost of eq. nonlinear_system with h(x) = H x, g(u) = u, s = 0."""
    T = prob.T
    J = 0.0
    for k in range(T):
        e = prob.H[0] @ x[k] - prob.r[k]
        J += 0.5 * e @ prob.X[k] @ e + 0.5 * u[k] @ prob.U[0] @ u[k]
    e = prob.HT @ x[T] - prob.rT
    return J + 0.5 * e @ prob.XT @ e


def _fd_jacobians(model, x, u, h=1e-6):
    n, m = x.shape[-1], u.shape[-1]
    Jx = np.zeros((n, n))
    Ju = np.zeros((n, m))
    for j in range(n):
        d = np.zeros(n)
        d[j] = h
        Jx[:, j] = (model.f((x + d)[None], u[None])[0] - model.f((x - d)[None], u[None])[0]) / (2 * h)
    for j in range(m):
        d = np.zeros(m)
        d[j] = h
        Ju[:, j] = (model.f(x[None], (u + d)[None])[0] - model.f(x[None], (u - d)[None])[0]) / (2 * h)
    return Jx, Ju


def _pins_hold(nl) -> bool:
    try:
        # Jacobians against central differences
        rng = np.random.default_rng(0)
        mdl = nl.Unicycle(0.1)
        xs = rng.standard_normal((5, 4)) * np.array([3, 3, 2, 2])
        us = rng.standard_normal((5, 2))
        Jx, Ju = mdl.jacobians(xs, us)
        for i in range(5):
            fx, fu = _fd_jacobians(mdl, xs[i], us[i])
            if np.abs(Jx[i] - fx).max() > 1e-8 or np.abs(Ju[i] - fu).max() > 1e-8:
                return False
        # a linear model: one pass = the LQT solution; further passes fixed
        import oracle

        prob = inputs.random_problem(3, 2, 2, T=9, seed=1, time_varying=False)
        lin = LinearModel(prob.F[0], prob.c[0], prob.L[0])
        ref = oracle.riccati(prob, keep_kv_kc=False)
        for passes in (1, 3):
            o = nl.iterated_lqt(lin, prob, passes)
            if any(rel_fro(o[f], ref[f]) > 1e-12 for f in ("S", "v", "K", "x", "u")):
                return False
        # the converged unicycle: true dynamics and a stationary nonlinear cost
        prob = inputs.unicycle_track(24, seed=2, ref_every=3)
        o = nl.iterated_lqt(mdl, prob, 30)
        if np.abs(nl.rollout(mdl, prob.x0, o["u"]) - o["x"]).max() > 1e-9:
            return False
        u = o["u"]
        h = 1e-6
        g = np.zeros_like(u)
        for k in range(u.shape[0]):
            for j in range(u.shape[1]):
                d = np.zeros_like(u)
                d[k, j] = h
                g[k, j] = (_nonlinear_cost(prob, nl.rollout(mdl, prob.x0, u + d), u + d)
                           - _nonlinear_cost(prob, nl.rollout(mdl, prob.x0, u - d), u - d)) / (2 * h)
        g0 = np.zeros_like(u)
        z = np.zeros_like(u)
        for k in range(u.shape[0]):
            for j in range(u.shape[1]):
                d = np.zeros_like(u)
                d[k, j] = h
                g0[k, j] = (_nonlinear_cost(prob, nl.rollout(mdl, prob.x0, z + d), z + d)
                            - _nonlinear_cost(prob, nl.rollout(mdl, prob.x0, z - d), z - d)) / (2 * h)
        return bool(np.abs(g).max() < 1e-5 * np.abs(g0).max())
    except (ArithmeticError, np.linalg.LinAlgError, ValueError, IndexError):
        return False


def test_nonlinear_pins_hold(orc):
    from oracle import nonlinear

    assert _pins_hold(nonlinear)


def test_unicycle_jacobians_match_central_differences(orc):
    from oracle import nonlinear as nl

    mdl = nl.Unicycle(0.25)
    rng = np.random.default_rng(3)
    xs = rng.standard_normal((8, 4)) * np.array([5, 5, 4, 3])
    us = rng.standard_normal((8, 2))
    Jx, Ju = mdl.jacobians(xs, us)
    for i in range(8):
        fx, fu = _fd_jacobians(mdl, xs[i], us[i])
        np.testing.assert_allclose(Jx[i], fx, atol=1e-8)
        np.testing.assert_allclose(Ju[i], fu, atol=1e-8)


def test_linearisation_is_exact_at_the_nominal(orc):
    """The affine model F x + c + L u equals f at (x̄, ū) and agrees to second
    order nearby (eq. nonlinear_linarisation)."""
    from oracle import nonlinear as nl

    mdl = nl.Unicycle(0.1)
    prob = inputs.unicycle_track(6, seed=1)
    rng = np.random.default_rng(4)
    xb = rng.standard_normal((7, 4))
    ub = rng.standard_normal((6, 2))
    lin = nl.linearise(mdl, prob, xb, ub)
    aff = np.einsum("kij,kj->ki", lin.F, xb[:6]) + lin.c + np.einsum("kij,kj->ki", lin.L, ub)
    np.testing.assert_allclose(aff, mdl.f(xb[:6], ub), atol=1e-14)
    dx = 1e-3 * rng.standard_normal((6, 4))
    aff2 = np.einsum("kij,kj->ki", lin.F, xb[:6] + dx) + lin.c + \
        np.einsum("kij,kj->ki", lin.L, ub)
    assert np.abs(aff2 - mdl.f(xb[:6] + dx, ub)).max() < 1e-5


@pytest.mark.parametrize("passes", [1, 2, 4])
def test_linear_model_passes_equal_the_lqt_solution(orc, passes):
    from oracle import nonlinear as nl

    prob = inputs.random_problem(4, 2, 3, T=12, seed=5, time_varying=False)
    lin = LinearModel(prob.F[0], prob.c[0], prob.L[0])
    ref = orc.riccati(prob)
    o = nl.iterated_lqt(lin, prob, passes)
    for f in ("S", "v", "K", "x", "u"):
        assert rel_fro(o[f], ref[f]) < 1e-12


def test_unicycle_converges_to_a_stationary_point(orc):
    """After the passes settle, x* is the rollout of the true dynamics under u*
    and the nonlinear cost has zero gradient in u (central differences)."""
    from oracle import nonlinear as nl

    assert _pins_hold(nl)
    mdl = nl.Unicycle(0.1)
    prob = inputs.unicycle_track(2000, seed=0)
    o = nl.iterated_lqt(mdl, prob, 10, keep_history=True)
    steps = [np.abs(a[0] - b[0]).max() for a, b in zip(o["history"][1:], o["history"][:-1])]
    assert steps[-1] < 1e-8 * max(steps[0], 1.0)
    assert np.abs(nl.rollout(mdl, prob.x0, o["u"]) - o["x"]).max() < 1e-8


NL_MUTATIONS = {
    "dpx_dtheta_sign": ("Jx[:, 0, 2] = -s * np.sin(th) * dt", "Jx[:, 0, 2] = s * np.sin(th) * dt"),
    "dpx_ds_sin": ("Jx[:, 0, 3] = np.cos(th) * dt", "Jx[:, 0, 3] = np.sin(th) * dt"),
    "controls_swapped": ("Ju[:, 2, 1] = dt", "Ju[:, 2, 0] = dt"),
    "offset_drops_Fx": ('ck = model.f(xbar[:T], ubar) - np.einsum("kij,kj->ki", Fk, xbar[:T])',
                        'ck = model.f(xbar[:T], ubar) - 0 * np.einsum("kij,kj->ki", Fk, xbar[:T])'),
    "nominal_off_by_one": ("Fk, Lk = model.jacobians(xbar[:T], ubar)",
                           "Fk, Lk = model.jacobians(xbar[1:T + 1], ubar)"),
    "f_heading_uses_a": ("th + om * dt,", "th + a * dt,"),
}


@pytest.mark.parametrize("name", sorted(NL_MUTATIONS))
def test_nonlinear_pins_catch_planted_mistake(orc, name):
    before, after = NL_MUTATIONS[name]
    src = open(NL_SRC).read()
    assert src.count(before) == 1, "mutation anchor must be unique: " + name
    mod = types.ModuleType("oracle._nonlinear_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(before, after), "nonlinear_mutant.py", "exec"), mod.__dict__)
    assert not _pins_hold(mod), name
