"""FP64 oracle for the iterated nonlinear LQT -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.

Sec. IV-D ("Extension to nonlinear control"), eq. nonlinear_system and
eq. nonlinear_linarisation: for dynamics x_{k+1} = f_k(x_k, u_k) and a
quadratic tracking cost in h_n(x) = H_n x and g_n(u) = u (the form of the
unicycle experiment, Sec. VI-E), each pass

  1. linearises f around the nominal trajectory (x̄_k, ū_k) by its first-order
     Taylor series, f(x, u) ≈ f(x̄, ū) + J^x (x - x̄) + J^u (u - ū), which is the
     affine dynamics of eq. LQT_problem with F_k = J^x, L_k = J^u and
     c_k = f(x̄_k, ū_k) - J^x x̄_k - J^u ū_k;
  2. solves that LQT problem (here by the sequential FP64 recursion of
     Sec. II-B, ``oracle.riccati``);
  3. takes its optimal states and controls as the next nominal trajectory.

The first nominal is x̄_k = x_0 for every k and ū_k = 0 (one of the two
initialisations the paper names) unless one is given.

The unicycle of Sec. VI-E: state (p_x, p_y, theta, s), control (a, omega),
f(x, u) = (p_x + s cos(theta) dt, p_y + s sin(theta) dt, theta + omega dt, s + a dt).

Pinned in ``tests/test_oracle_nonlinear.py``: Jacobians against central
differences of f, a linear model (one pass = the LQT solution, later passes
fixed), the converged unicycle trajectory against the true dynamics and
against a finite-difference gradient of the nonlinear cost, and planted
mistakes.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import riccati as _riccati


class Unicycle:
    """The unicycle model of Sec. VI-E with time step dt (n = 4, m = 2)."""

    n, m = 4, 2

    def __init__(self, dt: float = 0.1):
        self.dt = dt

    def f(self, x, u):
        """x_{k+1} = f(x_k, u_k) for stacks x (K, 4), u (K, 2)."""
        dt = self.dt
        px, py, th, s = x[..., 0], x[..., 1], x[..., 2], x[..., 3]
        a, om = u[..., 0], u[..., 1]
        return np.stack([px + s * np.cos(th) * dt, py + s * np.sin(th) * dt, th + om * dt,
                         s + a * dt], axis=-1)

    def jacobians(self, x, u):
        """(J^x, J^u) of f at stacks x (K, 4), u (K, 2): (K, 4, 4), (K, 4, 2)."""
        dt = self.dt
        K = x.shape[0]
        th, s = x[:, 2], x[:, 3]
        Jx = np.zeros((K, 4, 4))
        Jx[:, 0, 0] = 1.0
        Jx[:, 1, 1] = 1.0
        Jx[:, 2, 2] = 1.0
        Jx[:, 3, 3] = 1.0
        Jx[:, 0, 2] = -s * np.sin(th) * dt   # d(p_x')/d theta
        Jx[:, 0, 3] = np.cos(th) * dt        # d(p_x')/d s
        Jx[:, 1, 2] = s * np.cos(th) * dt    # d(p_y')/d theta
        Jx[:, 1, 3] = np.sin(th) * dt        # d(p_y')/d s
        Ju = np.zeros((K, 4, 2))
        Ju[:, 2, 1] = dt                     # d theta' / d omega
        Ju[:, 3, 0] = dt                     # d s' / d a
        return Jx, Ju


def linearise(model, prob, xbar, ubar):
    """The LQT problem of eq. LQT_problem whose dynamics are the first-order
    Taylor expansion of the model around (xbar_k, ubar_k), k = 0..T-1."""
    T = prob.T
    Fk, Lk = model.jacobians(xbar[:T], ubar)
    ck = model.f(xbar[:T], ubar) - np.einsum("kij,kj->ki", Fk, xbar[:T]) \
        - np.einsum("kij,kj->ki", Lk, ubar)
    return dataclasses.replace(prob, F=Fk, L=Lk, c=ck)


def iterated_lqt(model, prob, iterations: int, x_init=None, u_init=None,
                 keep_history: bool = False) -> dict:
    """Runs `iterations` linearise-and-solve passes (Sec. IV-D).  `prob` holds
    the cost (H, r, X, U, terminal terms) and x_0; its F, L, c are ignored.
    Returns the last pass's solution (S, v, K of the last linearisation, and
    x, u = the final nominal trajectory); with keep_history the nominal
    trajectories of every pass under "history"."""
    T, n, m = prob.T, prob.n, prob.m
    xbar = np.broadcast_to(prob.x0, (T + 1, n)).copy() if x_init is None else np.array(x_init)
    ubar = np.zeros((T, m)) if u_init is None else np.array(u_init)
    hist = []
    out = None
    for _ in range(iterations):
        lin = linearise(model, prob, xbar, ubar)
        out = _riccati(lin, keep_kv_kc=False)
        xbar, ubar = out["x"], out["u"]
        if keep_history:
            hist.append((xbar.copy(), ubar.copy()))
    if keep_history:
        out["history"] = hist
    return out


def rollout(model, x0, u):
    """States of the true nonlinear dynamics under controls u (T, m)."""
    x = [np.asarray(x0, dtype=np.float64)]
    for k in range(u.shape[0]):
        x.append(model.f(x[-1][None], u[k][None])[0])
    return np.stack(x)
