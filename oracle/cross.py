"""FP64 oracle for the generalised stage cost -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.

Sec. IV-D ("Extension to more general cost functions"), eq. generalised_cost:
the stage cost of eq. LQT_problem gains a cross term and a control offset,

    l_k(x, u) = 1/2 (H_k x - r_k)^T X_k (H_k x - r_k)
              + (H_k x - r_k)^T M_k (u - s_k)
              + 1/2 (u - s_k)^T U_k (u - s_k),

with M_k of size p x m and s_k of size m (the terminal cost is unchanged).
The paper factors the joint weight [[X, M], [M^T, U]] into
E^T blockdiag(X - M U^{-1} M^T, U) E with E = [[I, 0], [U^{-1} M^T, I]] and
substitutes u~_k = U_k^{-1} M_k^T (H_k x_k - r_k) + u_k - s_k, which turns the
problem into one of the form eq. LQT_problem with

    F~_k = F_k - L_k U_k^{-1} M_k^T H_k
    c~_k = c_k + L_k U_k^{-1} M_k^T r_k + L_k s_k
    X~_k = X_k - M_k U_k^{-1} M_k^T
    U~_k = U_k            (H_k, r_k, L_k and the terminal terms unchanged).

That problem is solved by the sequential FP64 recursion of Sec. II-B
(``oracle.riccati``); its value function is the original one (same S_k, v_k),
its states are the original optimal states, and the original controls come
back as u_k = u~_k - U_k^{-1} M_k^T (H_k x_k - r_k) + s_k.  Because
u~_k = -K~_k x_k + (terms free of x_k), the feedback gain of the original
control law is K_k = K~_k + U_k^{-1} M_k^T H_k.

Pinned by a dense KKT solve of the generalised quadratic program
(``tests/kkt.py``, with the cross term and offset written out in the cost),
by the value function read off that solve, and by planted mistakes
(``tests/test_oracle_cross.py``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import riccati as _riccati


def _per_step(a, T):
    """(T, ...) view of a per-step array with a leading axis of 1 or T."""
    return np.broadcast_to(a, (T,) + a.shape[1:]) if a.shape[0] == 1 else a


def transform(prob, M, s):
    """The substitution of Sec. IV-D: returns (transformed problem, W, WH) with
    W_k = U_k^{-1} M_k^T (m x p) and WH_k = W_k H_k (m x n), every per-step
    array expanded to T rows.  M or s may be None (zero)."""
    T, n, m, p = prob.T, prob.n, prob.m, prob.p
    F = _per_step(prob.F, T)
    L = _per_step(prob.L, T)
    U = _per_step(prob.U, T)
    H = _per_step(prob.H, T)
    X = _per_step(prob.X, T)
    c = np.zeros((T, n)) if prob.c is None else _per_step(prob.c, T)
    r = np.zeros((T, p)) if prob.r is None else _per_step(prob.r, T)
    Mk = np.zeros((T, p, m)) if M is None else _per_step(M, T)
    sk = np.zeros((T, m)) if s is None else _per_step(s, T)

    # per step k (batched over the time axis):
    W = np.linalg.solve(U, np.swapaxes(Mk, 1, 2)) if T > 0 else np.zeros((0, m, p))  # U^{-1} M^T
    WH = W @ H                                                      # U^{-1} M^T H
    Ft = F - L @ WH                                                 # F~
    ct = c + np.einsum("kij,kj->ki", L, np.einsum("kij,kj->ki", W, r) + sk)  # c~
    Xt = X - Mk @ W                                                 # X~
    tp = dataclasses.replace(prob, F=Ft, c=ct, L=np.array(L), U=np.array(U), H=np.array(H),
                             r=np.array(r), X=Xt)
    return tp, W, WH


def riccati_cross(prob, M, s) -> dict:
    """Optimal solution of the generalised-cost problem (Sec. IV-D):
    S, v (T+1 rows), K (the original control law's gains), x, u."""
    T, p = prob.T, prob.p
    tp, W, WH = transform(prob, M, s)
    o = _riccati(tp, keep_kv_kc=False)
    H = _per_step(prob.H, T)
    r = np.zeros((T, p)) if prob.r is None else _per_step(prob.r, T)
    sk = np.zeros((T, prob.m)) if s is None else _per_step(s, T)
    e = np.einsum("kij,kj->ki", H, o["x"][:T]) - r          # H x - r at the optimum
    u = o["u"] - np.einsum("kij,kj->ki", W, e) + sk          # u = u~ - U^{-1} M^T (H x - r) + s
    K = o["K"] + WH                                          # K = K~ + U^{-1} M^T H
    return {"S": o["S"], "v": o["v"], "K": K, "x": o["x"], "u": u}
