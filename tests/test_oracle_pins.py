"""Pins of the FP64 oracle to things other than itself (CPU only).

* dense KKT brute force of the quadratic program (eq. LQT_problem);
* the closed-form scalar steady-state Riccati solution;
* a T = 1 scalar problem solved by hand;
* invariants: S_k symmetric PSD, v = 0 for the regulator, zero adjoint
  gradient at u*, strictly positive second-order cost change;
* the operator of eq. lqt_comb against a brute-force minimisation over the
  middle state (Theorem v-comb with eq. V_ki_invertible_C), its
  associativity and neutral element;
* Lemma LQT_assoc (suffix fold = value function), Lemma lqt_fwd_init
  (forward affine fold = x*), Lemma LQT_trajectory_method2.
"""
import json
import math
import os

import numpy as np
import pytest

import kkt
from conftest import rel_fro
from paper_2104_03186_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SMALL = [
    dict(n=1, m=1, p=1, T=5, seed=1),
    dict(n=2, m=1, p=1, T=6, seed=2),
    dict(n=3, m=2, p=2, T=7, seed=3),
    dict(n=4, m=2, p=3, T=8, seed=4, pT=2),
    dict(n=4, m=4, p=4, T=5, seed=5, x_rank=2),
    dict(n=4, m=1, p=4, T=8, seed=6, time_varying=False),
]


def _problems():
    for kw in SMALL:
        yield inputs.random_problem(**kw)
    yield inputs.vehicle(8, seed=0)
    yield inputs.paper_tracking(9, seed=0)


# --------------------------------------------------------------------------
# golden: the vehicle model as printed in Sec. VI-A
# --------------------------------------------------------------------------

def test_vehicle_model_matches_printed_matrices():
    with open(os.path.join(GOLDEN, "vehicle_model.json")) as f:
        g = json.load(f)
    F, L = inputs.vehicle_model(g["dt"])
    assert np.array_equal(F, np.array(g["F"]))
    assert np.allclose(L, np.array(g["L"]), rtol=0, atol=1e-15)
    p = inputs.vehicle(5, seed=0)
    assert np.array_equal(p.H[0], np.array(g["H"]))
    assert np.allclose(p.U[0], np.array(g["U"]), rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# KKT brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("idx", range(len(SMALL) + 2))
def test_trajectory_matches_kkt(orc, idx):
    prob = list(_problems())[idx]
    o = orc.riccati(prob)
    u, x, _ = kkt.solve_from(prob, 0, prob.x0)
    assert rel_fro(o["u"], u) < 1e-10
    assert rel_fro(o["x"], x) < 1e-10


@pytest.mark.parametrize("idx", range(len(SMALL) + 2))
def test_value_function_and_gains_match_kkt(orc, idx):
    prob = list(_problems())[idx]
    o = orc.riccati(prob)
    for k in sorted({0, prob.T // 2, prob.T - 1, prob.T}):
        S, v, K, ff = kkt.value_function(prob, k)
        scale = max(1.0, np.abs(S).max())
        assert np.abs(o["S"][k] - S).max() < 1e-8 * scale, k
        assert np.abs(o["v"][k] - v).max() < 1e-8 * max(1.0, np.abs(v).max()), k
        if k < prob.T:
            assert np.abs(o["K"][k] - K).max() < 1e-8 * max(1.0, np.abs(K).max()), k
            c = np.zeros(prob.n) if prob.c is None else prob.c[0 if prob.c.shape[0] == 1 else k]
            ff_o = o["Kv"][k] @ o["v"][k + 1] - o["Kc"][k] @ c
            assert np.abs(ff_o - ff).max() < 1e-8 * max(1.0, np.abs(ff).max()), k


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def _dare_scalar(a, b, q, rho):
    beta = rho * (1 - a * a) - q * b * b
    return (-beta + math.sqrt(beta * beta + 4 * b * b * q * rho)) / (2 * b * b)


@pytest.mark.parametrize("a,b,q,rho", [(1.0, 0.1, 1.0, 0.1), (1.2, 1.0, 2.0, 1.0),
                                       (0.5, 2.0, 0.3, 5.0), (1.05, 0.3, 1.0, 1e-2)])
def test_scalar_steady_state_riccati(orc, a, b, q, rho):
    Sinf = _dare_scalar(a, b, q, rho)
    # started at the fixed point it stays there
    o = orc.riccati(inputs.scalar_lqr(a, b, q, rho, T=50, s_terminal=Sinf))
    assert np.abs(o["S"][:, 0, 0] - Sinf).max() < 1e-12 * Sinf
    Kinf = b * Sinf * a / (b * b * Sinf + rho)
    assert np.abs(o["K"][:, 0, 0] - Kinf).max() < 1e-12 * max(1.0, abs(Kinf))
    # from another terminal weight it converges geometrically
    o = orc.riccati(inputs.scalar_lqr(a, b, q, rho, T=400, s_terminal=0.0))
    assert abs(o["S"][0, 0, 0] - Sinf) < 1e-10 * Sinf
    d = np.abs(o["S"][:, 0, 0] - Sinf)
    assert d[200] <= d[300] + 1e-15 and d[300] <= d[399] + 1e-15
    # regulator: no tracking terms, so v = 0 and u = -K x
    assert np.all(o["v"] == 0.0)


def test_hand_solved_one_step_problem(orc):
    """T = 1, n = m = p = 1: minimise 1/2 q (x0 - r0)^2 + 1/2 rho u^2
    + 1/2 qT (a x0 + c + b u - rT)^2 by hand."""
    a, b, c, q, rho, qT, r0, rT, x0 = 0.9, 0.7, 0.3, 2.0, 0.5, 3.0, 0.4, -1.1, 1.7
    one = np.ones((1, 1, 1))
    prob = inputs.LQTProblem(F=a * one, c=np.array([[c]]), L=b * one, U=rho * one, H=one.copy(),
                             r=np.array([[r0]]), X=q * one, HT=np.ones((1, 1)), rT=np.array([rT]),
                             XT=np.array([[qT]]), x0=np.array([x0]), T=1)
    o = orc.riccati(prob)
    u = -b * qT * (a * x0 + c - rT) / (rho + b * b * qT)
    K = b * qT * a / (b * b * qT + rho)
    S0 = a * a * qT * rho / (b * b * qT + rho) + q
    v0 = (a - b * K) * (qT * rT - qT * c) + q * r0
    assert abs(o["u"][0, 0] - u) < 1e-14
    assert abs(o["x"][1, 0] - (a * x0 + c + b * u)) < 1e-14
    assert abs(o["S"][1, 0, 0] - qT) < 1e-15 and abs(o["v"][1, 0] - qT * rT) < 1e-15
    assert abs(o["K"][0, 0, 0] - K) < 1e-14
    assert abs(o["S"][0, 0, 0] - S0) < 1e-14 and abs(o["v"][0, 0] - v0) < 1e-14


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("idx", range(len(SMALL) + 2))
def test_value_matrix_symmetric_psd(orc, idx):
    prob = list(_problems())[idx]
    S = orc.riccati(prob)["S"]
    for Sk in S:
        sc = max(1.0, np.abs(Sk).max())
        assert np.abs(Sk - Sk.T).max() < 1e-12 * sc
        assert np.linalg.eigvalsh(0.5 * (Sk + Sk.T)).min() > -1e-10 * sc


def test_regulator_has_zero_v(orc):
    prob = inputs.random_problem(4, 2, 4, T=30, seed=9, with_c=False)
    prob.r = None
    prob.rT = None
    prob.H = np.eye(4)[None]
    prob.HT = np.eye(4)
    o = orc.riccati(prob)
    assert np.all(o["v"] == 0.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_gradient_vanishes_at_optimum(orc, seed):
    prob = inputs.random_problem(4, 2, 3, T=40, seed=seed)
    o = orc.riccati(prob)
    x, u = o["x"], o["u"]
    T = prob.T
    step = kkt._step
    lam = prob.HT.T @ prob.XT @ (prob.HT @ x[T] - prob.rT)
    grad = np.zeros_like(u)
    for t in range(T - 1, -1, -1):
        grad[t] = step(prob.U, t) @ u[t] + step(prob.L, t).T @ lam
        H, X = step(prob.H, t), step(prob.X, t)
        lam = step(prob.F, t).T @ lam + H.T @ X @ (H @ x[t] - step(prob.r, t))
    assert np.abs(grad).max() < 1e-10 * max(1.0, np.abs(u).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_perturbed_controls_cost_more_quadratically(orc, seed):
    prob = inputs.random_problem(3, 2, 2, T=25, seed=seed)
    u = orc.riccati(prob)["u"]
    J0 = kkt.total_cost(prob, u)
    rng = np.random.default_rng(100 + seed)
    for _ in range(5):
        d = rng.standard_normal(u.shape)
        d1 = kkt.total_cost(prob, u + 1e-2 * d) - J0
        d2 = kkt.total_cost(prob, u + 2e-2 * d) - J0
        assert d1 > 0 and d2 > 0
        assert abs(d2 / d1 - 4.0) < 1e-5


# --------------------------------------------------------------------------
# the associative operator
# --------------------------------------------------------------------------

def _rand_elem(rng, n, invertible_C=False):
    A = rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    B = rng.standard_normal((n, n if invertible_C else max(1, n // 2)))
    C = B @ B.T + (0.5 * np.eye(n) if invertible_C else 0)
    D = rng.standard_normal((n, n))
    J = D @ D.T / n
    eta = rng.standard_normal(n)
    return A, b, C, eta, J


def _cond_value(e, x, y):
    """V(x, y) of eq. V_ki_invertible_C without its constant."""
    A, b, C, eta, J = e
    d = y - A @ x - b
    return 0.5 * x @ J @ x - x @ eta + 0.5 * d @ np.linalg.solve(C, d)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_combine_equals_minimisation_over_middle_state(orc, n):
    rng = np.random.default_rng(n)
    a = _rand_elem(rng, n, invertible_C=True)
    b = _rand_elem(rng, n, invertible_C=True)
    ab = orc.combine(a, b)

    def brute(x, y):
        # min_z V_a(x, z) + V_b(z, y): quadratic in z, minimiser from its gradient
        Ca_inv = np.linalg.inv(a[2])
        Cb_inv = np.linalg.inv(b[2])
        Ab, bb = b[0], b[1]
        Hz = Ca_inv + b[4] + Ab.T @ Cb_inv @ Ab
        gz = Ca_inv @ (a[0] @ x + a[1]) + b[3] + Ab.T @ Cb_inv @ (y - bb)
        z = np.linalg.solve(Hz, gz)
        return _cond_value(a, x, z) + _cond_value(b, z, y)

    pts = [(rng.standard_normal(n), rng.standard_normal(n)) for _ in range(6)]
    ref = [brute(x, y) - brute(np.zeros(n), np.zeros(n)) for x, y in pts]
    got = [_cond_value(ab, x, y) - _cond_value(ab, np.zeros(n), np.zeros(n)) for x, y in pts]
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("n", [1, 2, 4, 5])
def test_combine_is_associative_with_neutral_element(orc, n):
    import oracle

    rng = np.random.default_rng(10 + n)
    a, b, c = (_rand_elem(rng, n) for _ in range(3))
    left = orc.combine(orc.combine(a, b), c)
    right = orc.combine(a, orc.combine(b, c))
    for L_, R_ in zip(left, right):
        assert rel_fro(L_, R_) < 1e-12
    e = oracle.neutral(n)
    for got in (orc.combine(a, e), orc.combine(e, a)):
        for g, w in zip(got, a):
            assert np.abs(g - w).max() < 1e-14 * max(1.0, np.abs(w).max())


@pytest.mark.parametrize("idx", range(len(SMALL) + 2))
def test_suffix_fold_of_elements_is_value_function(orc, idx):
    """Lemma LQT_assoc: a_k (x) ... (x) a_T has A = b = C = 0, J = S_k, eta = v_k."""
    prob = list(_problems())[idx]
    o = orc.riccati(prob)
    s = orc.element(prob, prob.T)
    assert np.all(s[0] == 0) and np.all(s[1] == 0) and np.all(s[2] == 0)
    for k in range(prob.T, -1, -1):
        if k < prob.T:
            s = orc.combine(orc.element(prob, k), s)
        assert np.all(s[0] == 0) and np.all(s[1] == 0) and np.all(s[2] == 0)
        assert rel_fro(s[4], o["S"][k]) < 1e-10, k
        assert rel_fro(s[3], o["v"][k]) < 1e-10, k


@pytest.mark.parametrize("idx", range(len(SMALL) + 2))
def test_forward_affine_fold_is_optimal_trajectory(orc, idx):
    """Lemma lqt_fwd_init with the closed-loop maps of Sec. IV-C (Method 1)."""
    prob = list(_problems())[idx]
    o = orc.riccati(prob)
    n = prob.n
    step = kkt._step
    maps = []
    for k in range(prob.T):
        F, L = step(prob.F, k), step(prob.L, k)
        c = np.zeros(n) if prob.c is None else step(prob.c, k)
        Ft = F - L @ o["K"][k]
        ct = c + L @ o["Kv"][k] @ o["v"][k + 1] - L @ o["Kc"][k] @ c
        maps.append((Ft, ct))
    first = (np.zeros((n, n)), maps[0][0] @ prob.x0 + maps[0][1])
    acc = first
    assert rel_fro(acc[1], o["x"][1]) < 1e-12
    for k in range(1, prob.T):
        acc = orc.affine_combine(acc, maps[k])
        assert np.all(acc[0] == 0)
        assert rel_fro(acc[1], o["x"][k + 1]) < 1e-10, k
    # the operator is composition: check against applying both maps
    rng = np.random.default_rng(0)
    f1 = (rng.standard_normal((n, n)), rng.standard_normal(n))
    f2 = (rng.standard_normal((n, n)), rng.standard_normal(n))
    F, c = orc.affine_combine(f1, f2)
    y = rng.standard_normal(n)
    assert np.allclose(F @ y + c, f2[0] @ (f1[0] @ y + f1[1]) + f2[1], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("idx", range(len(SMALL) + 2))
def test_method2_recovers_optimal_trajectory(orc, idx):
    """Remark LQT_init2 + forward fold + eq. lqt_method_2 give x*_k."""
    prob = list(_problems())[idx]
    o = orc.riccati(prob)
    n = prob.n
    acc = (np.zeros((n, n)), prob.x0.copy(), np.zeros((n, n)), np.zeros(n), np.zeros((n, n)))
    for k in range(prob.T + 1):
        x = orc.method2_state(acc, o["S"][k], o["v"][k], prob.x0)
        assert rel_fro(x, o["x"][k]) < 1e-9, k
        if k < prob.T:
            acc = orc.combine(acc, orc.element(prob, k))


def test_element_formulas(orc):
    """eq. lqt_init on one random step, including the terminal reading
    eta_T = H_T^T X_T r_T."""
    prob = inputs.random_problem(3, 2, 2, T=4, seed=7, pT=3)
    k = 2
    A, b, C, eta, J = orc.element(prob, k)
    assert np.array_equal(A, prob.F[k]) and np.array_equal(b, prob.c[k])
    assert np.allclose(C, prob.L[k] @ np.linalg.inv(prob.U[k]) @ prob.L[k].T, rtol=1e-13)
    assert np.allclose(J, prob.H[k].T @ prob.X[k] @ prob.H[k], rtol=1e-13)
    assert np.allclose(eta, prob.H[k].T @ prob.X[k] @ prob.r[k], rtol=1e-13)
    A, b, C, eta, J = orc.element(prob, prob.T)
    assert np.all(A == 0) and np.all(b == 0) and np.all(C == 0)
    assert np.allclose(eta, prob.HT.T @ prob.XT @ prob.rT, rtol=1e-13)
