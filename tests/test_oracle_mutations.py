"""The pins must catch plausible mistakes in the oracle (CPU only).

Each case plants one mistake (a dropped term, a wrong sign, a transposed
operand, a wrong index) in a temporary copy of ``oracle/lqt_oracle.c``,
compiles it, and checks that at least one pin of ``test_oracle_pins`` fails
for the mutant while all of them pass for the real oracle.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import kkt
from conftest import rel_fro
from paper_2104_03186_gb300 import inputs

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "lqt_oracle.c")

MUTATIONS = {
    "v_recursion_sign_of_Sc": ("w[i] = vn[i] - Sc[i];", "w[i] = vn[i] + Sc[i];"),
    "S_recursion_F_not_transposed": ("mtm(F, SFcl, Sk, n, n, n);", "mm(F, SFcl, Sk, n, n, n);"),
    "gain_wrong_U_weight": ("for (int i = 0; i < m * m; ++i) G[i] += U[i];\n\n        /* K",
                            "for (int i = 0; i < m * m; ++i) G[i] += 2.0 * U[i];\n\n        /* K"),
    "control_sign_of_Kc_term": ("uk[i] = -Kx[i] + Kvv[i] - Kcc[i];",
                                "uk[i] = -Kx[i] + Kvv[i] + Kcc[i];"),
    "eta_drops_X": ("mv(HtX, r, q, n, p);", "mtm(H, r, q, n, p, 1);"),
    "reference_off_by_one": ("at(P->r, P->sr, k), p, n, Q, q);",
                             "at(P->r, P->sr, k + 1 < P->T ? k + 1 : k), p, n, Q, q);"),
    "element_C_drops_Uinv": ("mm(L, Uinv, LUi, n, m, m);",
                             "memcpy(LUi, L, sizeof(double) * n * m);"),
    "combine_wrong_inverse_for_eta_J": ("mtm(A1, M2i, T3, n, n, n);",
                                        "mtm(A1, M1i, T3, n, n, n);"),
    "combine_drops_b2": ("for (int i = 0; i < n; ++i) b[i] += b2[i];",
                         "for (int i = 0; i < n; ++i) b[i] += 0.0 * b2[i];"),
    "combine_C_without_A2T": ("mm(T2, A2t, C, n, n, n);", "mm(T2, A2, C, n, n, n);"),
    "combine_eta_sign": ("w2[i] = eta2[i] - w2[i];", "w2[i] = eta2[i] + w2[i];"),
    "affine_operands_swapped": ("mm(F2, F1, F, n, n, n);", "mm(F1, F2, F, n, n, n);"),
    "method2_CS_order": ("mm(C, S, M, n, n, n);", "mm(S, C, M, n, n, n);"),
}


def _pins_hold(orc) -> bool:
    """A compact run of the pins; False as soon as one fails."""
    try:
        probs = [inputs.random_problem(3, 2, 2, T=6, seed=3),
                 inputs.random_problem(4, 2, 3, T=7, seed=4, pT=2)]
        for prob in probs:
            o = orc.riccati(prob)
            u, x, _ = kkt.solve_from(prob, 0, prob.x0)
            if rel_fro(o["u"], u) > 1e-10 or rel_fro(o["x"], x) > 1e-10:
                return False
            S, v, K, _ = kkt.value_function(prob, 1)
            if np.abs(o["S"][1] - S).max() > 1e-8 or np.abs(o["v"][1] - v).max() > 1e-8:
                return False
            # Lemma LQT_assoc
            s = orc.element(prob, prob.T)
            for k in range(prob.T - 1, -1, -1):
                s = orc.combine(orc.element(prob, k), s)
                if rel_fro(s[4], o["S"][k]) > 1e-10 or rel_fro(s[3], o["v"][k]) > 1e-10:
                    return False
            # Lemma lqt_fwd_init
            n = prob.n
            acc = None
            for k in range(prob.T):
                F, L, c = prob.F[k], prob.L[k], prob.c[k]
                Ft = F - L @ o["K"][k]
                ct = c + L @ o["Kv"][k] @ o["v"][k + 1] - L @ o["Kc"][k] @ c
                acc = (np.zeros((n, n)), Ft @ prob.x0 + ct) if acc is None else \
                    orc.affine_combine(acc, (Ft, ct))
                if rel_fro(acc[1], o["x"][k + 1]) > 1e-10:
                    return False
            # eq. lqt_method_2
            acc = (np.zeros((n, n)), prob.x0.copy(), np.zeros((n, n)), np.zeros(n),
                   np.zeros((n, n)))
            for k in range(prob.T + 1):
                if rel_fro(orc.method2_state(acc, o["S"][k], o["v"][k], prob.x0),
                           o["x"][k]) > 1e-9:
                    return False
                if k < prob.T:
                    acc = orc.combine(acc, orc.element(prob, k))
        # the affine operator is composition (map 1 first)
        rng = np.random.default_rng(1)
        f1 = (rng.standard_normal((3, 3)), rng.standard_normal(3))
        f2 = (rng.standard_normal((3, 3)), rng.standard_normal(3))
        F, c = orc.affine_combine(f1, f2)
        y = rng.standard_normal(3)
        if not np.allclose(F @ y + c, f2[0] @ (f1[0] @ y + f1[1]) + f2[1], rtol=1e-13, atol=1e-13):
            return False
        # associativity and brute-force minimisation over the middle state
        rng = np.random.default_rng(0)
        n = 3

        def el():
            B = rng.standard_normal((n, n))
            D = rng.standard_normal((n, n))
            return (rng.standard_normal((n, n)), rng.standard_normal(n), B @ B.T + 0.5 * np.eye(n),
                    rng.standard_normal(n), D @ D.T)

        a, b, c = el(), el(), el()
        l_ = orc.combine(orc.combine(a, b), c)
        r_ = orc.combine(a, orc.combine(b, c))
        if any(rel_fro(p, q) > 1e-12 for p, q in zip(l_, r_)):
            return False
        ab = orc.combine(a, b)

        def V(e, x, y):
            d = y - e[0] @ x - e[1]
            return 0.5 * x @ e[4] @ x - x @ e[3] + 0.5 * d @ np.linalg.solve(e[2], d)

        def brute(x, y):
            Ca, Cb = np.linalg.inv(a[2]), np.linalg.inv(b[2])
            Hz = Ca + b[4] + b[0].T @ Cb @ b[0]
            gz = Ca @ (a[0] @ x + a[1]) + b[3] + b[0].T @ Cb @ (y - b[1])
            z = np.linalg.solve(Hz, gz)
            return V(a, x, z) + V(b, z, y)

        z0 = np.zeros(n)
        for _ in range(4):
            x, y = rng.standard_normal(n), rng.standard_normal(n)
            if not math.isclose(V(ab, x, y) - V(ab, z0, z0), brute(x, y) - brute(z0, z0),
                                rel_tol=1e-10, abs_tol=1e-10):
                return False
        return True
    except (ArithmeticError, np.linalg.LinAlgError):
        return False


def test_pins_hold_for_the_real_oracle(orc):
    assert _pins_hold(orc)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    import oracle

    before, after = MUTATIONS[name]
    src = open(ORACLE_SRC).read()
    assert src.count(before) == 1, "mutation anchor must be unique: " + name
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(before, after))
    so = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", so, str(mutant),
                           "-lm"])
    assert not _pins_hold(oracle.Oracle(so)), name
