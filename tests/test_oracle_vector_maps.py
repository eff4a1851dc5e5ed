"""The linear maps behind the replayed top-level scan, checked on the CPU
against the oracle's operator (eq. lqt_comb), with no CUDA involved.

The second pass of a refined n <= 4 solve has the same matrices (A, C, J of
every element, S of every value) as the first and other vectors.  Its top
scan then evaluates only the vector parts, from maps the first pass recorded:

* combine e1 (x) e2, with M = I + C1 J2 and X1 = M^{-1} A1:
      b   = b2 + G1 b1 + G2 eta2,      G1 = A2 M^{-1},  G2 = A2 M^{-1} C1
      eta = eta1 + H1 eta2 + H2 b1,    H1 = X1^T,       H2 = -(J2 X1)^T
* value (S, v) through element P (the operator with the element (0, 0, 0, v, S)
  on the right, as in the proof of Lemma LQT_assoc), with X1 = (I + C_P S)^{-1} A_P:
      v' = eta_P + V1 v + V2 b_P,      V1 = X1^T,       V2 = -(S X1)^T

The maps are built here from the matrices alone and applied to fresh vectors;
the oracle combines the elements with those vectors in full.
"""
import numpy as np
import pytest

from conftest import rel_fro


def _psd(rng, n, k=None):
    B = rng.standard_normal((n, k or n))
    return B @ B.T / max(1, k or n)


def _matrices(rng, n):
    return rng.standard_normal((n, n)), _psd(rng, n), _psd(rng, n)  # A, C, J


def _combine_maps(A1, C1, A2, J2):
    n = A1.shape[0]
    Minv = np.linalg.inv(np.eye(n) + C1 @ J2)
    X1 = Minv @ A1
    return A2 @ Minv, A2 @ Minv @ C1, X1.T, -(J2 @ X1).T


def _apply_maps(A_P, C_P, S):
    n = A_P.shape[0]
    X1 = np.linalg.solve(np.eye(n) + C_P @ S, A_P)
    return X1.T, -(S @ X1).T


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_combine_vectors_follow_the_recorded_maps(orc, n):
    rng = np.random.default_rng(500 + n)
    A1, C1, J1 = _matrices(rng, n)
    A2, C2, J2 = _matrices(rng, n)
    G1, G2, H1, H2 = _combine_maps(A1, C1, A2, J2)
    for _ in range(3):  # vectors of "another pass", same matrices
        b1, h1, b2, h2 = (rng.standard_normal(n) for _ in range(4))
        A, b, C, eta, J = orc.combine((A1, b1, C1, h1, J1), (A2, b2, C2, h2, J2))
        assert rel_fro(b, b2 + G1 @ b1 + G2 @ h2) < 1e-12
        assert rel_fro(eta, h1 + H1 @ h2 + H2 @ b1) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_value_apply_vector_follows_the_recorded_maps(orc, n):
    rng = np.random.default_rng(600 + n)
    A_P, C_P, J_P = _matrices(rng, n)
    S = _psd(rng, n)
    V1, V2 = _apply_maps(A_P, C_P, S)
    zero = np.zeros((n, n))
    for _ in range(3):
        b_P, eta_P, v = (rng.standard_normal(n) for _ in range(3))
        _, _, _, v_new, S_new = orc.combine((A_P, b_P, C_P, eta_P, J_P),
                                            (zero, np.zeros(n), zero, v, S))
        assert rel_fro(v_new, eta_P + V1 @ v + V2 @ b_P) < 1e-12
        # the matrix part does not see the vectors: the next value's S is the
        # same for every pass
        _, _, _, _, S_other = orc.combine((A_P, -b_P, C_P, 2 * eta_P, J_P),
                                          (zero, np.zeros(n), zero, -v, S))
        assert rel_fro(S_other, S_new) < 1e-14


def test_maps_catch_a_wrong_sign_or_transpose(orc):
    """A plausible slip in the recorded maps (a dropped minus in H2, or G2
    without C1) fails the comparison."""
    rng = np.random.default_rng(7)
    n = 3
    A1, C1, J1 = _matrices(rng, n)
    A2, C2, J2 = _matrices(rng, n)
    G1, G2, H1, H2 = _combine_maps(A1, C1, A2, J2)
    b1, h1, b2, h2 = (rng.standard_normal(n) for _ in range(4))
    _, b, _, eta, _ = orc.combine((A1, b1, C1, h1, J1), (A2, b2, C2, h2, J2))
    assert rel_fro(eta, h1 + H1 @ h2 - H2 @ b1) > 1e-3
    assert rel_fro(b, b2 + G1 @ b1 + G1 @ h2) > 1e-3
