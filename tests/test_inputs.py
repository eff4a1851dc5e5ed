"""The seeded input generators against the workload recipes they implement
(no GPU): the vehicle model of Sec. VI-A, the random-stable dynamics of the
ragged batch and the serving pool, and the ill-conditioned precision study.
Each check is a property the recipe states, computed independently of the
generator (spectra, singular values, exact matrices)."""
import math

import numpy as np
import pytest

from paper_2104_03186_gb300 import inputs


def test_vehicle_model_is_the_printed_one():
    prob = inputs.vehicle(500, seed=1)
    dt = 0.1
    I2, Z2 = np.eye(2), np.zeros((2, 2))
    assert np.array_equal(prob.F[0], np.block([[I2, dt * I2], [Z2, I2]]))
    assert np.allclose(prob.L[0], np.vstack([0.5 * dt * dt * I2, dt * I2]), rtol=0, atol=1e-15)
    H = np.hstack([I2, Z2])
    assert np.array_equal(prob.H[0], H) and np.array_equal(prob.HT, H)
    assert np.array_equal(prob.X[0], I2) and np.array_equal(prob.U[0], 0.1 * I2)
    assert np.array_equal(prob.XT, 100.0 * I2)
    assert prob.c is None and prob.T == 500
    # time-invariant matrices carry a leading axis of 1; r is per step
    assert prob.F.shape == (1, 4, 4) and prob.r.shape == (500, 2) and prob.rT.shape == (2,)
    # the reference is the sinusoid plus N(0, 0.01^2) noise
    k = np.arange(501)
    clean = np.stack([np.sin(0.01 * k), np.cos(0.013 * k)], axis=1)
    noise = np.vstack([prob.r, prob.rT[None]]) - clean
    assert abs(noise.std() - 0.01) < 0.001 and abs(noise.mean()) < 0.002


def test_vehicle_is_reproducible_per_seed():
    a, b, c = inputs.vehicle(64, seed=3), inputs.vehicle(64, seed=3), inputs.vehicle(64, seed=4)
    assert np.array_equal(a.r, b.r) and np.array_equal(a.x0, b.x0)
    assert not np.array_equal(a.r, c.r)


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_diag_tracking_recipe(n):
    prob = inputs.diag_tracking(n, T=300, seed=n)
    m = n // 2
    rho = np.abs(np.linalg.eigvals(prob.F)).max(axis=-1)
    assert np.all(rho <= 1.05 * (1 + 1e-12))
    # F_k = I + 0.05 N(0, 1) before any rescaling: the off-diagonal spread
    off = prob.F[:, ~np.eye(n, dtype=bool)]
    assert 0.03 < off.std() < 0.06
    assert prob.L.shape == (300, n, m) and abs(prob.L.std() * math.sqrt(n) - 1.0) < 0.1
    d = np.diagonal(prob.X, axis1=1, axis2=2)
    assert np.array_equal(prob.X, d[:, :, None] * np.eye(n)[None])
    assert d.min() >= 0.5 and d.max() <= 2.0
    assert np.array_equal(prob.U[0], 0.1 * np.eye(m)) and np.array_equal(prob.H[0], np.eye(n))
    assert prob.c is None


def test_ragged_batch_recipe():
    batch = inputs.ragged_batch(count=150, seed=2)
    ns = np.array([p.n for p in batch])
    Ts = np.array([p.T for p in batch])
    assert set(ns.tolist()) == {4, 8, 16}
    assert Ts.min() >= 64 and Ts.max() <= 4096
    assert all(p.m == p.n // 2 for p in batch)
    for n in (4, 8, 16):  # a fixed draw of 150: loose bounds
        assert abs((ns == n).mean() - 1 / 3) < 0.12


def test_precision_study_recipe():
    n, m, T = 32, 16, 24
    prob = inputs.precision_study(T=T, seed=5)
    # cond(X_k) = 1e6 exactly, eigenvalues in [1e-6, 1], X_k symmetric
    for X in list(prob.X) + [prob.XT]:
        assert np.array_equal(X, X.T)
        lam = np.linalg.eigvalsh(X)
        assert lam.min() > 0
        assert abs(lam.max() - 1.0) < 1e-9 and abs(lam.min() / 1e-6 - 1.0) < 1e-6
    # F_k = 0.99 Q_k + a rank-2 perturbation: at least n - 4 singular values
    # are exactly 0.99 (those of directions the perturbation does not touch)
    for F in prob.F:
        s = np.linalg.svd(F, compute_uv=False)
        assert np.sum(np.abs(s - 0.99) < 1e-12) >= n - 4
    assert prob.L.shape == (T, n, m)
    assert np.array_equal(prob.U[0], 1e-3 * np.eye(m)) and np.array_equal(prob.H[0], np.eye(n))
