"""Generalised stage cost (Sec. IV-D, eq. generalised_cost) through
lqt_solve_cross: the transform kernel, the solve of the transformed problem and
the control post-transform, against the FP64 oracle (oracle/cross.py) at the
small sizes (thread-per-step path) and the lane-group sizes (chunked
pipeline), FP32 and FP64."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(prob, ct, dtype=np.float32, refine=None, method=0):
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(prob, dtype=dtype)
    C = None if ct is None else lqt.Cross.from_inputs(ct, dtype=dtype)
    opts = refine
    if method:
        opts = lqt.options(lqt.LQT_REFINE_AUTO if refine is None else refine, method)
    out = lqt.solve_cross(P, C, opts=opts)
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def _oracle(prob, ct):
    from oracle import cross

    return cross.riccati_cross(prob, None if ct is None else ct.M, None if ct is None else ct.s)


def _case(n, m, T, seed, dtype=np.float32, scale=0.5, ct_kw=None, **kw):
    prob = inputs.random_problem(n, m, T=T, seed=seed, **kw)
    ct = inputs.cross_terms(prob, seed=seed + 1, scale=scale, **(ct_kw or {}))
    if dtype == np.float32:
        prob, ct = prob.rounded_to(np.float32), ct.rounded_to(np.float32)
    return prob, ct


@pytest.mark.parametrize("n,m", [(2, 1), (3, 2), (4, 2), (4, 4)])
@pytest.mark.parametrize("T", [1, 7, 1000])
@pytest.mark.parametrize("refine", [0, 1])
def test_cross_small_fp32(n, m, T, refine):
    prob, ct = _case(n, m, T, seed=100 * n + T)
    compare(_solve(prob, ct, refine=refine), _oracle(prob, ct), FP32_TOL)


@pytest.mark.parametrize("n,m", [(8, 4), (16, 8), (32, 16)])
@pytest.mark.parametrize("T", [1, 333, 2000])
def test_cross_lanes_fp32(n, m, T):
    prob, ct = _case(n, m, T, seed=7 * n + T)
    compare(_solve(prob, ct, refine=1), _oracle(prob, ct), FP32_TOL)


@pytest.mark.parametrize("n,m", [(2, 1), (4, 2), (8, 4), (16, 8), (32, 16)])
def test_cross_fp64(n, m):
    prob, ct = _case(n, m, 600, seed=300 + n, dtype=np.float64, scale=0.8)
    compare(_solve(prob, ct, dtype=np.float64), _oracle(prob, ct), FP64_TOL)


@pytest.mark.parametrize("n,m,kw", [
    (4, 2, dict(p=2, pT=2)),            # the vehicle-sized shape, p < n
    (4, 2, dict(p=8)),                  # p = 2n
    (8, 4, dict(p=3, pT=1)),
    (16, 8, dict(p=32, pT=32)),         # p = 2n at a lane size
])
def test_cross_shapes(n, m, kw):
    prob, ct = _case(n, m, 500, seed=400 + n, **kw)
    compare(_solve(prob, ct), _oracle(prob, ct), FP32_TOL)


@pytest.mark.parametrize("n,m", [(4, 2), (16, 8)])
def test_cross_time_invariant(n, m):
    """Every matrix and M, s with step stride 0: the transform writes one row
    of F~, c~, X~ and the post terms.  Open-loop spectral radius up to 1.05
    held for all steps: S, v, K need the Newton step of the FULL refinement
    at FP32 (the plain problem behaves the same)."""
    from paper_2104_03186_gb300 import lqt

    prob, ct = _case(n, m, 700, seed=500 + n, time_varying=False,
                     ct_kw=dict(time_varying=False))
    assert ct.M.shape[0] == 1 and ct.s.shape[0] == 1
    compare(_solve(prob, ct, refine=lqt.LQT_REFINE_FULL), _oracle(prob, ct), FP32_TOL)
    prob64, ct64 = _case(n, m, 700, seed=510 + n, dtype=np.float64, time_varying=False,
                         ct_kw=dict(time_varying=False))
    compare(_solve(prob64, ct64, dtype=np.float64), _oracle(prob64, ct64), FP64_TOL)


@pytest.mark.parametrize("n,m", [(4, 2), (8, 4)])
def test_cross_partial_terms(n, m):
    """Only M (s = 0), only s (M = 0, F and X passed through), and neither (the
    plain problem)."""
    prob, ct = _case(n, m, 400, seed=600 + n)
    for c in (inputs.CrossTerms(M=ct.M, s=None), inputs.CrossTerms(M=None, s=ct.s), None):
        compare(_solve(prob, c), _oracle(prob, c), FP32_TOL)


def test_cross_method2_and_full_refinement():
    """The options apply to the transformed solve: Method 2 and FULL refinement."""
    prob, ct = _case(16, 8, 900, seed=700)
    ref = _oracle(prob, ct)
    from paper_2104_03186_gb300 import lqt

    compare(_solve(prob, ct, refine=1, method=2), ref, FP32_TOL)
    compare(_solve(prob, ct, refine=lqt.LQT_REFINE_FULL), ref, FP32_TOL)


def test_cross_vehicle_long_horizon_sampled():
    """The vehicle workload with cross terms at T = 1e6 (the launch
    configuration of the vehicle benchmark): every output against the oracle."""
    prob = inputs.vehicle(1_000_000, seed=0)
    ct = inputs.cross_terms(prob, seed=1, scale=0.5)
    prob, ct = prob.rounded_to(np.float32), ct.rounded_to(np.float32)
    compare(_solve(prob, ct), _oracle(prob, ct), FP32_TOL)


def test_cross_zero_horizon():
    prob, ct = _case(4, 2, 3, seed=800)
    prob.T = 0
    for f in ("F", "c", "L", "U", "H", "r", "X"):
        a = getattr(prob, f)
        if a is not None and a.shape[0] > 1:
            setattr(prob, f, a[:0])
    ct = inputs.CrossTerms(M=ct.M[:0], s=ct.s[:0])
    compare(_solve(prob, ct), _oracle(prob, ct), FP32_TOL, names=("S", "v", "x"))


def test_cross_reports_indefinite_U():
    """A U_k with a negative eigenvalue: the transform's Cholesky check reports
    LQT_ENOTSPD through the workspace status."""
    from paper_2104_03186_gb300 import lqt

    prob, ct = _case(4, 2, 50, seed=900)
    prob.U = prob.U.copy()
    prob.U[10] = -prob.U[10]
    P = lqt.Problem.from_inputs(prob)
    C = lqt.Cross.from_inputs(ct)
    with pytest.raises(lqt.LQTError) as e:
        lqt.solve_cross(P, C)
    assert e.value.status == lqt.LQT_ENOTSPD


@pytest.mark.parametrize("n,m", [(4, 2), (2, 1), (8, 4)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_cross_invariant_matrices_varying_vectors(n, m, dtype):
    """Time-invariant F, L, U, H, X and M with r_k, c_k and s_k varying: the
    transform's matrices come from step 0 alone and a per-step kernel forms
    g_k = W r_k + s_k and c~_k = c_k + L g_k.  F is scaled to spectral radius
    0.98: a fixed F with an unstable mode (1.04 here) grows by 1.04^T over
    the scan's spans, which no FP32 scan resolves to the tolerance."""
    prob = inputs.random_problem(n, m, T=1500, seed=41 + n, time_varying=False)
    prob.F = prob.F * (0.98 / np.abs(np.linalg.eigvals(prob.F[0])).max())
    ct = inputs.cross_terms(prob, seed=42, scale=0.5, time_varying=False)
    rng = np.random.default_rng(43)
    ct = inputs.CrossTerms(M=ct.M, s=rng.standard_normal((prob.T, m)))
    prob.c = rng.normal(0.0, 0.1, (prob.T, n))
    tol = FP64_TOL
    if dtype == np.float32:
        prob, ct, tol = prob.rounded_to(np.float32), ct.rounded_to(np.float32), FP32_TOL
    compare(_solve(prob, ct, dtype=dtype), _oracle(prob, ct), tol)
