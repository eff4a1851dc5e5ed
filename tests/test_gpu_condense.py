"""Partial condensing (Sec. V-C) through lqt_solve_condensed: the condensed
problem (blocks of B steps, stacked controls, generalised stage cost) solved by
lqt_solve_cross and expanded back to every step.  Condensing is exact, so the
oracle is the plain FP64 solution of the original problem."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(prob, B, dtype=np.float32, refine=None):
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(prob, dtype=dtype)
    out = lqt.solve_condensed(P, B, opts=refine)
    return {k: v.double().cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n,m,B", [(2, 1, 2), (3, 1, 2), (4, 1, 2), (4, 1, 4), (4, 2, 2)])
@pytest.mark.parametrize("T", [1, 7, 1000])
def test_condensed_fp32_matches_plain_oracle(n, m, B, T):
    """T = 7 leaves a shorter last block (padded)."""
    prob = inputs.random_problem(n, m, T=T, seed=10 * n + m + T).rounded_to(np.float32)
    compare(_solve(prob, B), oracle_solve(prob), FP32_TOL)


def test_condensed_fp64_matches_plain_oracle():
    for T in (5, 800):
        prob = inputs.random_problem(4, 1, T=T, seed=T)
        compare(_solve(prob, 2, dtype=np.float64), oracle_solve(prob), FP64_TOL)


def test_condensed_vehicle_and_time_invariant():
    """The vehicle workload (n = 4, m = 2, p = 2; condensed to m = 4, p = 4) and
    a time-invariant random problem with offsets."""
    prob = inputs.vehicle(4001, seed=3).rounded_to(np.float32)
    compare(_solve(prob, 2), oracle_solve(prob), FP32_TOL)
    prob = inputs.random_problem(4, 1, 3, T=999, seed=5, time_varying=False).rounded_to(np.float32)
    compare(_solve(prob, 4), oracle_solve(prob), FP32_TOL)


def test_condensed_vehicle_long_horizon():
    """The vehicle benchmark's horizon, T = 1e6, every output."""
    prob = inputs.vehicle(1_000_000, seed=0).rounded_to(np.float32)
    compare(_solve(prob, 2), oracle_solve(prob), FP32_TOL)


def test_condensed_unsupported_and_passthrough():
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(inputs.random_problem(8, 4, T=50, seed=1).rounded_to(np.float32))
    assert lqt.lqt_condensed_workspace_bytes(P, 2) == 0
    prob = inputs.random_problem(4, 2, T=300, seed=2).rounded_to(np.float32)
    compare(_solve(prob, 1), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("B", [3, 4, 8, 16])
@pytest.mark.parametrize("T", [1000, 4096, 1001])
def test_rank_reduced_condensing_vehicle(B, T):
    """Block sizes past the register kernels (B m > 4) go through the
    rank-reduced condensed problem (n controls per block, solved at (4, 4));
    T = 4096 with B | T takes the time-invariant block matrices, the others
    a padded last block."""
    prob = inputs.vehicle(T, seed=B).rounded_to(np.float32)
    compare(_solve(prob, B), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("B", [3, 8, 16])
def test_rank_reduced_condensing_time_varying(B):
    """Time-varying dynamics, costs, offsets c_k and control weights."""
    prob = inputs.random_problem(4, 2, p=2, T=777, seed=30 + B, pT=4).rounded_to(np.float32)
    compare(_solve(prob, B), oracle_solve(prob), FP32_TOL)


def test_rank_reduced_limits():
    from paper_2104_03186_gb300 import lqt

    # B p > 32: no plan
    P = lqt.Problem.from_inputs(inputs.random_problem(4, 2, p=4, T=100, seed=1).rounded_to(
        np.float32))
    assert lqt.lqt_condensed_workspace_bytes(P, 16) == 0
    assert lqt.lqt_condensed_workspace_bytes(P, 8) > 0


@pytest.mark.parametrize("B", [2, 16])
def test_condensed_refinement_restores_u(B):
    """The expansion rebuilds u from block starts and references of order one;
    the second (shifted) solve makes every term of the size of u, so all
    outputs stay near FP32 rounding at any B.  Unrefined, u carries the
    cancellation of the FP32 solve (about 1e-5 here, as for lqt_solve)."""
    from paper_2104_03186_gb300 import lqt

    prob = inputs.vehicle(100_000, seed=40 + B).rounded_to(np.float32)
    ref = oracle_solve(prob)
    errs = compare(_solve(prob, B), ref, FP32_TOL)
    assert max(errs.values()) <= 1e-6, errs
    off = compare(_solve(prob, B, refine=lqt.options(refine=lqt.LQT_REFINE_OFF)), ref, 1e-4,
                  step_tol=1e-2)
    assert errs["u"] < off["u"], (errs, off)


def test_condensed_refinement_with_offsets_and_terminal_reference():
    """The shifted data cover c_k, r_k and r_T; time-varying model, B = 8
    (rank-reduced) and B = 2 (register kernels)."""
    prob = inputs.random_problem(4, 2, p=2, T=1500, seed=77, pT=4).rounded_to(np.float32)
    ref = oracle_solve(prob)
    for B in (2, 8):
        compare(_solve(prob, B), ref, FP32_TOL)


@pytest.mark.parametrize("B", [2, 8])
def test_condensed_reports_indefinite_U(B):
    """A negative control weight: the failure recorded before the condensed
    solve (the reduction's factorisation at B = 8) or by it (B = 2) reaches
    the workspace status through both solves of the refinement."""
    from paper_2104_03186_gb300 import lqt

    prob = inputs.vehicle(400, seed=1).rounded_to(np.float32)
    prob.U = -prob.U
    with pytest.raises(lqt.LQTError) as e:
        _solve(prob, B)
    assert e.value.status == lqt.LQT_ENOTSPD
