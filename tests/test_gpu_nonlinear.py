"""Iterated nonlinear LQT (Sec. IV-D; the unicycle of Sec. VI-E) through
lqt_solve_nonlinear against the FP64 oracle (oracle/nonlinear.py) running the
same passes from the same first nominal."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu(prob, iterations=10, dtype=np.float32, sequential=False, opts=None, x_init=None,
         u_init=None):
    import torch

    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(prob, dtype=dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    xi = None if x_init is None else torch.from_numpy(x_init).to(tdt).cuda()
    ui = None if u_init is None else torch.from_numpy(u_init).to(tdt).cuda()
    out = lqt.solve_nonlinear(P, iterations=iterations, dt=0.1, sequential=sequential, opts=opts,
                              x_init=xi, u_init=ui)
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def _oracle(prob, iterations=10, x_init=None, u_init=None):
    from oracle import nonlinear as nl

    return nl.iterated_lqt(nl.Unicycle(0.1), prob, iterations, x_init, u_init)


@pytest.mark.parametrize("T", [1, 50, 2000])
def test_nonlinear_fp32_matches_oracle(T):
    prob = inputs.unicycle_track(T, seed=T).rounded_to(np.float32)
    compare(_gpu(prob), _oracle(prob), FP32_TOL)


@pytest.mark.parametrize("T", [50, 2000])
def test_nonlinear_fp64_matches_oracle(T):
    prob = inputs.unicycle_track(T, seed=T + 1)
    compare(_gpu(prob, dtype=np.float64), _oracle(prob), FP64_TOL)


def test_nonlinear_sequential_and_pass_counts():
    """The sequential recursion per pass, and 1 and 3 passes (before convergence:
    every pass must match the oracle's pass)."""
    prob = inputs.unicycle_track(600, seed=5).rounded_to(np.float32)
    compare(_gpu(prob, sequential=True), _oracle(prob), FP32_TOL)
    prob64 = inputs.unicycle_track(600, seed=6)
    for it in (1, 3):
        compare(_gpu(prob64, iterations=it, dtype=np.float64), _oracle(prob64, it), FP64_TOL)


def test_nonlinear_given_first_nominal():
    """x_init / u_init: 7 passes from the oracle's third nominal equal 10 passes
    from the default start."""
    from oracle import nonlinear as nl

    prob = inputs.unicycle_track(800, seed=7)
    o3 = nl.iterated_lqt(nl.Unicycle(0.1), prob, 3)
    ref = _oracle(prob, 10)
    compare(_gpu(prob, iterations=7, dtype=np.float64, x_init=o3["x"], u_init=o3["u"]), ref,
            FP64_TOL)


def test_nonlinear_method2_and_full_refinement():
    from paper_2104_03186_gb300 import lqt

    prob = inputs.unicycle_track(1500, seed=8).rounded_to(np.float32)
    ref = _oracle(prob)
    compare(_gpu(prob, opts=lqt.options(lqt.LQT_REFINE_ON, lqt.LQT_METHOD_2)), ref, FP32_TOL)
    compare(_gpu(prob, opts=lqt.LQT_REFINE_FULL), ref, FP32_TOL)


def test_nonlinear_long_track():
    """T = 1e5 (about 280 laps, unwrapped heading near 1760 rad), the benchmark's
    workload, FP32 with refinement: every output against the oracle."""
    prob = inputs.unicycle_track(100_000, seed=0).rounded_to(np.float32)
    compare(_gpu(prob), _oracle(prob), FP32_TOL)
