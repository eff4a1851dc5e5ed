"""lqt_solve_static: the solve for callers that cannot allocate device memory.

Some callers cannot hand the library a workspace -- a real-time control loop
that forbids device allocation once it runs, or a host framework that owns the
allocator.  lqt_solve_static gives them the same solve with its scratch space
in one fixed array inside the library.  These tests call it through the C ABI
and check its results against lqt_solve (which takes a caller workspace), on
two calls in a row so that state left in the shared array by the first call
cannot leak into the second.  This file is named to be collected last.
"""
import numpy as np
import pytest

from gpu_util import FP32_TOL, compare
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _with_workspace(lqt, P, opts):
    out = P.allocate_outputs()
    ws = lqt.workspace_for(P, opts=opts)
    lqt.lqt_solve(P, out, ws, None, opts)
    assert lqt.lqt_workspace_status(ws) == lqt.LQT_OK
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def _static(lqt, P, opts):
    out = P.allocate_outputs()
    st = lqt.lqt_solve_static(P, out, None, opts)
    assert st == lqt.LQT_OK
    return {k: v.double().cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("opts", [None, 0])
def test_static_scratch_matches_workspace_solve_twice(opts):
    import torch

    from paper_2104_03186_gb300 import lqt

    # two different problems back to back: the second must not see the first's state
    probs = [inputs.vehicle(100_003, seed=1).rounded_to(np.float32),
             inputs.random_problem(4, 2, 3, T=40_000, seed=9, pT=2).rounded_to(np.float32)]
    for prob in probs:
        P = lqt.Problem.from_inputs(prob)
        assert lqt.lqt_workspace_bytes(P, opts) <= lqt.LQT_STATIC_SCRATCH_BYTES
        ref = _with_workspace(lqt, P, opts)
        torch.cuda.synchronize()
        got = _static(lqt, P, opts)
        compare(got, ref, FP32_TOL)
    # and the same problem twice in a row
    P = lqt.Problem.from_inputs(probs[0])
    a = _static(lqt, P, opts)
    b = _static(lqt, P, opts)
    compare(b, a, FP32_TOL)


def test_static_scratch_rejects_too_large_problems():
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(inputs.vehicle(2_000_000, seed=0).rounded_to(np.float32))
    assert lqt.lqt_workspace_bytes(P) > lqt.LQT_STATIC_SCRATCH_BYTES
    out = P.allocate_outputs()
    out["x"].fill_(123.0)
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve_static(P, out)
    assert ei.value.status == lqt.LQT_ENOMEM
    assert bool((out["x"] == 123.0).all())  # nothing was launched


def test_static_scratch_reports_device_status():
    from paper_2104_03186_gb300 import lqt

    prob = inputs.vehicle(5000, seed=0).rounded_to(np.float32)
    prob.U = -prob.U
    P = lqt.Problem.from_inputs(prob)
    out = P.allocate_outputs()
    assert lqt.lqt_solve_static(P, out) == lqt.LQT_ENOTSPD
    # a good solve afterwards starts from a clean status word
    P2 = lqt.Problem.from_inputs(inputs.vehicle(5000, seed=0).rounded_to(np.float32))
    assert lqt.lqt_solve_static(P2, P2.allocate_outputs()) == lqt.LQT_OK
