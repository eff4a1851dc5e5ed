"""The bounded device waits: a wait that runs out records LQT_ETIMEOUT in the
workspace status word and the kernel carries on; the next solve on the same
workspace clears the word and returns LQT_OK.  The wait is made to run out by
the diagnostic option wait_probe_polls (a barrier that nothing completes), so
no copy is ever left in flight and nothing faults or hangs."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, compare, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("refine", [0, 1])
def test_wait_that_runs_out_flags_timeout_then_next_solve_is_ok(refine):
    import torch

    from paper_2104_03186_gb300 import lqt

    prob = inputs.vehicle(5000, seed=3).rounded_to(np.float32)
    ref = oracle_solve(prob)
    P = lqt.Problem.from_inputs(prob)
    out = P.allocate_outputs()
    ws = lqt.workspace_for(P, opts=refine)
    stream = torch.cuda.current_stream()
    probe = lqt.options(refine, wait_probe_polls=256)
    lqt.lqt_solve(P, out, ws, stream, probe)
    assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_ETIMEOUT
    # the kernel carried on after the wait ran out: the real copies had landed
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    tol = FP32_TOL if refine else 1e-4  # plain FP32: u* cancels (see the parity tests)
    compare(got, ref, tol, names=("S", "v", "K", "x"))
    # the next solve clears the word
    for v in out.values():
        v.zero_()
    lqt.lqt_solve(P, out, ws, stream, refine)
    assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_OK
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    compare(got, ref, tol, names=("S", "v", "K", "x"))


def test_wait_probe_argument_checks():
    import torch

    from paper_2104_03186_gb300 import lqt

    small = lqt.Problem.from_inputs(inputs.vehicle(64, seed=0).rounded_to(np.float32))
    ws = lqt.workspace_for(small)
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve(small, small.allocate_outputs(), ws, None, lqt.options(1, 0, -1))
    assert ei.value.status == lqt.LQT_EINVAL
    # the lane-group sizes have no bounded waits to probe
    big = lqt.Problem.from_inputs(
        inputs.diag_tracking(8, T=64, seed=0).rounded_to(np.float32))
    wsb = torch.empty(lqt.lqt_workspace_bytes(big, None), dtype=torch.uint8, device="cuda")
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve(big, big.allocate_outputs(), wsb, None, lqt.options(1, 0, 100))
    assert ei.value.status == lqt.LQT_EUNSUPPORTED
