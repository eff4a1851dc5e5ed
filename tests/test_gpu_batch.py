"""Ragged batches through lqt_solve_batched (one persistent launch per (n, m)):
every problem of a mixed batch against the FP64 oracle, batched results
against solo solves, and argument checks."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, compare, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batch(specs):
    probs = []
    for i, (n, T, kind) in enumerate(specs):
        if kind == "diag":
            pr = inputs.diag_tracking(n, T=T, seed=100 + i)
        else:
            pr = inputs.random_problem(n, n // 2, p=n if kind == "square" else max(1, n // 2),
                                       T=T, seed=200 + i, pT=n)
        probs.append(pr.rounded_to(np.float32))
    return probs


SPECS = [(4, 1, "diag"), (8, 2, "square"), (16, 3, "diag"), (4, 64, "square"),
         (8, 100, "diag"), (16, 257, "square"), (4, 1000, "diag"), (8, 513, "half"),
         (16, 1000, "diag"), (4, 4096, "square"), (8, 4096, "diag"), (16, 2048, "half"),
         (4, 7, "half"), (16, 64, "diag")]


def test_mixed_batch_matches_oracle():
    from paper_2104_03186_gb300 import lqt

    probs = _batch(SPECS)
    Ps = [lqt.Problem.from_inputs(p) for p in probs]
    outs = lqt.solve_batched(Ps)
    for p, out, spec in zip(probs, outs, SPECS):
        g = {k: v.double().cpu().numpy() for k, v in out.items()}
        compare(g, oracle_solve(p), FP32_TOL)


def test_batched_equals_solo_within_tolerance():
    from paper_2104_03186_gb300 import lqt

    probs = _batch([(4, 3000, "diag"), (4, 777, "square"), (4, 1, "half")])
    Ps = [lqt.Problem.from_inputs(p) for p in probs]
    outs = lqt.solve_batched(Ps)
    for P, out in zip(Ps, outs):
        solo = lqt.solve(P, opts=0)
        compare({k: v.double().cpu().numpy() for k, v in out.items()},
                {k: v.double().cpu().numpy() for k, v in solo.items()}, FP32_TOL)


def test_zero_horizon_in_batch():
    from paper_2104_03186_gb300 import lqt

    prob = inputs.diag_tracking(8, T=5, seed=1).rounded_to(np.float32)
    prob.T = 0
    for f in ("F", "L", "X", "r"):
        setattr(prob, f, getattr(prob, f)[:0])
    P = lqt.Problem.from_inputs(prob)
    out = lqt.solve_batched([P])[0]
    o = oracle_solve(prob)
    compare({k: out[k].double().cpu().numpy() for k in ("S", "v", "x")},
            {k: o[k] for k in ("S", "v", "x")}, FP32_TOL, names=("S", "v", "x"))


def test_batch_rejects_unsupported_items():
    import torch

    from paper_2104_03186_gb300 import lqt

    good = lqt.Problem.from_inputs(inputs.diag_tracking(4, T=10, seed=0).rounded_to(np.float32))
    bad = lqt.Problem.from_inputs(inputs.random_problem(5, 2, T=10, seed=0).rounded_to(np.float32))
    outs = [good.allocate_outputs(), bad.allocate_outputs()]
    assert lqt.lqt_batch_workspace_bytes([good, bad], outs) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve_batched([good, bad], outs, ws)
    assert ei.value.status == lqt.LQT_EUNSUPPORTED
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve_batched([good], [good.allocate_outputs()], small)
    assert ei.value.status in (lqt.LQT_ENOMEM, lqt.LQT_EINVAL)
