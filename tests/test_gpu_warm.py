"""Warm solves (lqt_solve_warm): a problem over steps [s, T) of an earlier
solve's model, with its own references, offsets and initial state, solved
from the earlier solve's S and K.  Each result matches a full solve of the
same problem and the FP64 oracle, at every compiled size, in FP32 and FP64,
alone and in mixed batches, including the empty and one-step horizons."""
import dataclasses

import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _shifted(prob, s, seed):
    """Steps [s, T) of prob with a fresh reference (and offsets, if any) and x_0."""
    rng = np.random.default_rng(seed)
    T = prob.T - s
    cut = {}
    for f in ("F", "c", "L", "U", "H", "X"):
        a = getattr(prob, f)
        cut[f] = None if a is None else (a if a.shape[0] == 1 else np.ascontiguousarray(a[s:]))
    r = rng.standard_normal((T, prob.p))
    if prob.c is not None:
        cut["c"] = 0.1 * rng.standard_normal((T, prob.n))
    return dataclasses.replace(prob, r=r, rT=rng.standard_normal(prob.pT),
                               x0=rng.standard_normal(prob.n), T=T, **cut)


def _warm_pair(prob, s, dtype, seed):
    """(warm problem rounded to dtype, known S and K from a full solve of prob)."""
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(prob, dtype=dtype)
    prior = lqt.solve(P, opts=lqt.LQT_REFINE_OFF)
    warm = _shifted(prob, s, seed).rounded_to(dtype)
    known = {"S": prior["S"][s:].contiguous(), "K": prior["K"][s:].contiguous()}
    return warm, known


def _host(out):
    return {k: v.double().cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_warm_matches_full_solve_and_oracle_fp32(n):
    from paper_2104_03186_gb300 import lqt

    prob = inputs.diag_tracking(n, T=1500, seed=40 + n).rounded_to(np.float32)
    warm, known = _warm_pair(prob, 377, np.float32, seed=n)
    P = lqt.Problem.from_inputs(warm)
    got = _host(lqt.solve_warm([P], [known])[0])
    cold = _host(lqt.solve(P, opts=lqt.LQT_REFINE_OFF))
    compare(got, cold, FP32_TOL)
    compare(got, oracle_solve(warm), FP32_TOL)


@pytest.mark.parametrize("n", [4, 8, 32])
def test_warm_fp64(n):
    from paper_2104_03186_gb300 import lqt

    prob = inputs.diag_tracking(n, T=900, seed=70 + n)
    warm, known = _warm_pair(prob, 123, np.float64, seed=n + 1)
    P = lqt.Problem.from_inputs(warm, dtype=np.float64)
    got = _host(lqt.solve_warm([P], [known])[0])
    compare(got, oracle_solve(warm), FP64_TOL)


def test_warm_with_offsets_and_general_costs():
    """c_k != 0, a rectangular H_k with a full X_k, time-varying U_k."""
    from paper_2104_03186_gb300 import lqt

    prob = inputs.random_problem(8, 4, p=5, T=2000, seed=9, pT=8).rounded_to(np.float32)
    assert prob.c is not None
    warm, known = _warm_pair(prob, 601, np.float32, seed=3)
    P = lqt.Problem.from_inputs(warm)
    got = _host(lqt.solve_warm([P], [known])[0])
    compare(got, oracle_solve(warm), FP32_TOL)


def test_warm_batch_mixed_sizes_and_edges():
    """One call over several sizes, long and short horizons, T = 1 and T = 0."""
    from paper_2104_03186_gb300 import lqt

    specs = [(4, 3000, 1000), (16, 800, 799), (8, 500, 17), (32, 700, 100), (4, 64, 64),
             (8, 2048, 1)]
    probs, outs, refs = [], [], []
    for i, (n, T, s) in enumerate(specs):
        prob = inputs.diag_tracking(n, T=T, seed=500 + i).rounded_to(np.float32)
        warm, known = _warm_pair(prob, s, np.float32, seed=600 + i)
        P = lqt.Problem.from_inputs(warm)
        o = P.allocate_outputs()
        o["S"], o["K"] = known["S"], known["K"]
        probs.append(P)
        outs.append(o)
        refs.append(oracle_solve(warm))
    import torch

    ws = torch.empty(lqt.lqt_warm_workspace_bytes(probs, outs), dtype=torch.uint8,
                     device="cuda")
    lqt.lqt_solve_warm(probs, outs, ws)
    assert lqt.lqt_workspace_status(ws) == lqt.LQT_OK
    for o, ref, (n, T, s) in zip(outs, refs, specs):
        names = ("S", "v", "K", "x", "u") if T - s > 0 else ("S", "v", "x")
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, ref, FP32_TOL, names=names)


def test_warm_rejects_bad_items():
    import torch

    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(inputs.random_problem(5, 2, T=10, seed=0).rounded_to(np.float32))
    o = P.allocate_outputs()
    assert lqt.lqt_warm_workspace_bytes([P], [o]) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve_warm([P], [o], ws)
    assert ei.value.status == lqt.LQT_EUNSUPPORTED
