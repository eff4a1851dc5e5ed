"""The benchmark's workloads at their own sizes against the FP64 oracle, with
the per-step check of every output:

* the precision study (n = 32, m = 16, p = 32, T = 65536, cond(X_k) = 1e6,
  U = 1e-3 I) with the default refinement (one KKT step) and with the full one
  (FP64 tree levels, one Newton step, the KKT step);
* a 512-problem slice of the ragged batch (n in {4, 8, 16}, m = n/2,
  T in U[64, 4096], time-varying F_k, L_k, X_k), every problem checked.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from gpu_util import FP32_TOL, compare, gpu_solve, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def precision_study():
    prob = inputs.precision_study(T=65536, seed=0).rounded_to(np.float32)
    return prob, oracle_solve(prob)


def test_precision_study_full_size_full_refinement(precision_study):
    from paper_2104_03186_gb300 import lqt

    prob, ref = precision_study
    errs = compare(gpu_solve(prob, refine=lqt.LQT_REFINE_FULL), ref, FP32_TOL)
    print("precision study, FULL:", dict(errs), errs.step)


def test_precision_study_full_size_default_refinement(precision_study):
    """The KKT step brings x* and u* to FP32 rounding.  S, v and K keep the
    plain FP32 scan's error, which this ill-conditioned problem amplifies (the
    sequential FP32 recursion shows the same three digits: K at 7.5e-6); FULL
    above takes them to FP32 rounding."""
    prob, ref = precision_study
    errs = compare(gpu_solve(prob), ref, FP32_TOL)
    print("precision study, ON:", dict(errs), errs.step)


def _ragged_slice(count, seed):
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray((4, 8, 16)), size=count)
    Ts = rng.integers(64, 4096 + 1, size=count)

    def one(i):
        return inputs.diag_tracking(int(ns[i]), T=int(Ts[i]),
                                    seed=int(seed) * 1_000_003 + i).rounded_to(np.float32)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(one, range(count)))


def test_ragged_batch_slice_every_problem_matches_oracle():
    from paper_2104_03186_gb300 import lqt

    probs = _ragged_slice(512, 7)
    Ps = [lqt.Problem.from_inputs(p) for p in probs]
    outs = lqt.solve_batched(Ps)
    got = [{k: v.double().cpu().numpy() for k, v in o.items()} for o in outs]
    del outs

    def check(i):
        return compare(got[i], oracle_solve(probs[i]), FP32_TOL)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        errs = list(ex.map(check, range(len(probs))))
    worst = {k: max(e[k] for e in errs) for k in errs[0]}
    worst_step = {k: max(e.step[k] for e in errs) for k in errs[0]}
    print("ragged slice, 512 problems:", worst, worst_step)
