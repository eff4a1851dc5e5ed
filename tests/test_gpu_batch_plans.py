"""Batches under non-default launch plans (lqt_batch_set_tuning): the
persistent cooperative launch, the per-level launches and the automatic choice
between them, with tuned chunk lengths from short to long, all match the FP64
oracle problem by problem; the committed tuned plan is restored afterwards.  A tuned length applies only up to
the one that fills the device, so the small batch runs the capped plan and the
filled batch the tuned short chunks."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, compare, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu

SPECS = [(8, 64), (8, 300), (8, 1500), (16, 77), (16, 600), (16, 2500), (8, 4096), (16, 4096),
         (4, 900), (32, 333)]


@pytest.fixture
def restore_plan():
    from paper_2104_03186_gb300 import lqt

    yield
    lqt.lqt_batch_set_tuning([], "auto")
    lqt.apply_tuned_plans()


MODES = ["persistent", "per_level", "auto"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("table", [[], [(8, 512, 8), (8, 4096, 128), (16, 1000, 16),
                                        (16, 4096, 256)]])
def test_plans_match_oracle(mode, table, restore_plan):
    from paper_2104_03186_gb300 import lqt

    lqt.lqt_batch_set_tuning(table, mode)
    probs = [inputs.diag_tracking(n, T=T, seed=900 + i).rounded_to(np.float32)
             for i, (n, T) in enumerate(SPECS)]
    outs = lqt.solve_batched([lqt.Problem.from_inputs(p) for p in probs])
    for p, o in zip(probs, outs):
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, oracle_solve(p), FP32_TOL)


@pytest.mark.parametrize("mode", MODES)
def test_filled_batch_takes_tuned_chunks(mode, restore_plan):
    """Enough steps per size (98k at n = 8, 49k at n = 16) that chunks of 8
    and 16 steps leave no resident group idle, so the table's lengths apply."""
    from paper_2104_03186_gb300 import lqt

    lqt.lqt_batch_set_tuning([(8, 4096, 8), (16, 4096, 16)], mode)
    specs = [(8, 2048)] * 48 + [(16, 2048)] * 24
    probs = [inputs.diag_tracking(n, T=T, seed=1300 + i).rounded_to(np.float32)
             for i, (n, T) in enumerate(specs)]
    outs = lqt.solve_batched([lqt.Problem.from_inputs(p) for p in probs])
    for p, o in zip(probs, outs):
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, oracle_solve(p), FP32_TOL)


def test_auto_mode_takes_both_paths(restore_plan):
    """Under the automatic launch mode each state size of a batch takes the
    persistent launch only where its grid needs at most half of the device's
    co-resident CTAs: 64 problems of 4096 steps in 4-step chunks (65 536 chunks
    at n = 8) take the per-level launches, two problems of 300 steps at n = 16
    (128 chunks) the persistent one.  One call, checked problem by problem."""
    from paper_2104_03186_gb300 import lqt

    lqt.lqt_batch_set_tuning([(8, 4096, 4), (16, 4096, 64)], "auto")
    specs = [(8, 4096)] * 64 + [(16, 300)] * 2
    probs = [inputs.diag_tracking(n, T=T, seed=1700 + i).rounded_to(np.float32)
             for i, (n, T) in enumerate(specs)]
    outs = lqt.solve_batched([lqt.Problem.from_inputs(p) for p in probs])
    for p, o in zip(probs, outs):
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, oracle_solve(p), FP32_TOL)
