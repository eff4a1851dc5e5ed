"""Batches under non-default launch plans (lqt_batch_set_tuning): the
persistent cooperative launch and the per-level launches, with tuned chunk
lengths from short to long, all match the FP64 oracle problem by problem; the
committed tuned plan is restored afterwards.  A tuned length applies only up to
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
    lqt.lqt_batch_set_tuning([], True)
    lqt.apply_tuned_plans()


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("table", [[], [(8, 512, 8), (8, 4096, 128), (16, 1000, 16),
                                        (16, 4096, 256)]])
def test_plans_match_oracle(persistent, table, restore_plan):
    from paper_2104_03186_gb300 import lqt

    lqt.lqt_batch_set_tuning(table, persistent)
    probs = [inputs.diag_tracking(n, T=T, seed=900 + i).rounded_to(np.float32)
             for i, (n, T) in enumerate(SPECS)]
    outs = lqt.solve_batched([lqt.Problem.from_inputs(p) for p in probs])
    for p, o in zip(probs, outs):
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, oracle_solve(p), FP32_TOL)


@pytest.mark.parametrize("persistent", [True, False])
def test_filled_batch_takes_tuned_chunks(persistent, restore_plan):
    """Enough steps per size (98k at n = 8, 49k at n = 16) that chunks of 8
    and 16 steps leave no resident group idle, so the table's lengths apply."""
    from paper_2104_03186_gb300 import lqt

    lqt.lqt_batch_set_tuning([(8, 4096, 8), (16, 4096, 16)], persistent)
    specs = [(8, 2048)] * 48 + [(16, 2048)] * 24
    probs = [inputs.diag_tracking(n, T=T, seed=1300 + i).rounded_to(np.float32)
             for i, (n, T) in enumerate(specs)]
    outs = lqt.solve_batched([lqt.Problem.from_inputs(p) for p in probs])
    for p, o in zip(probs, outs):
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, oracle_solve(p), FP32_TOL)
