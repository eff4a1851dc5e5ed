"""Single-tile solves (k_solo): a problem whose steps fit one tile with at
most lqt_set_single_tile_chunk steps per thread runs each pass as one launch
of one CTA, the in-tile trees kept in shared memory.  Parity against the FP64
oracle on both sides of the threshold, with single-tile solves on and off,
FP32 and FP64, refined and not; the plan and the profile name the one kernel."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare, gpu_solve, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chunk", [0, 2, 4])
@pytest.mark.parametrize("T", [1, 2, 31, 511, 512, 513, 1000, 1024, 1025, 2048])
def test_vehicle_fp32_single_tile_on_and_off(T, chunk, single_tile):
    single_tile(chunk)
    prob = inputs.vehicle(T, seed=T % 5).rounded_to(np.float32)
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("nmp", [(1, 1, 1), (2, 1, 2), (3, 2, 2), (4, 4, 3)],
                         ids=lambda v: "n%d_m%d_p%d" % v)
@pytest.mark.parametrize("refine", [0, 1])
def test_random_time_varying_single_tile(nmp, refine, single_tile):
    n, m, p = nmp
    prob = inputs.random_problem(n, m, p, T=777, seed=40 + n, pT=n).rounded_to(np.float32)
    compare(gpu_solve(prob, refine=refine), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("T", [5, 256, 512])
@pytest.mark.parametrize("refine", [0, 1])
def test_fp64_single_tile(T, refine, single_tile):
    """FP64 tiles are 256 threads: T <= 512 is one tile at two steps a thread."""
    prob = inputs.random_problem(4, 2, 2, T=T, seed=T)
    compare(gpu_solve(prob, dtype=np.float64, refine=refine), oracle_solve(prob), FP64_TOL)


def test_plan_and_profile_name_the_single_kernel(single_tile):
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(inputs.vehicle(1000).rounded_to(np.float32))
    plan = lqt.lqt_plan(P, 1)
    assert (plan["tiles"], plan["kernels"], plan["chunk_steps"]) == (1, 2, 2)
    assert lqt.lqt_plan(P, 0)["kernels"] == 1
    lqt.lqt_profile_enable(True)
    try:
        lqt.solve(P, opts=1)
        prof = lqt.lqt_profile_read()
    finally:
        lqt.lqt_profile_enable(False)
    assert [n for n, _ in prof] == ["solo", "solo.refine"]
    single_tile(0)
    assert lqt.lqt_plan(P, 1)["kernels"] == 10


def test_single_tile_refinement_keeps_S_v_K_bit_for_bit(single_tile):
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(inputs.vehicle(900, seed=3).rounded_to(np.float32))
    a = lqt.solve(P, opts=0)
    b = lqt.solve(P, opts=1)
    for k in ("S", "v", "K"):
        assert bool((a[k] == b[k]).all()), k


def test_single_tile_reports_indefinite_U(single_tile):
    from paper_2104_03186_gb300 import lqt

    prob = inputs.vehicle(600, seed=0).rounded_to(np.float32)
    prob.U = -prob.U
    with pytest.raises(lqt.LQTError) as ei:
        gpu_solve(prob)
    assert ei.value.status == lqt.LQT_ENOTSPD
