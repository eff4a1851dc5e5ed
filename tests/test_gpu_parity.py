"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  FP32 outputs must be within 1e-5 relative Frobenius error of
the oracle per output (S, v, K, x*, u*), FP64 outputs within 1e-11.

Sizes span several chunks and tiles with ragged tails (the launch plan puts
one thread per chunk and 512 chunks per tile in FP32), up to the full
benchmark workload (vehicle model, T = 10^6)."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare, gpu_solve, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _f32(prob):
    return prob.rounded_to(np.float32)


@pytest.mark.parametrize("T", [1, 2, 3, 17, 511, 512, 513, 1000, 4097, 77823, 77825, 100003])
def test_vehicle_fp32(T):
    prob = _f32(inputs.vehicle(T, seed=T % 7))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("seed", range(5))
def test_vehicle_T1000_seeds(seed):
    prob = _f32(inputs.vehicle(1000, seed=seed))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


def test_vehicle_full_size_T1e6():
    """The benchmark workload at full size, every output compared."""
    prob = _f32(inputs.vehicle(1_000_000, seed=0))
    errs = compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)
    print("T=1e6 errors", errs)


@pytest.mark.parametrize("T", [1000, 100_000])
def test_paper_tracking_costs_fp32(T):
    """Sec. VI-A cost set-up: X_k = c_k I with c_k in {100, 1e-6}, H_T = X_T = I_4."""
    prob = _f32(inputs.paper_tracking(T, seed=1))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


RANDOM = [(1, 1, 1, 1), (2, 1, 2, 1), (2, 2, 1, 2), (3, 1, 2, 3), (3, 2, 3, 3), (4, 1, 4, 4),
          (4, 2, 3, 2), (4, 4, 4, 4)]


@pytest.mark.parametrize("T", [7, 1000, 20011])
@pytest.mark.parametrize("nmpq", RANDOM, ids=lambda v: "n%d_m%d_p%d_pT%d" % v)
def test_random_time_varying_fp32(nmpq, T):
    n, m, p, pT = nmpq
    prob = _f32(inputs.random_problem(n, m, p, T=T, seed=n * 100 + m * 10 + p, pT=pT))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("T", [9, 5000])
def test_random_time_invariant_with_c_fp32(T):
    prob = _f32(inputs.random_problem(4, 2, 2, T=T, seed=3, time_varying=False))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


def test_rank_deficient_state_cost_fp32():
    prob = _f32(inputs.random_problem(4, 2, 4, T=3000, seed=5, x_rank=1))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


def test_diag_tracking_fp32():
    prob = _f32(inputs.diag_tracking(4, T=4096, seed=0))
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("T", [1000, 100003])
def test_vehicle_fp64(T):
    prob = inputs.vehicle(T, seed=2)
    compare(gpu_solve(prob, dtype=np.float64), oracle_solve(prob), FP64_TOL)


@pytest.mark.parametrize("nm", [(1, 1), (2, 1), (4, 2)])
def test_random_fp64(nm):
    n, m = nm
    prob = inputs.random_problem(n, m, T=20011, seed=11 + n)
    compare(gpu_solve(prob, dtype=np.float64), oracle_solve(prob), FP64_TOL)


@pytest.mark.parametrize("T", [1, 1000, 20000])
def test_sequential_gpu_baseline_fp32(T):
    prob = _f32(inputs.vehicle(T, seed=4))
    compare(gpu_solve(prob, sequential=True), oracle_solve(prob), FP32_TOL)


def test_sequential_gpu_baseline_random():
    prob = _f32(inputs.random_problem(4, 2, 3, T=777, seed=21, pT=2))
    compare(gpu_solve(prob, sequential=True), oracle_solve(prob), FP32_TOL)


def test_zero_horizon():
    """T = 0: only the terminal value and x*_0 = x_0."""
    prob = _f32(inputs.vehicle(1, seed=0))
    prob.T = 0
    prob.r = prob.r[:0]
    g = gpu_solve(prob)
    o = oracle_solve(prob)
    compare(g, o, FP32_TOL, names=("S", "v", "x"))


def test_host_buffer_solve():
    import torch

    from paper_2104_03186_gb300 import lqt

    prob = _f32(inputs.vehicle(10_000, seed=3))
    P = lqt.Problem.from_inputs(prob, pin=True)
    out = P.allocate_outputs(pin=True)
    buf = torch.empty(lqt.lqt_host_solve_bytes(P), dtype=torch.uint8, device="cuda")
    st = lqt.lqt_solve_host(P, out, buf)
    assert st == lqt.LQT_OK
    compare({k: v.double().numpy() for k, v in out.items()}, oracle_solve(prob), FP32_TOL)


@pytest.mark.timeout(300)
def test_host_buffer_solves_from_two_threads():
    """Two host threads call lqt_solve_host at once, each on its own stream
    with its own buffers and problem (the end-to-end benchmark does this), a
    few times each: every result matches its oracle."""
    import threading

    import torch

    from paper_2104_03186_gb300 import lqt

    probs = [_f32(inputs.vehicle(60_000 + 977 * i, seed=40 + i)) for i in range(2)]
    refs = [oracle_solve(p) for p in probs]
    dev = torch.cuda.current_device()
    ctx = []
    for prob in probs:
        P = lqt.Problem.from_inputs(prob, pin=True)
        out = P.allocate_outputs(pin=True)
        buf = torch.empty(lqt.lqt_host_solve_bytes(P), dtype=torch.uint8, device="cuda")
        ctx.append((P, out, buf, torch.cuda.Stream()))
    results, errors = [None, None], []

    def work(i):
        try:
            torch.cuda.set_device(dev)
            P, out, buf, s = ctx[i]
            for _ in range(4):
                assert lqt.lqt_solve_host(P, out, buf, s) == lqt.LQT_OK
            results[i] = {k: v.double().numpy() for k, v in out.items()}
        except BaseException as e:
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for res, ref in zip(results, refs):
        compare(res, ref, FP32_TOL)


def test_not_spd_control_cost_is_reported():
    from paper_2104_03186_gb300 import lqt

    prob = _f32(inputs.vehicle(5000, seed=0))
    prob.U = -prob.U
    with pytest.raises(lqt.LQTError) as ei:
        gpu_solve(prob)
    assert ei.value.status == lqt.LQT_ENOTSPD


def test_non_finite_input_is_reported():
    from paper_2104_03186_gb300 import lqt

    prob = _f32(inputs.vehicle(5000, seed=0))
    prob.r = prob.r.copy()
    prob.r[1234, 0] = np.nan
    with pytest.raises(lqt.LQTError) as ei:
        gpu_solve(prob)
    assert ei.value.status in (lqt.LQT_ENONFINITE, lqt.LQT_ESINGULAR)


def test_unsupported_size_is_rejected():
    from paper_2104_03186_gb300 import lqt

    prob = _f32(inputs.random_problem(5, 2, T=10, seed=0))
    P = lqt.Problem.from_inputs(prob)
    assert lqt.lqt_workspace_bytes(P) == 0
    out = P.allocate_outputs()
    import torch

    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve(P, out, ws)
    assert ei.value.status == lqt.LQT_EUNSUPPORTED


def test_workspace_too_small_is_rejected():
    import torch

    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(_f32(inputs.vehicle(100_000)))
    out = P.allocate_outputs()
    ws = torch.empty(lqt.lqt_workspace_bytes(P) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqt.LQTError) as ei:
        lqt.lqt_solve(P, out, ws)
    assert ei.value.status == lqt.LQT_ENOMEM


PASS = ["bwd_up", "bwd_top", "bwd_down", "fwd_top", "fwd_down"]


@pytest.mark.parametrize("refine", [0, 1])
def test_profile_reports_each_kernel(refine):
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(_f32(inputs.vehicle(100_000)))
    lqt.lqt_profile_enable(True)
    try:
        lqt.solve(P, opts=refine)
        prof = lqt.lqt_profile_read()
    finally:
        lqt.lqt_profile_enable(False)
    names = PASS if not refine else PASS + [n + ".refine" for n in PASS]
    assert [n for n, _ in prof] == names
    assert all(ms > 0 for _, ms in prof)
    plan = lqt.lqt_plan(P, refine)
    assert plan["kernels"] == len(names) and plan["tiles"] >= 1


# --------------------------------------------------------------------------
# refinement on and off
# --------------------------------------------------------------------------

@pytest.mark.parametrize("T", [1000, 100003])
def test_plain_fp32_without_refinement(T):
    """Without refinement S, v, K and x* meet 1e-5; u* of the vehicle workload
    is a small difference of large terms (||u|| ~ 0.017, ||K x|| ~ 2), so FP32
    rounding of S, v and x alone moves it by a few 1e-6 and the computed u*
    by up to ~2e-5.  The bound 1e-4 documents that conditioning; the default
    (refined) path meets 1e-5."""
    prob = _f32(inputs.vehicle(T, seed=1))
    g = gpu_solve(prob, refine=0)
    o = oracle_solve(prob)
    compare(g, o, FP32_TOL, names=("S", "v", "K", "x"))
    compare(g, o, 1e-4, names=("u",))


@pytest.mark.parametrize("nm", [(3, 2), (4, 2), (4, 4)])
def test_plain_fp32_random_without_refinement(nm):
    n, m = nm
    prob = _f32(inputs.random_problem(n, m, T=20011, seed=77 + n))
    compare(gpu_solve(prob, refine=0), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("T", [4097, 100003, 1_000_000])
def test_refinement_reaches_fp32_rounding_level(T):
    """With refinement every output is within a few FP32 roundings of the
    oracle: the shifted re-solve removes the cancellation in u* (about 2e-7 is
    expected; plain FP32 gives 5e-6 to 2e-5 on u*)."""
    prob = _f32(inputs.vehicle(T, seed=1))
    errs = compare(gpu_solve(prob, refine=1), oracle_solve(prob), 1e-6)
    assert errs["x"] < 1e-7, errs


def test_refinement_keeps_S_v_K_bit_for_bit():
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(_f32(inputs.vehicle(30000, seed=5)))
    a = lqt.solve(P, opts=0)
    b = lqt.solve(P, opts=1)
    for k in ("S", "v", "K"):
        assert bool((a[k] == b[k]).all()), k


def test_refined_fp64_on_request():
    prob = inputs.vehicle(20000, seed=2)
    compare(gpu_solve(prob, dtype=np.float64, refine=1), oracle_solve(prob), FP64_TOL)


@pytest.mark.parametrize("dt_nm", [("f32", 1, 1), ("f32", 2, 1), ("f32", 3, 2), ("f32", 4, 4),
                                   ("f64", 1, 1), ("f64", 2, 1)],
                         ids=lambda v: "%s_n%d_m%d" % v)
@pytest.mark.parametrize("T", [700, 150001])
def test_refined_second_pass_replays_top_scan(dt_nm, T, single_tile):
    """The refinement pass runs its top-level backward scan from the maps the
    first pass recorded (FP32 at every n <= 4, FP64 at n <= 2, where they fit
    the CTA's shared memory): a few tiles (one or two levels; single-tile
    solves off, which would take T = 700 in one CTA) and about 150 tiles
    (eight levels), time-varying random data."""
    single_tile(0)
    dt, n, m = dt_nm
    prob = inputs.random_problem(n, m, min(n, 2), T=T, seed=300 + n + m)
    if dt == "f32":
        prob = _f32(prob)
        compare(gpu_solve(prob, refine=1), oracle_solve(prob), FP32_TOL)
    else:
        compare(gpu_solve(prob, dtype=np.float64, refine=1), oracle_solve(prob), FP64_TOL)


def test_sequential_baseline_refined_matches_parallel():
    prob = _f32(inputs.vehicle(20000, seed=6))
    o = oracle_solve(prob)
    compare(gpu_solve(prob, sequential=True, refine=1), o, FP32_TOL)
    compare(gpu_solve(prob, refine=1), o, FP32_TOL)


def test_repeated_solves_are_deterministic():
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(_f32(inputs.vehicle(50_000, seed=9)))
    a = lqt.solve(P)
    b = lqt.solve(P)
    for k in a:
        assert bool((a[k] == b[k]).all()), k
