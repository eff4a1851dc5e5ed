"""Single problems at the lane-group sizes (n = 8, 16, 32) through lqt_solve:
the chunked pipeline (chunk folds, one launch per tree level, re-fold,
forward scan, rollout) against the FP64 oracle, in FP32, FP32 with FP64 tree
levels and refinement, and FP64; its one-chunk form through
lqt_riccati_sequential; and the precision-study workload."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, compare, gpu_solve, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(8, 4), (16, 8), (32, 16)]


def _rand(n, m, T, seed, **kw):
    return inputs.random_problem(n, m, T=T, seed=seed, **kw)


@pytest.mark.parametrize("n,m", SIZES)
@pytest.mark.parametrize("T", [1, 5, 333, 2000])
@pytest.mark.parametrize("refine", [0, 1])
def test_chain_fp32_matches_oracle(n, m, T, refine):
    prob = _rand(n, m, T, seed=n * 1000 + T).rounded_to(np.float32)
    compare(gpu_solve(prob, refine=refine), oracle_solve(prob), FP32_TOL)


@pytest.mark.parametrize("n,m", SIZES)
@pytest.mark.parametrize("T", [1, 333, 2000])
def test_chain_fp64_matches_oracle(n, m, T):
    prob = _rand(n, m, T, seed=7 + n + T)
    compare(gpu_solve(prob, dtype=np.float64), oracle_solve(prob), FP64_TOL)


@pytest.mark.parametrize("n,m", SIZES)
def test_chain_sequential_matches_oracle(n, m):
    prob = _rand(n, m, 300, seed=3 + n).rounded_to(np.float32)
    compare(gpu_solve(prob, sequential=True, refine=1), oracle_solve(prob), FP32_TOL)
    prob64 = _rand(n, m, 300, seed=4 + n)
    compare(gpu_solve(prob64, dtype=np.float64, sequential=True), oracle_solve(prob64), FP64_TOL)


@pytest.mark.parametrize("n,m,kw,refine", [
    (8, 4, dict(p=4, pT=1), 1),                 # p < n, one terminal row
    (8, 4, dict(p=16, pT=16), 1),               # p = 2n
    (16, 8, dict(with_c=False, pT=0), 1),       # no offsets, no terminal cost
    # step stride 0 for every matrix; F with spectral radius up to 1.05 held for
    # all steps makes S ill-conditioned enough (FP32 solve: S 8e-6, v 1.8e-5)
    # that S and v need the Newton step of the FULL refinement
    (16, 8, dict(time_varying=False), 3),
    (32, 16, dict(p=8, x_rank=3), 1),           # rank-deficient X_k
])
def test_chain_shapes(n, m, kw, refine):
    prob = _rand(n, m, 777, seed=11, **kw).rounded_to(np.float32)
    compare(gpu_solve(prob, refine=refine), oracle_solve(prob), FP32_TOL)
    prob64 = _rand(n, m, 777, seed=12, **kw)
    compare(gpu_solve(prob64, dtype=np.float64), oracle_solve(prob64), FP64_TOL)


@pytest.mark.parametrize("n,m", [(4, 2)] + SIZES)
@pytest.mark.parametrize("sequential", [False, True])
def test_chain_full_refinement(n, m, sequential):
    """FULL refinement (FP64 tree levels, Newton step for S, v, K, KKT step
    for x*, u*): every output at FP32 rounding level."""
    prob = _rand(n, m, 500, seed=21 + n).rounded_to(np.float32)
    errs = compare(gpu_solve(prob, refine=3, sequential=sequential), oracle_solve(prob), 1e-6)
    assert max(errs.values()) < 1e-6


def test_chain_kkt_refinement_fixes_trajectory():
    """ON refinement: x* and u* reach FP32 rounding level even where the plain
    FP32 solve misses 1e-5 (the precision-study workload)."""
    prob = inputs.precision_study(T=2048, seed=3).rounded_to(np.float32)
    ref = oracle_solve(prob)
    plain = compare(gpu_solve(prob, refine=0), ref, 1.0)
    refined = compare(gpu_solve(prob, refine=1), ref, FP32_TOL)
    assert refined["x"] < 1e-6 and refined["u"] < 1e-6
    assert refined["x"] < plain["x"] / 10


@pytest.mark.parametrize("n,m", SIZES)
def test_chain_zero_horizon(n, m):
    prob = _rand(n, m, 4, seed=1).rounded_to(np.float32)
    prob.T = 0
    for f in ("F", "c", "L", "U", "H", "r", "X"):
        a = getattr(prob, f)
        if a is not None and a.shape[0] > 1:
            setattr(prob, f, a[:0])
    g = gpu_solve(prob)
    o = oracle_solve(prob)
    compare(g, o, FP32_TOL, names=("S", "v", "x"))


def test_chain_plan_spans_levels():
    """The planner cuts a long problem into a power-of-two number of chunks."""
    from paper_2104_03186_gb300 import lqt

    for n, m in SIZES:
        P = lqt.Problem.from_inputs(_rand(n, m, 5000, seed=0).rounded_to(np.float32))
        plan = lqt.lqt_plan(P, 0)
        nc, B = plan["tiles"], plan["chunk_steps"]
        assert nc >= 2 and nc & (nc - 1) == 0
        assert B * nc >= 5000 and B >= 4


@pytest.mark.parametrize("T", [4096])
def test_precision_study_small(T):
    """The precision-study workload (n = 32, cond(X_k) = 1e6, U = 1e-3 I) at a
    short horizon: FP64 within 1e-11, the refined forms within 1e-5 (FULL
    within 1e-6)."""
    prob = inputs.precision_study(T=T, seed=1)
    o64 = oracle_solve(prob)
    compare(gpu_solve(prob, dtype=np.float64), o64, FP64_TOL)
    p32 = prob.rounded_to(np.float32)
    o32 = oracle_solve(p32)
    compare(gpu_solve(p32, refine=1), o32, FP32_TOL)
    compare(gpu_solve(p32, refine=3), o32, 1e-6)


def test_chain_fp64_refined_matches_oracle():
    """FP64 with the KKT refinement (ON) and the FULL refinement."""
    prob = _rand(16, 8, 600, seed=31)
    ref = oracle_solve(prob)
    compare(gpu_solve(prob, dtype=np.float64, refine=1), ref, FP64_TOL)
    compare(gpu_solve(prob, dtype=np.float64, refine=3), ref, FP64_TOL)


def test_chain_host_and_static_entry_points():
    """The host-buffer solve and the no-workspace solve at a lane size."""
    import torch

    from paper_2104_03186_gb300 import lqt

    prob = _rand(8, 4, 900, seed=41).rounded_to(np.float32)
    ref = oracle_solve(prob)
    Ph = lqt.Problem.from_inputs(prob, pin=True)
    out_h = Ph.allocate_outputs(pin=True)
    buf = torch.empty(lqt.lqt_host_solve_bytes(Ph, None), dtype=torch.uint8, device="cuda")
    assert lqt.lqt_solve_host(Ph, out_h, buf, None, None) == lqt.LQT_OK
    compare({k: v.double().numpy() for k, v in out_h.items()}, ref, FP32_TOL)
    P = lqt.Problem.from_inputs(prob)
    out = P.allocate_outputs()
    assert lqt.lqt_solve_static(P, out, None, None) == lqt.LQT_OK
    torch.cuda.synchronize()
    compare({k: v.double().cpu().numpy() for k, v in out.items()}, ref, FP32_TOL)


def test_chain_no_stage_cost():
    """p = 0: no stage tracking cost, only the terminal cost."""
    prob = _rand(8, 4, 300, seed=51, p=0).rounded_to(np.float32)
    compare(gpu_solve(prob), oracle_solve(prob), FP32_TOL)


def test_batch_mixes_lane_sizes_and_edge_items():
    """One batch with n = 4, 8, 16, 32 problems, p < n and p = 2n, a T = 0 item
    and several chunk counts: every item against the oracle."""
    from paper_2104_03186_gb300 import lqt

    specs = [(4, 2, 7, {}), (8, 4, 1, {}), (8, 4, 3000, dict(p=16, pT=16)),
             (16, 8, 513, dict(p=4, pT=2)), (32, 16, 2048, {}), (32, 16, 5, {}),
             (16, 8, 0, {}), (8, 4, 64, dict(with_c=False))]
    probs = []
    for i, (n, m, T, kw) in enumerate(specs):
        pr = _rand(n, m, max(T, 1), seed=60 + i, **kw).rounded_to(np.float32)
        if T == 0:
            pr.T = 0
            for f in ("F", "c", "L", "U", "H", "r", "X"):
                a = getattr(pr, f)
                if a is not None and a.shape[0] > 1:
                    setattr(pr, f, a[:0])
        probs.append(pr)
    Ps = [lqt.Problem.from_inputs(p) for p in probs]
    outs = lqt.solve_batched(Ps)
    for pr, out, (n, m, T, kw) in zip(probs, outs, specs):
        g = {k: v.double().cpu().numpy() for k, v in out.items()}
        names = ("S", "v", "x") if T == 0 else ("S", "v", "K", "x", "u")
        compare(g, oracle_solve(pr), FP32_TOL, names=names)


@pytest.mark.parametrize("n,m", [(4, 2)] + SIZES)
@pytest.mark.parametrize("refine", [0, 1])
def test_chain_method2_matches_oracle(n, m, refine):
    """Trajectory by Method 2 (Lemma LQT_trajectory_method2: forward element scan
    from (0, x_0, 0, 0, 0), x*_k = (I + C S_k)^{-1}(b + C v_k)) against the
    oracle, FP32 (plain and refined) and FP64."""
    prob = _rand(n, m, 700, seed=70 + n).rounded_to(np.float32)
    ref = oracle_solve(prob)
    compare(gpu_solve(prob, refine=refine, method=2), ref, FP32_TOL)
    prob64 = _rand(n, m, 700, seed=71 + n)
    compare(gpu_solve(prob64, dtype=np.float64, method=2), oracle_solve(prob64), FP64_TOL)


def test_chain_method2_sequential_and_edge_cases():
    """Method 2 with one chunk (the sequential path), T = 1, and the vehicle-style
    diagonal tracking model."""
    for T, seq in ((300, True), (1, False), (5, False)):
        prob = _rand(8, 4, T, seed=80 + T).rounded_to(np.float32)
        compare(gpu_solve(prob, refine=0, method=2, sequential=seq), oracle_solve(prob), FP32_TOL)
    prob = inputs.diag_tracking(16, T=2000, seed=4).rounded_to(np.float32)
    compare(gpu_solve(prob, method=2), oracle_solve(prob), FP32_TOL)


def test_small_size_full_refinement_routes_to_chain():
    """n = 4: FULL refinement and Method 2 run the chunked pipeline (n = 4 lane
    groups), whose Newton step brings S, v, K of a time-invariant problem with
    open-loop spectral radius up to 1.05 to FP32 level; the thread-per-step
    kernels (ON) leave S near 1e-4 there."""
    from paper_2104_03186_gb300 import lqt

    prob = _rand(4, 2, 700, seed=504, time_varying=False).rounded_to(np.float32)
    ref = oracle_solve(prob)
    full = compare(gpu_solve(prob, refine=3), ref, FP32_TOL)
    assert max(full.values()) < 2e-6
    P = lqt.Problem.from_inputs(prob)
    assert lqt.lqt_plan(P, 3)["tile_threads"] == 4      # lane group of n lanes
    assert lqt.lqt_plan(P, 1)["tile_threads"] != 4      # thread-per-step tiles
    compare(gpu_solve(prob, refine=3, method=2), ref, FP32_TOL)
    prob64 = _rand(4, 2, 700, seed=505, time_varying=False)
    compare(gpu_solve(prob64, dtype=np.float64, refine=3), oracle_solve(prob64), FP64_TOL)
    compare(gpu_solve(prob64, dtype=np.float64, method=2), oracle_solve(prob64), FP64_TOL)
