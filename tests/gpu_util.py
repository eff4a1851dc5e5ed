"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the
same seeded inputs and compare them output by output."""
import numpy as np

from paper_2104_03186_gb300.accuracy import rel_fro, step_rel_max

FP32_TOL = 1e-5   # relative error per output, FP32 path vs FP64 oracle
FP64_TOL = 1e-11  # same, FP64 path
# The per-step check (see compare) allows STEP_FACTOR times the whole-array
# tolerance: a correct solve's error is not spread evenly over the horizon
# (measured: at most 4x the whole-array bound on every parity test), while a
# slip confined to a few steps shows at about sqrt(T) times its whole-array
# size, far above the gate.
STEP_FACTOR = 10.0


def gpu_solve(prob, dtype=np.float32, sequential=False, refine=None, method=0):
    """CUDA path through the C ABI; refine=None takes the library default
    (refinement for FP32, none for FP64); method 2 takes Method 2 for the
    trajectory."""
    from paper_2104_03186_gb300 import lqt

    P = lqt.Problem.from_inputs(prob, dtype=dtype)
    opts = refine
    if method:
        opts = lqt.options(lqt.LQT_REFINE_AUTO if refine is None else refine, method)
    out = lqt.solve(P, sequential=sequential, opts=opts)
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def oracle_solve(prob):
    import oracle

    return oracle.riccati(prob, keep_kv_kc=False)


class Errs(dict):
    """Whole-array relative errors per output; .step holds the per-step maxima."""

    step: dict


def compare(gpu, ref, tol, names=("S", "v", "K", "x", "u"), step_tol=None):
    """Checks every output two ways and asserts both are within tolerance:
    the relative Frobenius error over the whole stacked array (<= tol) and the
    largest per-step relative error, max_k ||Y_k - Y_ref,k|| / max(||Y_ref,k||,
    rms_j ||Y_ref,j||) (<= step_tol, default STEP_FACTOR * tol).  The per-step
    check catches an error confined to a few steps (a chunk or tile
    boundary), which the whole-array norm dilutes by about 1/sqrt(T).
    Returns the whole-array errors; .step has the per-step ones."""
    step_tol = STEP_FACTOR * tol if step_tol is None else step_tol
    errs = Errs({k: rel_fro(gpu[k], ref[k]) for k in names})
    errs.step = {k: step_rel_max(gpu[k], ref[k]) for k in names}
    bad = {k: e for k, e in errs.items() if not (e <= tol)}
    bad_step = {k: e for k, e in errs.step.items() if not (e <= step_tol)}
    assert not bad and not bad_step, (
        "whole-array errors above %g: %s; per-step errors above %g: %s (all: %s; per step: %s)"
        % (tol, bad, step_tol, bad_step, dict(errs), errs.step))
    return errs
