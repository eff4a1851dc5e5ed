"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the
same seeded inputs and compare them output by output."""
import numpy as np

from conftest import rel_fro

FP32_TOL = 1e-5   # relative Frobenius error per output, FP32 path vs FP64 oracle
FP64_TOL = 1e-11  # same, FP64 path


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


def compare(gpu, ref, tol, names=("S", "v", "K", "x", "u")):
    """Relative Frobenius error of each output; asserts each is within tol."""
    errs = {k: rel_fro(gpu[k], ref[k]) for k in names}
    bad = {k: e for k, e in errs.items() if not (e <= tol)}
    assert not bad, "errors above %g: %s (all: %s)" % (tol, bad, errs)
    return errs
