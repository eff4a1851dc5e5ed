"""Error measures of a solve against a reference solution (no solver arithmetic).

The paper states that the sequential and the parallel method reach the same
solution (Sec. VI); it states no error metric.  Per output Y in {S, v, K, x*,
u*}, each array with the time step on its first axis:

* rel_fro: ||Y - Y_ref||_F / ||Y_ref||_F over the whole stacked array.
* step_rel_max: max over steps k of ||Y_k - Y_ref,k|| / max(||Y_ref,k||, rho),
  rho = the root mean square of the per-step reference norms ||Y_ref,j||.
  A whole-array norm dilutes an error confined to one step by about
  1/sqrt(T); this maximum does not, so a slip at one chunk or tile boundary
  shows at full size.  The floor rho is the output's typical step size: the
  rounding error of a correct solve at step k scales with the terms that form
  Y_k (u*_k = -K_k x*_k + d_k is a small difference of large terms), not with
  ||Y_k|| itself, so without a floor the measure would report how close Y_k
  comes to zero rather than how accurate it is.
* step_rel_max(..., floor=1e-6, scale="max"): the same with the floor
  1e-6 * max_j ||Y_ref,j||, reported beside the other for reference.
"""
from __future__ import annotations

import numpy as np

NAMES = ("S", "v", "K", "x", "u")


def rel_fro(a, b) -> float:
    """||a - b||_F / ||b||_F over the whole array (the plain norm when b is 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    return float(num if den == 0.0 else num / den)


def step_rel_max(a, b, floor: float = 1.0, scale: str = "rms") -> float:
    """Largest per-step relative error, steps on axis 0.  Each step's
    reference norm is floored at floor * (the RMS of the per-step reference
    norms) with scale="rms", or at floor * (their maximum) with scale="max"."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("shape mismatch %s vs %s" % (a.shape, b.shape))
    if a.size == 0:
        return 0.0
    a2 = a.reshape(a.shape[0], -1)
    b2 = b.reshape(b.shape[0], -1)
    d = np.linalg.norm(a2 - b2, axis=1)
    r = np.linalg.norm(b2, axis=1)
    if scale == "rms":
        ref = float(np.sqrt(np.mean(r * r)))
    elif scale == "max":
        ref = float(r.max())
    else:
        raise ValueError(scale)
    if ref == 0.0:
        return float(d.max())
    return float((d / np.maximum(r, floor * ref)).max())


def errors(got, ref, names=NAMES) -> dict:
    """Per output: the whole-array error, the per-step maximum (RMS floor) and
    the per-step maximum with the 1e-6 * max floor."""
    return {k: {"fro": rel_fro(got[k], ref[k]),
                "step_max": step_rel_max(got[k], ref[k]),
                "step_max_floor_1e-6max": step_rel_max(got[k], ref[k], 1e-6, "max")}
            for k in names}
