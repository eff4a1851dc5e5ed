"""The error measures the parity tests and the benchmark use: the per-step
maximum catches an error confined to one step that the whole-array norm
dilutes, and its floor keeps steps whose reference is near zero from
dominating."""
import numpy as np

from paper_2104_03186_gb300.accuracy import errors, rel_fro, step_rel_max


def test_one_step_slip_at_full_size():
    rng = np.random.default_rng(0)
    T = 1_000_000
    ref = rng.standard_normal((T + 1, 4))
    got = ref.copy()
    nrm = np.linalg.norm(ref, axis=1)
    rms = np.sqrt(np.mean(nrm ** 2))
    k = int(np.argmin(np.where(nrm >= rms, nrm, np.inf)))  # a step of typical size
    got[k] *= 1.0 + 5e-3  # one step wrong by 5e-3 relative (a chunk-boundary slip)
    assert rel_fro(got, ref) < 1e-5          # the whole-array norm misses it
    assert abs(step_rel_max(got, ref) - 5e-3) < 1e-12   # 50x the per-step gate of 1e-4
    assert abs(step_rel_max(got, ref, 1e-6, "max") - 5e-3) < 1e-12


def test_floors_and_exact_values():
    ref = np.array([[3.0, 4.0], [0.0, 0.0], [6.0, 8.0]])
    rms = np.sqrt((25.0 + 0.0 + 100.0) / 3.0)
    got = ref + np.array([[0.0, 0.0], [1e-9, 0.0], [0.3, 0.4]])
    # step 2: 0.5 / 10; step 1: 1e-9 / rms
    assert abs(step_rel_max(got, ref) - 0.05) < 1e-15
    got2 = ref + np.array([[0.0, 0.0], [1e-3, 0.0], [0.0, 0.0]])
    assert abs(step_rel_max(got2, ref) - 1e-3 / rms) < 1e-15
    # the 1e-6 * max floor: 1e-3 / (1e-6 * 10)
    assert abs(step_rel_max(got2, ref, 1e-6, "max") - 100.0) < 1e-9
    assert step_rel_max(np.zeros((0, 3)), np.zeros((0, 3))) == 0.0
    assert step_rel_max(np.ones((2, 2)), np.zeros((2, 2))) == np.sqrt(2.0)


def test_errors_on_matrices_per_step():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((5, 3, 3))
    k = int(np.argmax(np.linalg.norm(S.reshape(5, -1), axis=1)))
    bad = S.copy()
    bad[k, 2, 1] += 1e-3 * np.linalg.norm(S[k])
    e = errors({"S": bad}, {"S": S}, names=("S",))["S"]
    assert abs(e["step_max"] - 1e-3) < 1e-12
    assert e["fro"] < e["step_max"]
