"""Python binding of the C ABI declared in include/lqt.h.

Argument marshalling only: every step of the solve runs in the CUDA kernels of
``liblqt_gb300.so``.  PyTorch is used for device memory and streams.  If the
library has not been built the import of this module fails loudly; there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblqt_gb300.so")

LQT_OK, LQT_EINVAL, LQT_ENOTSPD, LQT_ENONFINITE, LQT_ENOMEM = 0, 1, 2, 3, 4
LQT_ECUDA, LQT_ETIMEOUT, LQT_EUNSUPPORTED, LQT_ESINGULAR = 5, 6, 7, 8
LQT_F32, LQT_F64 = 0, 1

STEP_FIELDS = ("F", "c", "L", "U", "H", "r", "X")
TERMINAL_FIELDS = ("HT", "rT", "XT", "x0")
OUTPUT_FIELDS = ("S", "v", "K", "x", "u")


class lqt_in(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("step_stride", ctypes.c_int64)]


class lqt_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("p", ctypes.c_int32),
                ("pT", ctypes.c_int32), ("T", ctypes.c_int64), ("dtype", ctypes.c_int32)] + \
               [(f, lqt_in) for f in STEP_FIELDS] + \
               [(f, ctypes.c_void_p) for f in TERMINAL_FIELDS]


class lqt_solution(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in OUTPUT_FIELDS]


class lqt_batch_item(ctypes.Structure):
    _fields_ = [("problem", lqt_problem), ("solution", lqt_solution)]


class lqt_cross(ctypes.Structure):
    _fields_ = [("M", lqt_in), ("s", lqt_in)]


LQT_MODEL_UNICYCLE = 1


class lqt_nonlinear(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("sequential", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("dt", ctypes.c_double), ("x_init", ctypes.c_void_p), ("u_init", ctypes.c_void_p)]


LQT_REFINE_OFF, LQT_REFINE_ON, LQT_REFINE_AUTO, LQT_REFINE_FULL = 0, 1, 2, 3


LQT_METHOD_DEFAULT, LQT_METHOD_1, LQT_METHOD_2 = 0, 1, 2


class lqt_batch_tune_entry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("chunk_steps", ctypes.c_int32), ("t_max", ctypes.c_int64)]


class lqt_options(ctypes.Structure):
    _fields_ = [("refine", ctypes.c_int32), ("method", ctypes.c_int32),
                ("wait_probe_polls", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


def options(refine: int = LQT_REFINE_AUTO, method: int = LQT_METHOD_DEFAULT,
            wait_probe_polls: int = 0) -> lqt_options:
    """lqt_options; wait_probe_polls > 0 runs the diagnostic wait that runs out
    (n <= 4 sizes, see include/lqt.h)."""
    o = lqt_options()
    o.refine = refine
    o.method = method
    o.wait_probe_polls = wait_probe_polls
    return o


def _opts(o):
    if o is None:
        return None
    if isinstance(o, int):
        o = options(o)
    return ctypes.byref(o)


class LQTError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, lqt_strerror(status), status))


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblqt_gb300.so is not built (run paper_2104_03186_gb300.build.build()); "
                          "the LQT solver has no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, S = ctypes.POINTER(lqt_problem), ctypes.POINTER(lqt_solution)
    O = ctypes.POINTER(lqt_options)
    vp, sz, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    sig = {
        "lqt_workspace_bytes": (sz, [P, O]),
        "lqt_solve": (st, [P, S, O, vp, sz, vp]),
        "lqt_riccati_sequential": (st, [P, S, O, vp, sz, vp]),
        "lqt_workspace_status": (st, [vp, vp]),
        "lqt_host_solve_bytes": (sz, [P, O]),
        "lqt_solve_host": (st, [P, S, O, vp, sz, vp]),
        "lqt_strerror": (ctypes.c_char_p, [st]),
        "lqt_profile_enable": (st, [ctypes.c_int]),
        "lqt_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]),
        "lqt_plan": (st, [P, O] + [ctypes.POINTER(ctypes.c_int32)] * 4),
        "lqt_solve_static": (st, [P, S, O, vp]),
        "lqt_batch_workspace_bytes": (sz, [ctypes.POINTER(lqt_batch_item), ctypes.c_int32]),
        "lqt_solve_batched": (st, [ctypes.POINTER(lqt_batch_item), ctypes.c_int32, vp, sz, vp]),
        "lqt_warm_workspace_bytes": (sz, [ctypes.POINTER(lqt_batch_item), ctypes.c_int32]),
        "lqt_batch_set_tuning": (st, [ctypes.POINTER(lqt_batch_tune_entry), ctypes.c_int32,
                                      ctypes.c_int32]),
        "lqt_solve_warm": (st, [ctypes.POINTER(lqt_batch_item), ctypes.c_int32, vp, sz, vp]),
        "lqt_cross_workspace_bytes": (sz, [P, ctypes.POINTER(lqt_cross), O]),
        "lqt_solve_cross": (st, [P, ctypes.POINTER(lqt_cross), S, O, vp, sz, vp]),
        "lqt_nonlinear_workspace_bytes": (sz, [P, ctypes.POINTER(lqt_nonlinear), O]),
        "lqt_condensed_workspace_bytes": (sz, [P, ctypes.c_int32, O]),
        "lqt_solve_condensed": (st, [P, ctypes.c_int32, S, O, vp, sz, vp]),
        "lqt_solve_nonlinear": (st, [P, ctypes.POINTER(lqt_nonlinear), S, O, vp, sz, vp]),
        "lqt_set_single_tile_chunk": (st, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def library() -> ctypes.CDLL:
    return _lib


def lqt_set_single_tile_chunk(max_chunk_steps: int) -> int:
    """Problems of at most max_chunk_steps steps per thread of one tile run in
    one CTA per pass (0: never); returns the previous setting."""
    prev = ctypes.c_int32(0)
    st = _lib.lqt_set_single_tile_chunk(int(max_chunk_steps), ctypes.byref(prev))
    if st != LQT_OK:
        raise LQTError(st, "lqt_set_single_tile_chunk")
    return int(prev.value)


# ---------------------------------------------------------------------------
# batch launch plan (tuned by paper_2104_03186_gb300.tune)
# ---------------------------------------------------------------------------

TUNED_PLANS = os.path.join(_PKG, "tuned_batch_plans.json")


LQT_BATCH_PER_LEVEL, LQT_BATCH_PERSISTENT, LQT_BATCH_AUTO = 0, 1, 2
BATCH_MODES = {"per_level": LQT_BATCH_PER_LEVEL, "persistent": LQT_BATCH_PERSISTENT,
               "auto": LQT_BATCH_AUTO}


def lqt_batch_set_tuning(entries, mode="auto") -> None:
    """Set the chunk-length table and the launch mode of lqt_solve_batched for
    the lane-group sizes: entries are (n, t_max, chunk_steps) triples; mode is
    "per_level", "persistent" or "auto" (True / False: persistent /
    per_level)."""
    if isinstance(mode, bool):
        code = LQT_BATCH_PERSISTENT if mode else LQT_BATCH_PER_LEVEL
    else:
        code = BATCH_MODES[mode]
    arr = (lqt_batch_tune_entry * max(len(entries), 1))()
    for i, (n, t_max, b) in enumerate(entries):
        arr[i].n, arr[i].t_max, arr[i].chunk_steps = int(n), int(t_max), int(b)
    st = _lib.lqt_batch_set_tuning(arr, len(entries), code)
    if st != LQT_OK:
        raise LQTError(st, "lqt_batch_set_tuning")


def apply_tuned_plans(path: str = TUNED_PLANS) -> bool:
    """Apply the tuner's table (if the file exists); returns whether it did."""
    import json

    if not os.path.exists(path):
        return False
    with open(path) as f:
        plan = json.load(f)
    if "launch_mode" in plan:
        mode = plan["launch_mode"]
    else:  # a plan that only says whether the persistent launch won
        mode = bool(plan.get("persistent", True))
    lqt_batch_set_tuning([(e["n"], e["t_max"], e["chunk_steps"]) for e in plan["entries"]],
                         mode)
    return True


apply_tuned_plans()


# ---------------------------------------------------------------------------
# marshalling
# ---------------------------------------------------------------------------

def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _check_array(where: str, a, code: int, per_step: Optional[int] = None, steps: int = 0,
                 numel: Optional[int] = None) -> None:
    """What a pointer cannot carry through the C ABI, checked on the array
    itself: C-contiguous storage, the element type of the problem's dtype code
    (not checked for other codes, which the library rejects), and the extent.
    per_step: a per-step array of `per_step` elements a step, with one step
    (stride 0) or at least `steps`; numel: at least that many elements.
    Raises LQTError(LQT_EINVAL) naming the array."""
    shape = tuple(a.shape)
    if isinstance(a, np.ndarray):
        contiguous = a.flags.c_contiguous
        want = {LQT_F32: np.float32, LQT_F64: np.float64}.get(code)
    else:
        import torch

        contiguous = a.is_contiguous()
        want = {LQT_F32: torch.float32, LQT_F64: torch.float64}.get(code)
    if not contiguous:
        raise LQTError(LQT_EINVAL, "%s: not contiguous" % where)
    if want is not None and a.dtype != want:
        raise LQTError(LQT_EINVAL, "%s: element type %s, the problem's is %s" % (where, a.dtype, want))
    if per_step is not None:
        got = int(np.prod(shape[1:])) if shape else 0
        if not shape or got != per_step:
            raise LQTError(LQT_EINVAL, "%s: %d elements a step, expected %d" % (where, got, per_step))
        if shape[0] != 1 and shape[0] < steps:
            raise LQTError(LQT_EINVAL, "%s: %d steps, expected 1 or at least %d"
                           % (where, shape[0], steps))
    if numel is not None and int(np.prod(shape)) < numel:
        raise LQTError(LQT_EINVAL, "%s: %d elements, expected at least %d"
                       % (where, int(np.prod(shape)), numel))


class Problem:
    """An LQT problem whose arrays are torch tensors (device or pinned host) or
    numpy arrays (host), plus the lqt_problem struct that points at them."""

    def __init__(self, n, m, p, pT, T, dtype, arrays: Dict[str, object]):
        self.n, self.m, self.p, self.pT, self.T = n, m, p, pT, T
        self.dtype = dtype
        self.arrays = arrays
        s = lqt_problem()
        s.n, s.m, s.p, s.pT, s.T, s.dtype = n, m, p, pT, T, dtype
        step_size = {"F": n * n, "c": n, "L": n * m, "U": m * m, "H": p * n, "r": p, "X": p * p}
        for f in STEP_FIELDS:
            a = arrays.get(f)
            if a is None:
                setattr(s, f, lqt_in(None, 0))
            else:
                _check_array(f, a, dtype, per_step=step_size[f], steps=T)
                setattr(s, f, lqt_in(_ptr(a), 0 if a.shape[0] == 1 else step_size[f]))
        terminal_size = {"HT": pT * n, "rT": pT, "XT": pT * pT, "x0": n}
        for f in TERMINAL_FIELDS:
            a = arrays.get(f)
            if a is not None:
                _check_array(f, a, dtype, numel=terminal_size[f])
            setattr(s, f, _ptr(a))
        self.struct = s

    @classmethod
    def from_inputs(cls, prob, dtype=np.float32, device="cuda", pin: bool = False):
        """Copy a problem of paper_2104_03186_gb300.inputs (float64 numpy) to torch
        tensors of `dtype` on `device` (or to pinned host memory with pin=True)."""
        import torch

        tdt = torch.float32 if np.dtype(dtype) == np.float32 else torch.float64
        arrays = {}
        for f in STEP_FIELDS + TERMINAL_FIELDS:
            a = getattr(prob, f)
            if a is None:
                continue
            t = torch.from_numpy(np.ascontiguousarray(a)).to(tdt)
            arrays[f] = t.pin_memory() if pin else t.to(device)
        code = LQT_F32 if tdt == torch.float32 else LQT_F64
        return cls(prob.n, prob.m, prob.p, prob.pT, prob.T, code, arrays)

    def allocate_outputs(self, device="cuda", pin: bool = False):
        import torch

        tdt = torch.float32 if self.dtype == LQT_F32 else torch.float64
        n, m, T = self.n, self.m, self.T
        shapes = {"S": (T + 1, n, n), "v": (T + 1, n), "K": (T, m, n), "x": (T + 1, n),
                  "u": (T, m)}
        if pin:
            return {k: torch.empty(s, dtype=tdt).pin_memory() for k, s in shapes.items()}
        return {k: torch.empty(s, dtype=tdt, device=device) for k, s in shapes.items()}


class Cross:
    """Cross weights M_k (p x m) and control offsets s_k (m) of the generalised
    stage cost (Sec. IV-D) as tensors, plus the lqt_cross struct that points
    at them.  Either may be None (zero)."""

    def __init__(self, M=None, s=None):
        self.M, self.s = M, s
        c = lqt_cross()
        for f, a in (("M", M), ("s", s)):
            if a is None:
                setattr(c, f, lqt_in(None, 0))
            else:
                per_step = int(np.prod(a.shape[1:]))
                setattr(c, f, lqt_in(_ptr(a), 0 if a.shape[0] == 1 else per_step))
        self.struct = c

    @classmethod
    def from_inputs(cls, ct, dtype=np.float32, device="cuda"):
        """Copy an inputs.CrossTerms (float64 numpy) to `dtype` tensors on `device`."""
        import torch

        tdt = torch.float32 if np.dtype(dtype) == np.float32 else torch.float64

        def cv(a):
            return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(
                tdt).to(device)

        return cls(cv(ct.M), cv(ct.s))


def _cross(c, prob: "Problem"):
    """The lqt_cross struct of `c` (None: no cross terms), its arrays checked
    against `prob`: M_k is p x m, s_k has m entries, one step or at least T."""
    if c is None:
        return None
    for f, a, size in (("cross M", c.M, prob.p * prob.m), ("cross s", c.s, prob.m)):
        if a is not None:
            _check_array(f, a, prob.dtype, per_step=size, steps=prob.T)
    return ctypes.byref(c.struct)


def solution_struct(out: Dict[str, object], prob: Optional["Problem"] = None) -> lqt_solution:
    """The lqt_solution struct of the output arrays; with `prob`, each array is
    first checked (contiguous, the problem's element type, at least the
    elements the solve writes)."""
    s = lqt_solution()
    if prob is not None:
        n, m, T = prob.n, prob.m, prob.T
        size = {"S": (T + 1) * n * n, "v": (T + 1) * n, "K": T * m * n, "x": (T + 1) * n,
                "u": T * m}
        for f in OUTPUT_FIELDS:
            _check_array(f, out[f], prob.dtype, numel=size[f])
    for f in OUTPUT_FIELDS:
        setattr(s, f, _ptr(out[f]) if out[f].numel() > 0 else None)
    return s


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------------------
# the C ABI, one function each
# ---------------------------------------------------------------------------

def lqt_strerror(status: int) -> str:
    return _lib.lqt_strerror(int(status)).decode()


def lqt_workspace_bytes(prob: Problem, opts=None) -> int:
    return int(_lib.lqt_workspace_bytes(ctypes.byref(prob.struct), _opts(opts)))


def lqt_plan(prob: Problem, opts=None):
    vals = [ctypes.c_int32() for _ in range(4)]
    st = _lib.lqt_plan(ctypes.byref(prob.struct), _opts(opts), *[ctypes.byref(v) for v in vals])
    if st != LQT_OK:
        raise LQTError(st, "lqt_plan")
    return dict(chunk_steps=vals[0].value, tile_threads=vals[1].value, tiles=vals[2].value,
                kernels=vals[3].value)


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def lqt_solve(prob: Problem, out: Dict[str, object], workspace, stream=None, opts=None) -> None:
    sol = solution_struct(out, prob)
    st = _lib.lqt_solve(ctypes.byref(prob.struct), ctypes.byref(sol), _opts(opts),
                        _ptr(workspace), _nbytes(workspace), _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve")


def lqt_riccati_sequential(prob: Problem, out: Dict[str, object], workspace, stream=None,
                           opts=None) -> None:
    sol = solution_struct(out, prob)
    st = _lib.lqt_riccati_sequential(ctypes.byref(prob.struct), ctypes.byref(sol), _opts(opts),
                                     _ptr(workspace), _nbytes(workspace), _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_riccati_sequential")


def lqt_cross_workspace_bytes(prob: Problem, cross: Optional[Cross], opts=None) -> int:
    return int(_lib.lqt_cross_workspace_bytes(ctypes.byref(prob.struct), _cross(cross, prob),
                                              _opts(opts)))


def lqt_solve_cross(prob: Problem, cross: Optional[Cross], out: Dict[str, object], workspace,
                    stream=None, opts=None) -> None:
    """Generalised-cost solve (Sec. IV-D); asynchronous like lqt_solve."""
    sol = solution_struct(out, prob)
    st = _lib.lqt_solve_cross(ctypes.byref(prob.struct), _cross(cross, prob), ctypes.byref(sol),
                              _opts(opts), _ptr(workspace), _nbytes(workspace),
                              _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_cross")


def nonlinear(iterations: int = 10, dt: float = 0.1, sequential: bool = False,
              model: int = LQT_MODEL_UNICYCLE, x_init=None, u_init=None) -> lqt_nonlinear:
    """An lqt_nonlinear struct; x_init / u_init are device tensors (kept alive
    by the caller) or None."""
    nl = lqt_nonlinear()
    nl.model, nl.iterations, nl.sequential, nl.reserved = model, iterations, int(sequential), 0
    nl.dt = dt
    nl.x_init = _ptr(x_init)
    nl.u_init = _ptr(u_init)
    return nl


def _check_nominal(prob: Problem, x_init, u_init) -> None:
    """A first nominal of the iterated solve: x_init (T+1) x n, u_init T x m,
    of the problem's element type and contiguous (LQTError(LQT_EINVAL))."""
    if x_init is not None:
        _check_array("x_init", x_init, prob.dtype, numel=(prob.T + 1) * prob.n)
    if u_init is not None:
        _check_array("u_init", u_init, prob.dtype, numel=prob.T * prob.m)


def lqt_nonlinear_workspace_bytes(prob: Problem, nl: lqt_nonlinear, opts=None) -> int:
    return int(_lib.lqt_nonlinear_workspace_bytes(ctypes.byref(prob.struct), ctypes.byref(nl),
                                                  _opts(opts)))


def lqt_solve_nonlinear(prob: Problem, nl: lqt_nonlinear, out: Dict[str, object], workspace,
                        stream=None, opts=None) -> None:
    """Iterated nonlinear LQT (Sec. IV-D); asynchronous like lqt_solve."""
    sol = solution_struct(out, prob)
    st = _lib.lqt_solve_nonlinear(ctypes.byref(prob.struct), ctypes.byref(nl), ctypes.byref(sol),
                                  _opts(opts), _ptr(workspace), _nbytes(workspace),
                                  _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_nonlinear")


def lqt_condensed_workspace_bytes(prob: Problem, B: int, opts=None) -> int:
    return int(_lib.lqt_condensed_workspace_bytes(ctypes.byref(prob.struct), int(B), _opts(opts)))


def lqt_solve_condensed(prob: Problem, B: int, out: Dict[str, object], workspace, stream=None,
                        opts=None) -> None:
    """Partial condensing in blocks of B steps (Sec. V-C); asynchronous like lqt_solve."""
    sol = solution_struct(out, prob)
    st = _lib.lqt_solve_condensed(ctypes.byref(prob.struct), int(B), ctypes.byref(sol),
                                  _opts(opts), _ptr(workspace), _nbytes(workspace),
                                  _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_condensed")


def lqt_workspace_status(workspace, stream=None) -> int:
    return int(_lib.lqt_workspace_status(_ptr(workspace), _stream_handle(stream)))


def lqt_host_solve_bytes(prob: Problem, opts=None) -> int:
    return int(_lib.lqt_host_solve_bytes(ctypes.byref(prob.struct), _opts(opts)))


def lqt_solve_host(prob: Problem, out: Dict[str, object], device_buffer, stream=None,
                   opts=None) -> int:
    """Host-pointer solve; returns the device status (raises on launch errors)."""
    sol = solution_struct(out, prob)
    st = _lib.lqt_solve_host(ctypes.byref(prob.struct), ctypes.byref(sol), _opts(opts),
                             _ptr(device_buffer), _nbytes(device_buffer), _stream_handle(stream))
    if st in (LQT_EINVAL, LQT_ENOMEM, LQT_EUNSUPPORTED, LQT_ECUDA):
        raise LQTError(st, "lqt_solve_host")
    return int(st)


def _items(problems, outputs):
    count = len(problems)
    arr = (lqt_batch_item * max(count, 1))()
    for i, (P, out) in enumerate(zip(problems, outputs)):
        arr[i].problem = P.struct
        arr[i].solution = solution_struct(out, P)
    return arr


def lqt_batch_workspace_bytes(problems, outputs) -> int:
    """Workspace bytes of lqt_solve_batched for these problems and outputs
    (0: an item is invalid or unsupported)."""
    return int(_lib.lqt_batch_workspace_bytes(_items(problems, outputs), len(problems)))


def lqt_solve_batched(problems, outputs, workspace, stream=None) -> None:
    """Solve a ragged batch: problems[i] (Problem, device tensors) into
    outputs[i] (dict of device tensors).  Asynchronous; read the device status
    with lqt_workspace_status(workspace)."""
    st = _lib.lqt_solve_batched(_items(problems, outputs), len(problems), _ptr(workspace),
                                _nbytes(workspace), _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_batched")


# numpy mirror of lqt_batch_item, for building descriptor arrays column-wise
BATCH_ITEM = np.dtype(lqt_batch_item)


def lqt_batch_workspace_bytes_array(items: np.ndarray) -> int:
    """lqt_batch_workspace_bytes over a C-contiguous numpy array of BATCH_ITEM."""
    return int(_lib.lqt_batch_workspace_bytes(
        items.ctypes.data_as(ctypes.POINTER(lqt_batch_item)), len(items)))


def lqt_solve_batched_array(items: np.ndarray, workspace, stream=None) -> None:
    """lqt_solve_batched over a C-contiguous numpy array of BATCH_ITEM."""
    if items.dtype != BATCH_ITEM or not items.flags.c_contiguous:
        raise LQTError(LQT_EINVAL, "items must be a contiguous BATCH_ITEM array")
    st = _lib.lqt_solve_batched(items.ctypes.data_as(ctypes.POINTER(lqt_batch_item)), len(items),
                                _ptr(workspace), _nbytes(workspace), _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_batched")


def lqt_warm_workspace_bytes_array(items: np.ndarray) -> int:
    """lqt_warm_workspace_bytes over a C-contiguous numpy array of BATCH_ITEM."""
    return int(_lib.lqt_warm_workspace_bytes(
        items.ctypes.data_as(ctypes.POINTER(lqt_batch_item)), len(items)))


def lqt_solve_warm_array(items: np.ndarray, workspace, stream=None) -> None:
    """lqt_solve_warm over a C-contiguous numpy array of BATCH_ITEM (each
    solution's S and K hold the known S_k, K_k on entry)."""
    if items.dtype != BATCH_ITEM or not items.flags.c_contiguous:
        raise LQTError(LQT_EINVAL, "items must be a contiguous BATCH_ITEM array")
    st = _lib.lqt_solve_warm(items.ctypes.data_as(ctypes.POINTER(lqt_batch_item)), len(items),
                             _ptr(workspace), _nbytes(workspace), _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_warm")


def lqt_warm_workspace_bytes(problems, outputs) -> int:
    return int(_lib.lqt_warm_workspace_bytes(_items(problems, outputs), len(problems)))


def lqt_solve_warm(problems, outputs, workspace, stream=None) -> None:
    """Warm solves: outputs[i]["S"] and ["K"] hold the known S_k and K_k of
    problems[i] on entry (they are only read); v, x, u are written.
    Asynchronous; read the device status with lqt_workspace_status."""
    st = _lib.lqt_solve_warm(_items(problems, outputs), len(problems), _ptr(workspace),
                             _nbytes(workspace), _stream_handle(stream))
    if st != LQT_OK:
        raise LQTError(st, "lqt_solve_warm")


def solve_warm(problems, known, stream=None, check: bool = True):
    """Allocate v, x, u with torch and run lqt_solve_warm; known[i] is a dict
    with the device tensors "S" ((T+1) x n x n) and "K" (T x m x n) of
    problems[i], used in place."""
    import torch

    outs = []
    for P, kn in zip(problems, known):
        o = P.allocate_outputs()
        o["S"], o["K"] = kn["S"], kn["K"]
        outs.append(o)
    nbytes = lqt_warm_workspace_bytes(problems, outs)
    if nbytes == 0:
        raise LQTError(LQT_EUNSUPPORTED, "lqt_warm_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lqt_solve_warm(problems, outs, ws, stream)
    if check:
        st = lqt_workspace_status(ws, stream)
        if st != LQT_OK:
            raise LQTError(st, "device status")
    return outs


def solve_batched(problems, stream=None, check: bool = True):
    """Allocate outputs and a workspace with torch and run lqt_solve_batched."""
    import torch

    outs = [P.allocate_outputs() for P in problems]
    nbytes = lqt_batch_workspace_bytes(problems, outs)
    if nbytes == 0:
        raise LQTError(LQT_EUNSUPPORTED, "lqt_batch_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lqt_solve_batched(problems, outs, ws, stream)
    if check:
        st = lqt_workspace_status(ws, stream)
        if st != LQT_OK:
            raise LQTError(st, "device status")
    return outs


LQT_STATIC_SCRATCH_BYTES = 32 << 20


def lqt_solve_static(prob: Problem, out: Dict[str, object], stream=None, opts=None) -> int:
    """lqt_solve with the library's built-in scratch array instead of a workspace,
    for callers that cannot allocate device memory.  Waits for the stream and
    returns the device status of the solve; raises on argument, size
    (LQT_ENOMEM: the problem needs more than LQT_STATIC_SCRATCH_BYTES) and
    launch errors.  Calls that overlap on the GPU share the array and race."""
    sol = solution_struct(out, prob)
    st = _lib.lqt_solve_static(ctypes.byref(prob.struct), ctypes.byref(sol), _opts(opts),
                               _stream_handle(stream))
    if st in (LQT_EINVAL, LQT_ENOMEM, LQT_EUNSUPPORTED, LQT_ECUDA):
        raise LQTError(st, "lqt_solve_static")
    return int(st)


def lqt_profile_enable(enable: bool) -> None:
    _lib.lqt_profile_enable(1 if enable else 0)


def lqt_profile_read(max_entries: int = 16):
    ms = (ctypes.c_float * max_entries)()
    names = (ctypes.c_char_p * max_entries)()
    k = _lib.lqt_profile_read(ms, names, max_entries)
    if k < 0:
        raise LQTError(LQT_ECUDA, "lqt_profile_read")
    return [(names[i].decode(), float(ms[i])) for i in range(min(k, max_entries))]


# ---------------------------------------------------------------------------
# convenience: allocate with torch, call the C ABI
# ---------------------------------------------------------------------------

def workspace_for(prob: Problem, device="cuda", opts=None):
    import torch

    nbytes = lqt_workspace_bytes(prob, opts)
    if nbytes == 0:
        raise LQTError(LQT_EUNSUPPORTED, "lqt_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def solve(prob: Problem, stream=None, check: bool = True, workspace=None, sequential=False,
          opts=None):
    """Allocate outputs (and a workspace) with torch and run lqt_solve (or the
    sequential baseline).  With check=True the stream is synchronised and a
    non-OK device status raises LQTError."""
    out = prob.allocate_outputs()
    ws = workspace if workspace is not None else workspace_for(prob, opts=opts)
    if sequential:
        lqt_riccati_sequential(prob, out, ws, stream, opts)
    else:
        lqt_solve(prob, out, ws, stream, opts)
    if check:
        st = lqt_workspace_status(ws, stream)
        if st != LQT_OK:
            raise LQTError(st, "device status")
    return out


def solve_cross(prob: Problem, cross: Optional[Cross], stream=None, check: bool = True,
                opts=None):
    """Allocate outputs and a workspace with torch and run lqt_solve_cross."""
    import torch

    out = prob.allocate_outputs()
    nbytes = lqt_cross_workspace_bytes(prob, cross, opts)
    if nbytes == 0:
        raise LQTError(LQT_EUNSUPPORTED, "lqt_cross_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lqt_solve_cross(prob, cross, out, ws, stream, opts)
    if check:
        st = lqt_workspace_status(ws, stream)
        if st != LQT_OK:
            raise LQTError(st, "device status")
    return out


def solve_nonlinear(prob: Problem, iterations: int = 10, dt: float = 0.1, sequential=False,
                    stream=None, check: bool = True, opts=None, x_init=None, u_init=None):
    """Allocate outputs and a workspace with torch and run lqt_solve_nonlinear
    (the unicycle model)."""
    import torch

    _check_nominal(prob, x_init, u_init)
    nl = nonlinear(iterations, dt, sequential, LQT_MODEL_UNICYCLE, x_init, u_init)
    out = prob.allocate_outputs()
    nbytes = lqt_nonlinear_workspace_bytes(prob, nl, opts)
    if nbytes == 0:
        raise LQTError(LQT_EUNSUPPORTED, "lqt_nonlinear_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lqt_solve_nonlinear(prob, nl, out, ws, stream, opts)
    if check:
        st = lqt_workspace_status(ws, stream)
        if st != LQT_OK:
            raise LQTError(st, "device status")
    return out


def solve_condensed(prob: Problem, B: int, stream=None, check: bool = True, opts=None):
    """Allocate outputs and a workspace with torch and run lqt_solve_condensed."""
    import torch

    out = prob.allocate_outputs()
    nbytes = lqt_condensed_workspace_bytes(prob, B, opts)
    if nbytes == 0:
        raise LQTError(LQT_EUNSUPPORTED, "lqt_condensed_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lqt_solve_condensed(prob, B, out, ws, stream, opts)
    if check:
        st = lqt_workspace_status(ws, stream)
        if st != LQT_OK:
            raise LQTError(st, "device status")
    return out
