"""FP64 CPU oracle for the LQT problem -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never loads it, and the oracle shares no code with that path.

The arithmetic lives in ``lqt_oracle.c`` (plain C, float64), which follows the
paper's formulas step by step:

* ``riccati``         Sec. II-B: S_k, v_k, K_k, K^v_k, K^c_k backward, then
                      u*_k (eq. Control_LQT) and x*_k (eq. optimal_trajectory).
* ``element``         Lemma LQT_assoc / eq. lqt_init (and the terminal element).
* ``combine``         Lemma LQT_combination / eq. lqt_comb.
* ``affine_combine``  Lemma LQT_trajectory_combination.
* ``method2_state``   Lemma LQT_trajectory_method2 / eq. lqt_method_2.

``oracle.cross`` (numpy, float64) adds the generalised stage cost of
Sec. IV-D (cross weight M_k, control offset s_k) by the paper's substitution
around ``riccati``.  ``oracle.nonlinear`` runs the iterated linearise-and-solve
passes of Sec. IV-D for the unicycle of Sec. VI-E around ``riccati``.

Pins (tests that tie these to something other than themselves) live in
``tests/test_oracle_*.py``.  Every function here is pinned.

Problems are duck-typed: any object with the fields of an LQT problem
(F, c, L, U, H, r, X with a leading time axis of 1 or T; HT, rT, XT, x0; T).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqt_oracle.c")
_SO = os.path.join(_HERE, "liblqt_oracle.so")
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int), ("pT", ctypes.c_int),
        ("T", ctypes.c_long),
        ("F", _dp), ("c", _dp), ("L", _dp), ("U", _dp),
        ("H", _dp), ("r", _dp), ("X", _dp),
        ("sF", ctypes.c_long), ("sc", ctypes.c_long), ("sL", ctypes.c_long),
        ("sU", ctypes.c_long), ("sH", ctypes.c_long), ("sr", ctypes.c_long),
        ("sX", ctypes.c_long),
        ("HT", _dp), ("rT", _dp), ("XT", _dp), ("x0", _dp),
    ]


def build(force: bool = False, src: str = _SRC, so: str = _SO) -> str:
    """Compile the C oracle (gcc, -O2, no host-specific flags) into ``so``."""
    with _lock:
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + ".tmp.%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src,
                                   "-lm"])
            os.replace(tmp, so)
    return so


def _ptr(a):
    if a is None:
        return ctypes.cast(None, _dp)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Marshalled:
    """Keeps the float64 copies alive while the C code reads them."""

    def __init__(self, prob):
        self.arrays = {}
        s = _Problem()
        s.n = int(prob.F.shape[-1])
        s.m = int(prob.L.shape[-1])
        s.p = int(prob.H.shape[-2])
        s.pT = int(prob.HT.shape[0])
        s.T = int(prob.T)
        for name in ("F", "c", "L", "U", "H", "r", "X"):
            a = _f64(getattr(prob, name))
            self.arrays[name] = a
            setattr(s, name, _ptr(a))
            stride = 0 if (a is None or a.shape[0] == 1) else int(np.prod(a.shape[1:]))
            setattr(s, "s" + name, stride)
        for name in ("HT", "rT", "XT", "x0"):
            a = _f64(getattr(prob, name))
            self.arrays[name] = a
            setattr(s, name, _ptr(a))
        self.s = s
        self.n, self.m, self.T = s.n, s.m, s.T


class Oracle:
    """The oracle's entry points bound to one compiled copy of ``lqt_oracle.c``."""

    def __init__(self, so_path: str):
        lib = ctypes.CDLL(so_path)
        lib.oracle_riccati.restype = ctypes.c_int
        lib.oracle_riccati.argtypes = [ctypes.POINTER(_Problem)] + [_dp] * 7
        lib.oracle_element.restype = ctypes.c_int
        lib.oracle_element.argtypes = [ctypes.POINTER(_Problem), ctypes.c_long] + [_dp] * 5
        lib.oracle_combine.restype = ctypes.c_int
        lib.oracle_combine.argtypes = [ctypes.c_int] + [_dp] * 15
        lib.oracle_affine_combine.restype = None
        lib.oracle_affine_combine.argtypes = [ctypes.c_int] + [_dp] * 6
        lib.oracle_method2_state.restype = ctypes.c_int
        lib.oracle_method2_state.argtypes = [ctypes.c_int] + [_dp] * 7
        self.lib = lib

    def riccati(self, prob, keep_kv_kc: bool = True) -> dict:
        """Sequential FP64 LQT solution (Sec. II-B).

        Returns a dict of float64 arrays: S (T+1,n,n), v (T+1,n), K (T,m,n),
        Kv (T,m,n), Kc (T,m,n), x (T+1,n), u (T,m)."""
        mp = _Marshalled(prob)
        n, m, T = mp.n, mp.m, mp.T
        out = {
            "S": np.zeros((T + 1, n, n)), "v": np.zeros((T + 1, n)), "K": np.zeros((T, m, n)),
            "x": np.zeros((T + 1, n)), "u": np.zeros((T, m)),
        }
        if keep_kv_kc:
            out["Kv"] = np.zeros((T, m, n))
            out["Kc"] = np.zeros((T, m, n))
        rc = self.lib.oracle_riccati(ctypes.byref(mp.s), _ptr(out["S"]), _ptr(out["v"]),
                                     _ptr(out["K"]), _ptr(out.get("Kv")), _ptr(out.get("Kc")),
                                     _ptr(out["x"]), _ptr(out["u"]))
        if rc != 0:
            raise ArithmeticError("oracle: L^T S L + U is singular")
        return out

    def element(self, prob, k: int):
        """Element a_k = (A, b, C, eta, J) of eq. lqt_init; k == T gives the terminal element."""
        mp = _Marshalled(prob)
        n = mp.n
        A, b, C, eta, J = (np.zeros((n, n)), np.zeros(n), np.zeros((n, n)), np.zeros(n),
                           np.zeros((n, n)))
        rc = self.lib.oracle_element(ctypes.byref(mp.s), int(k), _ptr(A), _ptr(b), _ptr(C),
                                     _ptr(eta), _ptr(J))
        if rc != 0:
            raise ArithmeticError("oracle: U_k is singular")
        return A, b, C, eta, J

    def combine(self, e1, e2):
        """e1 (x) e2 by eq. lqt_comb; e1 covers k -> j and e2 covers j -> i."""
        e1 = [_f64(a) for a in e1]
        e2 = [_f64(a) for a in e2]
        n = e1[0].shape[0]
        A, b, C, eta, J = (np.zeros((n, n)), np.zeros(n), np.zeros((n, n)), np.zeros(n),
                           np.zeros((n, n)))
        rc = self.lib.oracle_combine(n, *[_ptr(a) for a in e1], *[_ptr(a) for a in e2], _ptr(A),
                                     _ptr(b), _ptr(C), _ptr(eta), _ptr(J))
        if rc != 0:
            raise ArithmeticError("oracle: I + C1 J2 is singular")
        return A, b, C, eta, J

    def affine_combine(self, f1, f2):
        """(F, c) of x -> f2(f1(x)) for affine maps f = (F, c)
        (Lemma LQT_trajectory_combination)."""
        F1, c1 = _f64(f1[0]), _f64(f1[1])
        F2, c2 = _f64(f2[0]), _f64(f2[1])
        n = F1.shape[0]
        F, c = np.zeros((n, n)), np.zeros(n)
        self.lib.oracle_affine_combine(n, _ptr(F1), _ptr(c1), _ptr(F2), _ptr(c2), _ptr(F),
                                       _ptr(c))
        return F, c

    def method2_state(self, fwd_elem, S, v, xS):
        """x*_k of eq. lqt_method_2 from the forward element (A, b, C) of V_{S->k}
        and the value function (S_k, v_k)."""
        A, b, C = (_f64(a) for a in fwd_elem[:3])
        S, v, xS = _f64(S), _f64(v), _f64(xS)
        n = A.shape[0]
        x = np.zeros(n)
        rc = self.lib.oracle_method2_state(n, _ptr(A), _ptr(b), _ptr(C), _ptr(S), _ptr(v),
                                           _ptr(xS), _ptr(x))
        if rc != 0:
            raise ArithmeticError("oracle: I + C S is singular")
        return x


def neutral(n: int):
    """The neutral element (I, 0, 0, 0, 0) of eq. lqt_comb: e (x) a = a (x) e = a."""
    return np.eye(n), np.zeros(n), np.zeros((n, n)), np.zeros(n), np.zeros((n, n))


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


_default = None


def riccati(prob, keep_kv_kc: bool = True) -> dict:
    return default().riccati(prob, keep_kv_kc)


def element(prob, k: int):
    return default().element(prob, k)


def combine(e1, e2):
    return default().combine(e1, e2)


def affine_combine(f1, f2):
    return default().affine_combine(f1, f2)


def method2_state(fwd_elem, S, v, xS):
    return default().method2_state(fwd_elem, S, v, xS)
