"""The C-ABI library loads and exports every entry point include/*.h declares
(CPU only: no compute call is made)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_03186_gb300 import build

    build.build()
    from paper_2104_03186_gb300 import lqt

    return lqt


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lqt_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_api():
    names = _declared_functions()
    for required in ("lqt_solve", "lqt_workspace_bytes", "lqt_workspace_status",
                     "lqt_riccati_sequential", "lqt_solve_host", "lqt_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_strerror_covers_all_codes(lib):
    for code in range(9):
        assert lib.lqt_strerror(code) not in ("", "unknown status")
    assert lib.lqt_strerror(99) == "unknown status"


def _host_problem(lib, **over):
    from paper_2104_03186_gb300 import inputs

    p = inputs.vehicle(16)
    arr = {f: np.ascontiguousarray(getattr(p, f), dtype=np.float32)
           for f in lib.STEP_FIELDS + lib.TERMINAL_FIELDS if getattr(p, f) is not None}
    arr.update(over)
    return lib.Problem(p.n, p.m, p.p, p.pT, p.T, lib.LQT_F32, arr), arr


def test_invalid_arguments_rejected_before_any_device_work(lib):
    so = lib.library()
    P, arr = _host_problem(lib)
    out = {k: np.zeros(s, np.float32) for k, s in
           {"S": (17, 4, 4), "v": (17, 4), "K": (16, 2, 4), "x": (17, 4), "u": (16, 2)}.items()}
    sol = lib.lqt_solution(*[o.ctypes.data for o in out.values()])
    # NULL problem / solution / workspace
    assert so.lqt_solve(None, ctypes.byref(sol), None, None, 0, None) == lib.LQT_EINVAL
    assert so.lqt_solve(ctypes.byref(P.struct), None, None, None, 0, None) == lib.LQT_EINVAL
    assert so.lqt_solve(ctypes.byref(P.struct), ctypes.byref(sol), None, None, 0, None) == lib.LQT_EINVAL
    # bad sizes
    bad = lib.lqt_problem.from_buffer_copy(P.struct)
    bad.n = 0
    assert so.lqt_solve(ctypes.byref(bad), ctypes.byref(sol), None, None, 0, None) == lib.LQT_EINVAL
    bad = lib.lqt_problem.from_buffer_copy(P.struct)
    bad.T = -1
    assert so.lqt_solve(ctypes.byref(bad), ctypes.byref(sol), None, None, 0, None) == lib.LQT_EINVAL
    # a time-varying stride shorter than one step
    bad = lib.lqt_problem.from_buffer_copy(P.struct)
    bad.r.step_stride = 1
    assert so.lqt_solve(ctypes.byref(bad), ctypes.byref(sol), None, None, 0, None) == lib.LQT_EINVAL
    # missing required input
    bad = lib.lqt_problem.from_buffer_copy(P.struct)
    bad.F.ptr = None
    assert so.lqt_solve(ctypes.byref(bad), ctypes.byref(sol), None, None, 0, None) == lib.LQT_EINVAL
    # misaligned output
    sol2 = lib.lqt_solution.from_buffer_copy(sol)
    sol2.S = out["S"].ctypes.data + 4
    assert so.lqt_solve(ctypes.byref(P.struct), ctypes.byref(sol2), None, None, 0, None) == lib.LQT_EINVAL
    # bad options
    opts = lib.options(5)
    fake_ws = ctypes.c_void_p(1 << 20)  # aligned, never dereferenced: options fail first
    assert so.lqt_solve(ctypes.byref(P.struct), ctypes.byref(sol), ctypes.byref(opts), fake_ws,
                        1 << 30, None) == lib.LQT_EINVAL
    opts = lib.options(lib.LQT_REFINE_ON)
    opts.reserved[3] = 1
    assert so.lqt_workspace_bytes(ctypes.byref(P.struct), ctypes.byref(opts)) == 0
    # an unknown trajectory method; Method 2 where no chain variant is compiled
    opts = lib.options(lib.LQT_REFINE_ON, method=7)
    assert so.lqt_solve(ctypes.byref(P.struct), ctypes.byref(sol), ctypes.byref(opts), fake_ws,
                        1 << 30, None) == lib.LQT_EINVAL
    opts = lib.options(lib.LQT_REFINE_ON, method=lib.LQT_METHOD_2)
    small = lib.lqt_problem.from_buffer_copy(P.struct)
    small.n, small.m = 2, 1  # no chain variant at (2, 1): Method 2 is not compiled there
    assert so.lqt_solve(ctypes.byref(small), ctypes.byref(sol), ctypes.byref(opts), fake_ws,
                        1 << 30, None) == lib.LQT_EUNSUPPORTED
    assert so.lqt_workspace_bytes(ctypes.byref(small), ctypes.byref(opts)) == 0
    # unsupported size reports 0 workspace
    bad = lib.lqt_problem.from_buffer_copy(P.struct)
    bad.dtype = 7
    assert so.lqt_workspace_bytes(ctypes.byref(bad), None) == 0


def test_cross_arguments_rejected_before_any_device_work(lib):
    """lqt_solve_cross: NULL or misaligned workspace, a cross weight stride
    shorter than one step, a misaligned offset vector."""
    so = lib.library()
    P, arr = _host_problem(lib)
    out = {k: np.zeros(s, np.float32) for k, s in
           {"S": (17, 4, 4), "v": (17, 4), "K": (16, 2, 4), "x": (17, 4), "u": (16, 2)}.items()}
    sol = lib.lqt_solution(*[o.ctypes.data for o in out.values()])
    M = np.zeros((16, 2, 2), np.float32)
    s = np.zeros((16, 3), np.float32)
    fake_ws = ctypes.c_void_p(1 << 20)
    good = lib.lqt_cross(lib.lqt_in(M.ctypes.data, 4), lib.lqt_in(s.ctypes.data, 3))
    args = (ctypes.byref(P.struct), ctypes.byref(good), ctypes.byref(sol), None)
    assert so.lqt_solve_cross(*args, None, 0, None) == lib.LQT_EINVAL
    assert so.lqt_solve_cross(*args, ctypes.c_void_p((1 << 20) + 8), 1 << 30,
                              None) == lib.LQT_EINVAL
    short = lib.lqt_cross(lib.lqt_in(M.ctypes.data, 3), lib.lqt_in(None, 0))
    assert so.lqt_solve_cross(ctypes.byref(P.struct), ctypes.byref(short), ctypes.byref(sol),
                              None, fake_ws, 1 << 30, None) == lib.LQT_EINVAL
    assert so.lqt_cross_workspace_bytes(ctypes.byref(P.struct), ctypes.byref(short), None) == 0
    skew = lib.lqt_cross(lib.lqt_in(None, 0), lib.lqt_in(s.ctypes.data + 2, 3))
    assert so.lqt_solve_cross(ctypes.byref(P.struct), ctypes.byref(skew), ctypes.byref(sol),
                              None, fake_ws, 1 << 30, None) == lib.LQT_EINVAL
    assert so.lqt_solve_cross(None, ctypes.byref(good), ctypes.byref(sol), None, fake_ws,
                              1 << 30, None) == lib.LQT_EINVAL


def test_nonlinear_arguments_rejected_before_any_device_work(lib):
    """lqt_solve_nonlinear: unknown model, zero passes, a size other than the
    unicycle's, reserved field set, misaligned first nominal."""
    so = lib.library()
    P, arr = _host_problem(lib)
    out = {k: np.zeros(s, np.float32) for k, s in
           {"S": (17, 4, 4), "v": (17, 4), "K": (16, 2, 4), "x": (17, 4), "u": (16, 2)}.items()}
    sol = lib.lqt_solution(*[o.ctypes.data for o in out.values()])
    fake_ws = ctypes.c_void_p(1 << 20)

    def call(nl, prob=P.struct):
        return so.lqt_solve_nonlinear(ctypes.byref(prob), ctypes.byref(nl), ctypes.byref(sol),
                                      None, fake_ws, 1 << 30, None)

    nl = lib.nonlinear(10, 0.1)
    assert so.lqt_solve_nonlinear(ctypes.byref(P.struct), ctypes.byref(nl), ctypes.byref(sol),
                                  None, None, 0, None) == lib.LQT_EINVAL
    bad = lib.nonlinear(10, 0.1, model=7)
    assert call(bad) == lib.LQT_EINVAL
    assert call(lib.nonlinear(0, 0.1)) == lib.LQT_EINVAL
    bad = lib.nonlinear(10, 0.1)
    bad.reserved = 1
    assert call(bad) == lib.LQT_EINVAL
    assert call(lib.nonlinear(10, float("nan"))) == lib.LQT_EINVAL
    bad = lib.nonlinear(10, 0.1)
    bad.x_init = (1 << 20) + 2
    assert call(bad) == lib.LQT_EINVAL
    small = lib.lqt_problem.from_buffer_copy(P.struct)
    small.n, small.m = 2, 1
    assert call(nl, small) == lib.LQT_EINVAL
    assert so.lqt_nonlinear_workspace_bytes(ctypes.byref(small), ctypes.byref(nl), None) == 0


def test_warm_arguments_rejected_before_any_device_work(lib):
    """lqt_solve_warm and its workspace query check every item on the host."""
    assert lib._lib.lqt_warm_workspace_bytes(None, -1) == 0
    items = (lib.lqt_batch_item * 1)()
    p = items[0].problem
    p.n, p.m, p.p, p.pT, p.T, p.dtype = 5, 2, 5, 5, 10, lib.LQT_F32   # no (5, 2) variant
    assert lib._lib.lqt_warm_workspace_bytes(items, 1) == 0
    ws = ctypes.c_void_p(256)  # never dereferenced: the item check fails first
    assert lib._lib.lqt_solve_warm(items, 1, ws, 1 << 20, None) == lib.LQT_EUNSUPPORTED
    p.n, p.m = 8, 4
    p.dtype = 7
    assert lib._lib.lqt_solve_warm(items, 1, ws, 1 << 20, None) == lib.LQT_EINVAL
    p.dtype = lib.LQT_F32
    p.x0 = None  # no initial state
    assert lib._lib.lqt_solve_warm(items, 1, ws, 1 << 20, None) == lib.LQT_EINVAL


def test_single_tile_setting_round_trip(lib):
    """lqt_set_single_tile_chunk needs no device: a negative value is
    rejected, a valid one returns the previous setting."""
    so = lib.library()
    prev = ctypes.c_int32(-7)
    assert so.lqt_set_single_tile_chunk(-1, ctypes.byref(prev)) == lib.LQT_EINVAL
    assert prev.value == -7  # untouched on error
    old = lib.lqt_set_single_tile_chunk(5)
    assert lib.lqt_set_single_tile_chunk(old) == 5
    assert so.lqt_set_single_tile_chunk(old, None) == lib.LQT_OK


def test_batch_launch_modes(lib):
    """lqt_batch_set_tuning needs no device: the three launch modes are
    accepted, any other value is rejected; the committed plan is restored."""
    so = lib.library()
    entry = (lib.lqt_batch_tune_entry * 1)()
    entry[0].n, entry[0].t_max, entry[0].chunk_steps = 8, 512, 16
    try:
        for mode in (lib.LQT_BATCH_PER_LEVEL, lib.LQT_BATCH_PERSISTENT, lib.LQT_BATCH_AUTO):
            assert so.lqt_batch_set_tuning(entry, 1, mode) == lib.LQT_OK
        for bad in (-1, 3, 7):
            assert so.lqt_batch_set_tuning(entry, 1, bad) == lib.LQT_EINVAL
        for name in ("per_level", "persistent", "auto", True, False):
            lib.lqt_batch_set_tuning([(8, 512, 16)], name)
    finally:
        lib.lqt_batch_set_tuning([], "auto")
        lib.apply_tuned_plans()


def test_binding_checks_arrays_before_the_call(lib):
    """The binding rejects what a pointer cannot carry through the C ABI: a
    non-contiguous array, the wrong element type, too few steps, the wrong
    per-step size, too small a terminal or output array."""
    P, arr = _host_problem(lib)
    T = P.T

    def rejected(**over):
        a = dict(arr, **over)
        with pytest.raises(lib.LQTError) as ei:
            lib.Problem(P.n, P.m, P.p, P.pT, T, lib.LQT_F32, a)
        assert ei.value.status == lib.LQT_EINVAL
        return str(ei.value)

    assert "not contiguous" in rejected(r=np.zeros((T, 4), np.float32)[:, ::2])
    assert "element type" in rejected(F=arr["F"].astype(np.float64))
    assert "steps" in rejected(r=np.zeros((T - 1, 2), np.float32))
    assert "elements a step" in rejected(X=np.zeros((T, 3, 3), np.float32))
    assert "x0" in rejected(x0=np.zeros(3, np.float32))
    # one step (stride 0), exactly T steps and more than T steps are all valid
    for r in (np.zeros((1, 2), np.float32), np.zeros((T, 2), np.float32),
              np.zeros((T + 5, 2), np.float32)):
        lib.Problem(P.n, P.m, P.p, P.pT, T, lib.LQT_F32, dict(arr, r=r))
    # outputs: at least the elements the solve writes, the problem's type
    n, m = P.n, P.m
    out = {"S": np.zeros((T + 1, n, n), np.float32), "v": np.zeros((T + 1, n), np.float32),
           "K": np.zeros((T, m, n), np.float32), "x": np.zeros((T + 1, n), np.float32),
           "u": np.zeros((T, m), np.float32)}

    class _Arr(np.ndarray):  # numpy arrays with a torch-style numel()
        def numel(self):
            return self.size

    out = {k: v.view(_Arr) for k, v in out.items()}
    lib.solution_struct(out, P)
    for k, bad in (("K", np.zeros((T - 1, m, n), np.float32)),
                   ("u", np.zeros((T, m), np.float64)),
                   ("S", np.zeros((T + 1, n, 2 * n), np.float32)[:, :, ::2])):
        with pytest.raises(lib.LQTError) as ei:
            lib.solution_struct(dict(out, **{k: bad.view(_Arr)}), P)
        assert ei.value.status == lib.LQT_EINVAL and k in str(ei.value)


def test_binding_checks_cross_arrays(lib):
    P, _ = _host_problem(lib)
    T, p, m = P.T, P.p, P.m
    good = lib.Cross(np.zeros((T, p, m), np.float32), np.zeros((1, m), np.float32))
    assert lib._cross(good, P) is not None
    for M, s, what in ((np.zeros((T, p, m + 1), np.float32), None, "elements a step"),
                       (np.zeros((T - 3, p, m), np.float32), None, "steps"),
                       (None, np.zeros((T, m), np.float64), "element type")):
        with pytest.raises(lib.LQTError) as ei:
            lib._cross(lib.Cross(M, s), P)
        assert ei.value.status == lib.LQT_EINVAL and what in str(ei.value)


def test_binding_checks_the_first_nominal(lib):
    P, _ = _host_problem(lib)
    T, n, m = P.T, P.n, P.m
    lib._check_nominal(P, np.zeros((T + 1, n), np.float32), np.zeros((T, m), np.float32))
    lib._check_nominal(P, None, None)
    for x, u, what in ((np.zeros((T, n), np.float32), None, "x_init"),
                       (None, np.zeros((T, m), np.float64), "u_init"),
                       (np.zeros((T + 1, 2 * n), np.float32)[:, ::2], None, "x_init")):
        with pytest.raises(lib.LQTError) as ei:
            lib._check_nominal(P, x, u)
        assert ei.value.status == lib.LQT_EINVAL and what in str(ei.value)


def test_binding_constants_match_the_header(lib):
    """Every enumerator and #define of include/lqt.h has the same value in the
    binding."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lqt.h")).read(), flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, re.S):
        for name, val in re.findall(r"(LQT_\w+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    for name, expr in re.findall(r"#define[ \t]+(LQT_\w+)[ \t]+(.+)", src):
        if re.fullmatch(r"\(\(size_t\)\s*\d+\s*<<\s*\d+\)", expr.strip()):
            a, b = re.findall(r"\d+", expr)
            consts[name] = int(a) << int(b)
    assert len(consts) >= 20, consts
    for name, val in consts.items():
        assert getattr(lib, name) == val, name


def test_binding_structs_match_the_header(lib, tmp_path):
    """Size and field offsets of every struct of include/lqt.h, from a C program
    compiled against the header, equal those of the binding's ctypes mirrors."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {name: getattr(lib, name) for name in (
        "lqt_in", "lqt_problem", "lqt_solution", "lqt_options", "lqt_batch_item",
        "lqt_batch_tune_entry", "lqt_cross", "lqt_nonlinear")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lqt.h"', "int main(void) {"]
    for name, ct in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in ct._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", exe],
                   check=True, capture_output=True, timeout=120)
    got = {}
    for ln in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for name, ct in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(ct), name
        for f, _ in ct._fields_:
            assert got[(name, f)] == getattr(ct, f).offset, (name, f)
