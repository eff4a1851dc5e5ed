"""Benchmark: LQT time-steps/s of the temporally parallel solve on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one "step" = one full solve, Sec. V-A: elements, backward scan,
gains, forward scan, x* and u*): the 2-D constant-velocity vehicle tracking
problem, nx = 4, nu = 2, T = 10^6, FP32 with mixed-precision refinement
(the path that meets the 1e-5 error bound on every output).  Inputs are
resident in HBM; L2 is flushed (256 MiB write) before every timed step.
Prints one JSON line (rank 0).  N > 1 (torchrun) runs one independent
problem per GPU (weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle (sequential Riccati) on the
host cores for the same metric; it is a deliberately slow baseline.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2104_03186_gb300 import accuracy  # noqa: E402  (numpy only: error measures)

METRIC = "LQT steps/s: parallel scan vs sequential Riccati, 1 GB300, ≤1e-5 err; p99 ms"
UNIT = "time-steps/s"
T_HEADLINE = 1_000_000
SWEEP_T = (100, 1000, 10_000, 100_000, 1_000_000)
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (4 SMSPs x 32)

# Algorithmic work per time step of the k_bwd_down kernel (first pass), the
# kernel with the largest share of the solve: one Riccati step with gains,
# the closed-loop chunk map, reading r_k and writing S_k, v_k, K_k.
# Flops for n = 4, m = 2, p = 2 counted from the kernel's arithmetic.
BWD_DOWN_BYTES_PER_STEP = {"in_r": 2 * 4, "out_S": 16 * 4, "out_v": 4 * 4, "out_K": 8 * 4}
BWD_DOWN_FLOPS_PER_STEP = 2 * (32 + 12 + 64 + 32 + 40 + 6 + 24 + 32 + 8 + 8 + 16 + 8 + 64 + 16)


def workload_config(T):
    return {
        "workload": "2-D constant-velocity vehicle tracking, nx=4, nu=2, p=2, T=%d, single "
                    "problem per GPU" % T,
        "model": "F=[[I,0.1I],[0,I]], L=[[0.005I],[0.1I]], c=0, H=[I 0], X_k=I, U_k=0.1I, "
                 "X_T=100I; r_k=(sin 0.01k, cos 0.013k)+N(0,0.01^2), x0~N(0,I)",
        "T": T, "nx": 4, "nu": 2,
        "precision": "fp32 scan + mixed-precision refinement (shifted re-solve)",
        "l2": "flushed before every timed step (256 MiB write)",
        "inputs": "device-resident",
        "launch": "one solve captured once in a CUDA graph, replayed each step",
    }


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# --------------------------------------------------------------------------
# host-side helpers (covered by CPU tests)
# --------------------------------------------------------------------------

def max_over_ranks(value: float, world: int) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Host threads of the end-to-end measurement.  lqt_solve_host returns when its
# outputs are in host memory, so one caller leaves the host link idle while
# its kernels run; a second caller's copies fill that time (the link carries
# both directions at once).
E2E_THREADS = 2


def e2e_concurrent(prob, opts, steps: int) -> float:
    """Wall seconds for E2E_THREADS host threads to run `steps` lqt_solve_host
    calls each (own stream, device buffer and pinned host buffers per thread),
    every call copying its inputs in and its outputs back."""
    import threading

    import torch

    from paper_2104_03186_gb300 import lqt

    dev = torch.cuda.current_device()
    ctx = []
    for _ in range(E2E_THREADS):
        Ph = lqt.Problem.from_inputs(prob, dtype=np.float32, pin=True)
        out_h = Ph.allocate_outputs(pin=True)
        buf = torch.empty(lqt.lqt_host_solve_bytes(Ph, opts), dtype=torch.uint8, device="cuda")
        ctx.append((Ph, out_h, buf, torch.cuda.Stream()))
    start = threading.Barrier(E2E_THREADS + 1)
    ends = [0.0] * E2E_THREADS
    errs = []

    def work(i):
        try:
            torch.cuda.set_device(dev)
            Ph, out_h, buf, s = ctx[i]
            lqt.lqt_solve_host(Ph, out_h, buf, s, opts)  # warm-up
            start.wait()
            for _ in range(steps):
                st = lqt.lqt_solve_host(Ph, out_h, buf, s, opts)
                if st != lqt.LQT_OK:
                    raise lqt.LQTError(st, "host solve")
            ends[i] = time.perf_counter()
        except BaseException as e:  # reported after the join
            errs.append(e)
            start.abort()

    threads = [threading.Thread(target=work, args=(i,)) for i in range(E2E_THREADS)]
    for t in threads:
        t.start()
    try:
        start.wait()
    except threading.BrokenBarrierError:
        pass
    t0 = time.perf_counter()
    for t in threads:
        t.join()
    if errs:
        raise errs[0]
    del ctx
    return max(ends) - t0


def secondary(name: str, fn):
    """Run one secondary measurement (no collectives inside).  An exception is
    reported in its place, so that the headline line is still printed."""
    try:
        return fn()
    except Exception as e:
        sys.stderr.write("bench: %s failed: %r\n" % (name, e))
        return {"error": "%s failed: %r" % (name, e)}


def throughput(total_units: float, seconds: float) -> float:
    return total_units / seconds if seconds > 0 else float("nan")


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


def parse_clocks(csv_text: str):
    """Median SM clock under load, max SM clock and active throttle reasons from
    `nvidia-smi --query-gpu=index,clocks.sm,clocks.max.sm,power.draw,
    clocks_event_reasons.active,...hw_slowdown,...hw_thermal_slowdown,
    ...sw_thermal_slowdown,...sw_power_cap --format=csv` samples."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in csv_text.strip().splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9 or not parts[1].split()[0].replace(".", "").isdigit():
            continue
        try:
            sm.append(float(parts[1].split()[0]))
            smax.append(float(parts[2].split()[0]))
        except ValueError:
            continue
        for name, flag in zip(names, parts[5:9]):
            if flag.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return None
    loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
    return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": float(max(smax)),
            "reasons": sorted(reasons), "samples": len(sm)}


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="lqt_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def result(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        with open(self.path) as f:
            text = f.read()
        os.unlink(self.path)
        return parse_clocks(text)


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on host cores
# --------------------------------------------------------------------------

def oracle_throughput(T: int, min_seconds: float, max_reps: int = 50):
    """Time the FP64 oracle (sequential Riccati + forward pass, one core) on the
    vehicle workload; returns (steps/s, reps, seconds, sample description)."""
    import oracle
    from paper_2104_03186_gb300 import inputs

    prob = inputs.vehicle(T, seed=0).rounded_to(np.float32)
    oracle.riccati(prob, keep_kv_kc=False)  # build/load outside the timing
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.riccati(prob, keep_kv_kc=False)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    return T * reps / el, reps, el, "vehicle T=%d, %d full solves (%.1f s), 1 thread" % (
        T, reps, el)


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def run_reference(args):
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    import oracle
    from paper_2104_03186_gb300 import inputs

    T = T_HEADLINE
    prob = inputs.vehicle(T, seed=0).rounded_to(np.float32)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.riccati(prob, keep_kv_kc=False)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = throughput(T * len(times), total)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / max(len(times), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(T),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "vehicle T=%d, one full FP64 solve per step, 1 thread, %s" % (
                             T, cpu_model())},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p99_ms": 1e3 * percentile(times, 99), "p50_ms": 1e3 * percentile(times, 50),
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def solve_graph(launch):
    """Capture one solve, launch(stream), in a CUDA graph on a side stream;
    returns (replay, graph): replay() launches the same kernels on the current
    stream.  The solve must have run once before (its one-time set-up is not
    capturable)."""
    import torch

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        launch(s)
    torch.cuda.current_stream().wait_stream(s)
    return g.replay, g


def graph_timed(launch, reps, flush, stream):
    """Device times (ms) of one call, launch(s), captured once in a CUDA graph and
    replayed (the headline's method; the host launch work stays out of the
    timed region), or of eager calls on `stream` if the call cannot be
    captured.  The call must have run once before.  `stream` must be the
    current stream: a graph replays there, and the events are recorded on
    `stream`.  Returns (times, how)."""
    import torch

    try:
        replay, graph = solve_graph(launch)
    except Exception:  # not capturable: time the eager calls instead
        torch.cuda.synchronize()
        return _time_solves(lambda: launch(stream), reps, flush, stream), "eager calls"
    replay()
    times = _time_solves(replay, reps, flush, stream)
    del graph
    return times, "CUDA graph replay"


def _time_solves(fn, reps, flush, stream):
    """Per-call device time (ms) with CUDA events on `stream`, L2 flushed before each."""
    import torch

    out = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def run_ours(args):
    import torch

    rank, local_rank, world = _env_rank()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2104_03186_gb300 import inputs, lqt

    T = T_HEADLINE
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    prob = inputs.vehicle(T, seed=rank).rounded_to(np.float32)
    P = lqt.Problem.from_inputs(prob, dtype=np.float32)
    out = P.allocate_outputs()
    opts = lqt.LQT_REFINE_ON
    ws = lqt.workspace_for(P, opts=opts)
    plan = lqt.lqt_plan(P, opts)

    def launch(s):
        lqt.lqt_solve(P, out, ws, s, opts)

    # the timed step replays one solve captured in a CUDA graph (the same ten
    # kernels, launched by the graph instead of one host call each)
    launch(stream)
    torch.cuda.synchronize()
    step, _graph = solve_graph(launch)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = lqt.lqt_workspace_status(ws, stream)
    if st != lqt.LQT_OK:
        raise lqt.LQTError(st, "warm-up solve")

    compute_peaks = measured_compute_peaks()

    # accuracy of this exact configuration against the FP64 oracle (untimed)
    errors = None
    cpu = None
    if rank == 0:
        import oracle

        t0 = time.perf_counter()
        ref = oracle.riccati(prob, keep_kv_kc=False)
        oracle_s = time.perf_counter() - t0
        got = {k: v.double().cpu().numpy() for k, v in out.items()}
        errors = accuracy.errors(got, ref)
        del got

    # ---- timed region: K solves, one event pair per solve ---------------------
    kern = {}
    times = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.__enter__()  # sampled through the timed steps, the T sweep and the batch
    for _ in range(args.steps):
        times += _time_solves(step, 1, flush, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    # ---- the same K solves with an event pair around every kernel (the
    # library's per-kernel events on the launching stream); kept out of the
    # headline loop because the extra event records lengthen a solve by ~5% ----
    lqt.lqt_profile_enable(True)
    for _ in range(args.steps):
        _time_solves(lambda: launch(stream), 1, flush, stream)
        for i, (name, ms) in enumerate(lqt.lqt_profile_read()):
            kern.setdefault((i, name), []).append(ms)
    lqt.lqt_profile_enable(False)
    st = lqt.lqt_workspace_status(ws, stream)
    if st != lqt.LQT_OK:
        raise lqt.LQTError(st, "timed solve")
    total_s = max_over_ranks(sum(times) / 1e3, world)
    value = throughput(world * T * args.steps, total_s)

    # ---- end to end through the host-buffer entry point ---------------------
    Ph = lqt.Problem.from_inputs(prob, dtype=np.float32, pin=True)
    out_h = Ph.allocate_outputs(pin=True)
    dev_buf = torch.empty(lqt.lqt_host_solve_bytes(Ph, opts), dtype=torch.uint8, device="cuda")
    h2d = sum(int(t.numel() * t.element_size()) for t in Ph.arrays.values())
    d2h = sum(int(t.numel() * t.element_size()) for t in out_h.values())
    lqt.lqt_solve_host(Ph, out_h, dev_buf, stream, opts)
    e2e_steps = max(3, min(args.steps, 10))
    e2e_times = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stt = lqt.lqt_solve_host(Ph, out_h, dev_buf, stream, opts)
        e2e_times.append(time.perf_counter() - t0)
        if stt != lqt.LQT_OK:
            raise lqt.LQTError(stt, "host solve")
    e2e_single_s = max_over_ranks(float(np.median(e2e_times)), world)
    del dev_buf, out_h, Ph
    e2e_threads, e2e_note = E2E_THREADS, None
    try:
        e2e_wall = e2e_concurrent(prob, opts, e2e_steps)
    except Exception as e:  # keep the line: fall back to the single-thread figure
        e2e_threads, e2e_note = 1, "concurrent measurement failed: %r" % (e,)
        e2e_wall = e2e_single_s * e2e_steps
    e2e_s = max_over_ranks(e2e_wall, world) / (e2e_threads * e2e_steps)  # per solve

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    # ---- per-kernel times and the roofline of the dominant kernel ---------
    # launch order: pass 1 (5 kernels), then pass 2 (the same five, ".refine")
    per_kernel = {name: float(np.mean(v)) for (i, name), v in sorted(kern.items())}
    dom = max(per_kernel, key=per_kernel.get)
    bwd_ms = per_kernel["bwd_down"]
    alg_bytes = sum(BWD_DOWN_BYTES_PER_STEP.values()) * T
    alg_flops = BWD_DOWN_FLOPS_PER_STEP * T
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    if compute_peaks["fp32_tflops"] > 0:
        fp32_peak = compute_peaks["fp32_tflops"]
        fp32_src = "measured (FMA microbenchmark, this run)"
    else:
        fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) \
            * 1e6 / 1e12
        fp32_src = "derived: SMs x 128 FP32 lanes x 2 x max SM clock"
    hbm_time = alg_bytes / (hbm_peak * 1e9)
    alu_time = alg_flops / (fp32_peak * 1e12)
    hbm_ach = alg_bytes / (bwd_ms * 1e-3) / 1e9
    alu_ach = alg_flops / (bwd_ms * 1e-3) / 1e12
    hbm_roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_ach / hbm_peak,
                "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)"}
    alu_roof = {"bound": "alu", "achieved": alu_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": alu_ach / fp32_peak, "peak_source": fp32_src}
    # the roof with the longer ideal time binds; the other is reported beside it
    roof, other = (hbm_roof, alu_roof) if hbm_time >= alu_time else (alu_roof, hbm_roof)
    roof = dict(roof)
    roof["other_roof"] = other
    roof.update({
        "kernel": "k_bwd_down (first pass)",
        "algorithmic_bytes_per_launch": alg_bytes,
        "algorithmic_flops_per_launch": alg_flops,
        "per_unit": "per time step: %d B (r in; S, v, K out), %d flop" % (
            sum(BWD_DOWN_BYTES_PER_STEP.values()), BWD_DOWN_FLOPS_PER_STEP),
        "launch_ms": bwd_ms,
        "traffic": TRAFFIC_BWD_DOWN,
        "dominant_kernel_by_time": dom,
    })

    # ---- T sweep: parallel vs sequential Riccati on this GPU ---------------
    sweep = []

    def run_sweep():
        for Ts in SWEEP_T:
            ps = inputs.vehicle(Ts, seed=0).rounded_to(np.float32)
            Pq = lqt.Problem.from_inputs(ps, dtype=np.float32)
            o2 = Pq.allocate_outputs()
            w2 = lqt.workspace_for(Pq, opts=opts)
            lqt.lqt_solve(Pq, o2, w2, stream, opts)
            torch.cuda.synchronize()
            par, graph = solve_graph(lambda s: lqt.lqt_solve(Pq, o2, w2, s, opts))
            seq = lambda: lqt.lqt_riccati_sequential(Pq, o2, w2, stream, opts)  # noqa: E731
            # 20 warm-ups; 200 timed replays below T = 1e6, 20 at 1e6
            for _ in range(20):
                par()
            tp = _time_solves(par, 200 if Ts < T_HEADLINE else 20, flush, stream)
            seq()
            ts = _time_solves(seq, 3 if Ts <= 100_000 else 1, flush, stream)
            sweep.append({"T": Ts, "reps": len(tp),
                          "parallel_steps_per_s": Ts / (np.median(tp) * 1e-3),
                          "parallel_p50_ms": percentile(tp, 50), "parallel_p99_ms": percentile(tp, 99),
                          "sequential_steps_per_s": Ts / (np.median(ts) * 1e-3),
                          "sequential_ms": float(np.median(ts)),
                          "speedup": float(np.median(ts) / np.median(tp))})
            del o2, w2, Pq, graph, par

    if not args.no_sweep:
        err = secondary("sweep", run_sweep)
        if err is not None:
            sweep.append(err)

    # ---- ragged batch: 4096 problems, one persistent launch per (n, m) ----
    batch = None if args.no_batch else secondary("batch", lambda: run_batch(args, stream, flush))

    # ---- serving: Poisson request streams through the continuous batcher ----
    serving = None if args.no_serve else secondary("serving", lambda: run_serving(args))

    # ---- precision study (n = 32) -------------------------------------------
    precision = None if args.no_precision else secondary("precision study", lambda: run_precision(
        args, stream, flush, compute_peaks["fp32_tflops"], compute_peaks["fp64_tflops"]))

    # ---- generalised stage cost (cross weights, control offsets) -------------
    cross = None if args.no_cross else secondary("cross", lambda: run_cross(args, stream, flush))

    # ---- partial condensing of the headline workload ----------------------
    condensed = None
    if not args.no_condensed:
        condensed = secondary("condensed", lambda: run_condensed(
            args, stream, flush, prob, ref, float(np.median(times))))
    del ref

    # ---- iterated nonlinear LQT (unicycle) ----------------------------------
    nonlinear = None if args.no_nonlinear else secondary(
        "nonlinear", lambda: run_nonlinear(args, stream, flush))

    clk.__exit__(None, None, None)
    clocks = clk.result()

    # ---- CPU baseline (oracle on the host) ---------------------------------
    cpu_v, reps, el, sample = oracle_throughput(T, 10.0, max_reps=20)
    cpu = {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": sample + ", " + cpu_model()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "p50_ms": percentile(times, 50), "p99_ms": percentile(times, 99),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(T),
        "error_vs_fp64_oracle": errors,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": world * T / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms": 1e3 * e2e_s,
                "entry_point": "lqt_solve_host (pinned host buffers, copies inside)",
                "host_threads": e2e_threads,
                "timing": e2e_note or (
                    "%d host threads, each with its own stream, device buffer and pinned "
                    "buffers, %d solves each; every solve copies its inputs in and all "
                    "outputs back; value = all solves' steps / wall time" %
                    (e2e_threads, e2e_steps)),
                "single_thread_ms": 1e3 * e2e_single_s,
                "single_thread_value": world * T / e2e_single_s},
        "clocks": clocks,
        "measured_compute_peaks": compute_peaks,
        "gpu_launches": plan["kernels"] * args.steps,
        "kernels_ms": per_kernel,
        "plan": plan,
        "sweep": sweep,
        "batch": batch,
        "serving": serving,
        "precision_study": precision,
        "cross": cross,
        "nonlinear": nonlinear,
        "condensed": condensed,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def gen_batch(count: int, seed: int):
    """The ragged batch of inputs.ragged_batch, drawn on a thread pool (numpy's
    LAPACK eigenvalue loops release the GIL), rounded to FP32."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_2104_03186_gb300 import inputs

    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray((4, 8, 16)), size=count)
    Ts = rng.integers(64, 4096 + 1, size=count)

    def one(i):
        return inputs.diag_tracking(int(ns[i]), T=int(Ts[i]),
                                    seed=int(seed) * 1_000_003 + i).astype(np.float32)

    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(count)))


def run_batch(args, stream, flush):
    """Ragged batch (4096 problems, n in {4, 8, 16}, m = n/2, T in U[64, 4096],
    time-varying F_k, L_k, X_k): total time-steps/s of lqt_solve_batched, with
    the FP64 oracle on sampled problems."""
    import torch

    import oracle
    from paper_2104_03186_gb300 import lqt

    t0 = time.perf_counter()
    probs = gen_batch(args.batch_count, 7)
    gen_s = time.perf_counter() - t0
    Ps = [lqt.Problem.from_inputs(p, dtype=np.float32) for p in probs]
    outs = [P.allocate_outputs() for P in Ps]
    ws = torch.empty(lqt.lqt_batch_workspace_bytes(Ps, outs), dtype=torch.uint8, device="cuda")
    steps = sum(p.T for p in probs)

    def run():
        lqt.lqt_solve_batched(Ps, outs, ws, stream)

    for _ in range(2):
        run()
    torch.cuda.synchronize()
    # eager calls: the host builds and uploads 4096 descriptors and launches
    # about 200 kernels inside the timed region
    eager = _time_solves(run, 3, flush, stream)
    # the timed batch: captured once in a CUDA graph, replayed each step
    replay, graph = solve_graph(lambda s: lqt.lqt_solve_batched(Ps, outs, ws, s))
    for _ in range(2):
        replay()
    times = _time_solves(replay, 5, flush, stream)
    st = lqt.lqt_workspace_status(ws, stream)
    del graph
    med = float(np.median(times))
    # accuracy on sampled problems of each size
    errs = {}
    rng = np.random.default_rng(0)
    for n in (4, 8, 16):
        idx = [i for i, p in enumerate(probs) if p.n == n]
        for i in rng.choice(idx, size=min(2, len(idx)), replace=False):
            pr = probs[int(i)].astype(np.float64)
            ref = oracle.riccati(pr, keep_kv_kc=False)
            got = {k: v.double().cpu().numpy() for k, v in outs[int(i)].items()}
            for k, v in accuracy.errors(got, ref).items():
                w = errs.setdefault(k, {"fro": 0.0, "step_max": 0.0})
                w["fro"] = max(w["fro"], v["fro"])
                w["step_max"] = max(w["step_max"], v["step_max"])
    by_n = {int(n): int(sum(p.T for p in probs if p.n == n)) for n in (4, 8, 16)}
    return {"workload": "%d problems, n in {4,8,16} uniform, m=n/2, T uniform in [64,4096], "
                        "time-varying F_k (I+0.05N(0,1), spectral radius <= 1.05), L_k~N(0,1/n), "
                        "X_k=diag(U[0.5,2]), U=0.1I, r_k~N(0,1), H=I; FP32, no refinement"
                        % len(probs),
            "launch": "one lqt_solve_batched call captured once in a CUDA graph, replayed each "
                      "step; eager_ms: the same call from the host, descriptor building, "
                      "upload and launches included",
            "time_steps": int(steps), "steps_by_n": by_n,
            "value": steps / (med * 1e-3), "unit": UNIT, "ms_p50": med,
            "ms_p99": percentile(times, 99), "eager_ms": float(np.median(eager)),
            "status": int(st),
            "max_error_vs_fp64_oracle_sampled": errs,
            "generation_s": gen_s}


def run_serving(args):
    """20000-request Poisson streams at 2k..50k requests/s: n in {4,8,16,32},
    m = n/2, T log-uniform in [32, 2048], 30% warm starts (receding horizon
    from the previous request's device-resident state), admission by a device
    memory budget of 8 GiB, up to 8 batches of at most 256 requests in
    flight."""
    from paper_2104_03186_gb300 import serve

    pool = serve.ModelPool((4, 8, 16, 32), steps=4096, seed=11)
    warm = serve.make_requests(200, rate=20000.0, seed=99)
    serve.Server(pool, memory_budget=8 << 30).run(warm)  # warm-up
    out = []
    for rate in (2000, 5000, 10000, 20000, 50000):
        for reuse in ((True, False) if rate >= 20000 else (True,)):
            reqs = serve.make_requests(args.serve_requests, rate=float(rate), seed=rate)
            _, summ = serve.Server(pool, memory_budget=8 << 30, streams=8, max_batch=256,
                                   reuse_warm=reuse).run(reqs)
            summ["arrival_rate_per_s"] = rate
            summ["reuse_warm"] = reuse
            summ["time_steps_per_s"] = summ["time_steps"] / (args.serve_requests / rate) \
                if summ["solves_per_s"] >= rate * 0.98 else None
            out.append(summ)
    return {"workload": "Poisson stream of %d LQT requests per rate; n in {4,8,16,32}, m=n/2, "
                        "T log-uniform in [32,2048], time-varying device-resident models "
                        "(diag tracking), fresh reference and x0 per request, 30%% warm starts "
                        "with shifted horizon; 8 GiB admission budget; up to 8 batches of at "
                        "most 256 requests in flight; FP32; reuse_warm: warm "
                        "requests solved from the S, K of the request that computed them "
                        "(lqt_solve_warm), else in full" % args.serve_requests,
            "rates": out, "warm_vs_cold_solve": run_warm_vs_cold()}


def run_warm_vs_cold():
    """Device time of one warm solve (S, K known: lqt_solve_warm) against a full
    solve of the same problem (lqt_solve_batched with one item, the path the
    server takes for cold requests), per state size, on a horizon of 2048
    steps shifted by 256 from a 2304-step model."""
    import torch

    from paper_2104_03186_gb300 import inputs, lqt

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    res = []
    for n in (4, 8, 16, 32):
        prob = inputs.diag_tracking(n, T=2304, seed=n).astype(np.float32)
        Pp = lqt.Problem.from_inputs(prob)
        prior = lqt.solve_batched([Pp])[0]
        warm = inputs.diag_tracking(n, T=2304, seed=n).astype(np.float32)
        for f in ("F", "L", "X", "r"):
            setattr(warm, f, np.ascontiguousarray(getattr(warm, f)[256:]))
        warm.T = 2048
        P = lqt.Problem.from_inputs(warm)
        cold_out = P.allocate_outputs()
        ws_c = torch.empty(lqt.lqt_batch_workspace_bytes([P], [cold_out]), dtype=torch.uint8,
                           device="cuda")
        wo = P.allocate_outputs()
        wo["S"], wo["K"] = prior["S"][256:].contiguous(), prior["K"][256:].contiguous()
        ws_w = torch.empty(lqt.lqt_warm_workspace_bytes([P], [wo]), dtype=torch.uint8,
                           device="cuda")
        cold = lambda: lqt.lqt_solve_batched([P], [cold_out], ws_c, stream)  # noqa: E731
        hot = lambda: lqt.lqt_solve_warm([P], [wo], ws_w, stream)  # noqa: E731
        for f in (cold, hot):
            for _ in range(3):
                f()
        tc = _time_solves(cold, 20, flush, stream)
        tw = _time_solves(hot, 20, flush, stream)
        err = {k: accuracy.rel_fro(wo[k].double().cpu().numpy(),
                                   cold_out[k].double().cpu().numpy()) for k in ("v", "x", "u")}
        res.append({"n": n, "T": 2048, "full_solve_ms": float(np.median(tc)),
                    "warm_solve_ms": float(np.median(tw)),
                    "speedup": float(np.median(tc) / np.median(tw)),
                    "warm_vs_full_rel_error": err})
    return res


def measured_compute_peaks():
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s), from the
    microbenchmark library built beside the solver (independent FMA chains on
    every SM, CUDA-event timed; best of a few runs)."""
    import ctypes

    path = os.path.join(ROOT, "paper_2104_03186_gb300", "libpeaks_gb300.so")
    lib = ctypes.CDLL(path)
    for f in ("peaks_fp32_tflops", "peaks_fp64_tflops"):
        getattr(lib, f).restype = ctypes.c_double
        getattr(lib, f).argtypes = [ctypes.c_int]
    fp32 = max(lib.peaks_fp32_tflops(20000) for _ in range(3))
    fp64 = max(lib.peaks_fp64_tflops(2000) for _ in range(2))
    return {"fp32_tflops": fp32, "fp64_tflops": fp64,
            "how": "independent FMA chains (8 per thread, 256 threads x 8 CTAs per SM), "
                   "2 flop per FMA, CUDA events, best of 3 (FP32) / 2 (FP64)"}


def chain_flops_per_step(n: int, m: int, p: int) -> dict:
    """Algorithmic flops per time step of the chunked lane-group pipeline,
    counted from its arithmetic (multiply-add = 2 flops): the step model
    (X H, H^T X H, H^T X r), the low-rank fold of the step into the chunk total
    (fold_step), the Riccati step with gains and the chunk map (re-fold), and
    the rollout."""
    nr = 2 * n + 1
    model = 2 * (p * p * n + p * n * n + p * p + p * n)
    fold = 2 * (2 * n * n * n + 2 * n * n * m + 2 * n * n          # J2 F, J2 L, w; A2 F, A2 L, A2 c
                + m * n * m + m * n * n + m * n + n * n * n      # G, Z, L^T w; F^T J2 F
                + m * m * (m + nr)                               # Gauss-Jordan on [G | rhs]
                + n * m * n + n * m + n * m * n + m * n * n + m * n + n * n)  # A, b, C, J, eta
    riccati = 2 * (n * n * m + n * n * n + n * n + m * n * m + m * n * n + m * n
                   + m * m * (m + n + 1) + 2 * n * m * n + n * m + n * n * n + n * n)
    chunk_map = 2 * (n * n * n + n * n)
    roll = 2 * (m * n + n * n + n * m)
    return {"model": 2 * model, "fold": fold, "riccati": riccati, "chunk_map": chunk_map,
            "rollout": roll, "total": 2 * model + fold + riccati + chunk_map + roll}


def run_precision(args, stream, flush, fp32_peak=None, fp64_peak=None):
    """Precision study (n = 32, m = 16, p = 32, cond(X_k) = 1e6, U = 1e-3 I,
    F_k = 0.99 Haar + rank-2): errors of S, v, K, x*, u* against the FP64
    oracle for the plain FP32 scan, FP32 with FP64 tree levels and one
    refinement pass, the FP64 scan and the sequential Riccati recursion on the
    GPU, with their device times.  All forms solve the same FP32-representable
    inputs."""
    import oracle
    from paper_2104_03186_gb300 import inputs, lqt

    T = args.precision_T
    t0 = time.perf_counter()
    prob = inputs.precision_study(T=T, seed=0).rounded_to(np.float32)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ref = oracle.riccati(prob, keep_kv_kc=False)
    oracle_s = time.perf_counter() - t0
    # (name, dtype, refine option, sequential): OFF = plain FP32 scan; ON = one
    # KKT refinement step (x*, u*); FULL = FP64 tree levels + one Newton step of
    # the Riccati recursion (S, v, K) + the KKT step; the FP64 scan; the
    # sequential Riccati recursion on the GPU with the same ON refinement
    forms = [("fp32_scan", np.float32, 0, False),
             ("fp32_kkt_refined", np.float32, 1, False),
             ("fp32_fp64tree_newton_kkt_refined", np.float32, 3, False),
             ("fp64_scan", np.float64, 0, False),
             ("fp32_kkt_refined_method2", np.float32, 1, False),
             ("fp32_sequential_riccati_kkt_refined", np.float32, 1, True)]
    flops = chain_flops_per_step(prob.n, prob.m, prob.p)
    out = {}
    for name, dt, refine, seq in forms:
        P = lqt.Problem.from_inputs(prob, dtype=dt)
        o = P.allocate_outputs()
        if name.endswith("method2"):  # trajectory by Method 2 (forward element scan)
            refine = lqt.options(refine, lqt.LQT_METHOD_2)
        ws = lqt.workspace_for(P, opts=refine)
        launch = (lambda s: lqt.lqt_riccati_sequential(P, o, ws, s, refine)) if seq else \
            (lambda s: lqt.lqt_solve(P, o, ws, s, refine))
        call = lambda: launch(stream)  # noqa: E731
        call()
        reps = 1 if seq else 5
        times, how = graph_timed(launch, reps, flush, stream)
        st = lqt.lqt_workspace_status(ws, stream)
        lqt.lqt_profile_enable(1)
        call()
        kms = {}
        for name_k, ms_k in lqt.lqt_profile_read(32):
            kms[name_k] = kms.get(name_k, 0.0) + ms_k
        lqt.lqt_profile_enable(0)
        got = {k: v.double().cpu().numpy() for k, v in o.items()}
        errs = accuracy.errors(got, ref)
        med = float(np.median(times))
        e = {"status": int(st), "ms": med, "steps_per_s": T / (med * 1e-3), "timing": how,
             "error_vs_fp64_oracle": errs, "plan": lqt.lqt_plan(P, refine) if not seq else None,
             "kernels_ms": kms}
        if not seq and not refine:
            e["achieved_tflops"] = flops["total"] * T / (med * 1e-3) / 1e12
            if fp32_peak:
                pk = fp32_peak if dt == np.float32 else fp64_peak
                e["frac_of_measured_fma_peak"] = e["achieved_tflops"] / pk
        out[name] = e
        del o, ws, P
    out["fp32_sequential_riccati_kkt_refined"]["speedup_of_refined_scan"] = \
        out["fp32_sequential_riccati_kkt_refined"]["ms"] / out["fp32_kkt_refined"]["ms"]
    return {"workload": "precision study: n=32, m=16, p=32, T=%d; F_k=0.99 Haar + 0.01 rank-2, "
                        "X_k=V diag(10^U[-6,0]) V^T with cond 1e6, L_k~N(0,1/n), U=1e-3 I, "
                        "H=I, c=0, r_k~N(0,1); inputs rounded to FP32" % T,
            "forms": out, "flops_per_step": flops, "generation_s": gen_s,
            "oracle_s": oracle_s}


def run_cross(args, stream, flush):
    """Generalised stage cost (Sec. IV-D) on the vehicle workload at T = 1e6:
    cross weights M_k = 0.5 X^{1/2} G_k U^{1/2} and offsets s_k ~ N(0, 1)
    (time-varying).  lqt_solve_cross (transform kernel, the refined solve of the
    transformed problem, post kernel) against the same solve of the plain
    problem, and its errors against the FP64 oracle."""
    from oracle import cross as ocross
    from paper_2104_03186_gb300 import inputs, lqt

    T = T_HEADLINE
    prob = inputs.vehicle(T, seed=0)
    ct = inputs.cross_terms(prob, seed=1, scale=0.5)
    prob, ct = prob.rounded_to(np.float32), ct.rounded_to(np.float32)
    opts = lqt.LQT_REFINE_ON
    P = lqt.Problem.from_inputs(prob, dtype=np.float32)
    C = lqt.Cross.from_inputs(ct, dtype=np.float32)
    o = P.allocate_outputs()
    ws = torch_empty_bytes(lqt.lqt_cross_workspace_bytes(P, C, opts))
    launch = lambda s: lqt.lqt_solve_cross(P, C, o, ws, s, opts)  # noqa: E731
    for _ in range(3):
        launch(stream)
    times, how = graph_timed(launch, 10, flush, stream)
    st = lqt.lqt_workspace_status(ws, stream)
    got = {k: v.double().cpu().numpy() for k, v in o.items()}
    ws_plain = lqt.workspace_for(P, opts=opts)
    plain = lambda s: lqt.lqt_solve(P, o, ws_plain, s, opts)  # noqa: E731
    for _ in range(3):
        plain(stream)
    tplain, _ = graph_timed(plain, 10, flush, stream)
    t0 = time.perf_counter()
    ref = ocross.riccati_cross(prob, ct.M, ct.s)
    oracle_s = time.perf_counter() - t0
    errs = accuracy.errors(got, ref)
    med, medp = float(np.median(times)), float(np.median(tplain))
    return {"workload": "vehicle T=%d with time-varying cross weights M_k (2x2) and control "
                        "offsets s_k; inputs rounded to FP32; refinement ON" % T,
            "status": int(st), "ms": med, "steps_per_s": T / (med * 1e-3), "timing": how,
            "plain_solve_ms": medp, "transform_overhead_ms": med - medp,
            "error_vs_fp64_oracle": errs, "oracle_s": oracle_s}


def run_nonlinear(args, stream, flush):
    """Iterated nonlinear LQT (Sec. IV-D, Sec. VI-E): the unicycle on a stadium
    track at T = 1e5 (about 280 laps), 10 linearise-and-solve passes, FP32
    with refinement ON.  Parallel passes (Method 1, and Method 2) against the
    sequential recursion on the GPU, and errors against the FP64 oracle."""
    from oracle import nonlinear as onl
    from paper_2104_03186_gb300 import inputs, lqt

    T, iters = 100_000, 10
    prob = inputs.unicycle_track(T, seed=0).rounded_to(np.float32)
    P = lqt.Problem.from_inputs(prob, dtype=np.float32)
    o = P.allocate_outputs()
    forms = {"method1": (lqt.LQT_REFINE_ON, False),
             "method2": (lqt.options(lqt.LQT_REFINE_ON, lqt.LQT_METHOD_2), False),
             "sequential": (lqt.LQT_REFINE_ON, True)}
    t0 = time.perf_counter()
    ref = onl.iterated_lqt(onl.Unicycle(0.1), prob, iters)
    oracle_s = time.perf_counter() - t0
    res = {}
    for name, (opts, seq) in forms.items():
        nl = lqt.nonlinear(iters, 0.1, seq)
        ws = torch_empty_bytes(lqt.lqt_nonlinear_workspace_bytes(P, nl, opts))
        launch = lambda s: lqt.lqt_solve_nonlinear(P, nl, o, ws, s, opts)  # noqa: E731
        launch(stream)
        times, how = graph_timed(launch, 1 if seq else 5, flush, stream)
        st = lqt.lqt_workspace_status(ws, stream)
        got = {k: v.double().cpu().numpy() for k, v in o.items()}
        errs = accuracy.errors(got, ref)
        med = float(np.median(times))
        res[name] = {"status": int(st), "ms": med, "steps_per_s": iters * T / (med * 1e-3),
                     "timing": how, "error_vs_fp64_oracle": errs}
        del ws
    for name in ("method1", "method2"):
        res[name]["speedup_vs_sequential"] = res["sequential"]["ms"] / res[name]["ms"]
    return {"workload": "unicycle (n=4, m=2, p=3) on a stadium track, T=%d, %d passes, "
                        "reference points every 10th step; inputs rounded to FP32; "
                        "refinement ON" % (T, iters),
            "forms": res, "oracle_s": oracle_s}


def run_condensed(args, stream, flush, prob, ref, plain_ms):
    """Partial condensing (Sec. V-C) of the vehicle workload: blocks of B steps
    (n = 4, stacked m = 2B, p = 2B, generalised stage cost), solved by
    lqt_solve_condensed (B = 2 as the condensed problem itself, B >= 3 through
    the rank-reduced blocks), beside the plain solve, at T = 1e5 and the
    headline's T = 1e6; the same FP32 inputs and refinement as the headline,
    errors against the FP64 oracle."""
    import oracle
    from paper_2104_03186_gb300 import inputs, lqt

    opts = lqt.LQT_REFINE_ON
    out = []
    for T in (100_000, prob.T):
        pr = prob if T == prob.T else inputs.vehicle(T, seed=0).rounded_to(np.float32)
        rf = ref if T == prob.T else oracle.riccati(pr, keep_kv_kc=False)
        P = lqt.Problem.from_inputs(pr, dtype=np.float32)
        for B in (1, 2, 4, 8, 16):
            o = P.allocate_outputs()
            ws = torch_empty_bytes(lqt.lqt_condensed_workspace_bytes(P, B, opts))
            launch = lambda s: lqt.lqt_solve_condensed(P, B, o, ws, s, opts)  # noqa: E731
            for _ in range(3):
                launch(stream)
            times, how = graph_timed(launch, 10, flush, stream)
            st = lqt.lqt_workspace_status(ws, stream)
            got = {k: v.double().cpu().numpy() for k, v in o.items()}
            med = float(np.median(times))
            out.append({"T": T, "B": B, "status": int(st), "ms": med, "timing": how,
                        "steps_per_s": T / (med * 1e-3),
                        "error_vs_fp64_oracle": accuracy.errors(got, rf)})
            del o, ws, got
        del P
    return {"workload": "vehicle (n=4, m=2, p=2) condensed in blocks of B steps (stacked "
                        "controls 2B, outputs 2B, T/B steps; B >= 3 rank-reduced to 4 controls "
                        "per block); FP32, refinement ON; B = 1 is the plain solve",
            "plain_solve_ms_headline": plain_ms, "sweep": out}


def torch_empty_bytes(nbytes):
    import torch

    if nbytes == 0:
        raise RuntimeError("workspace query returned 0")
    return torch.empty(nbytes, dtype=torch.uint8, device="cuda")


# dram__bytes_read.sum + dram__bytes_write.sum of one k_bwd_down launch
# (first pass, vehicle T = 1e6) from an ncu capture of the current kernel;
# None when the kernel has changed since the counters were taken.
TRAFFIC_BWD_DOWN = 112.59e6


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-sweep", action="store_true", help="skip the T sweep")
    ap.add_argument("--no-batch", action="store_true", help="skip the ragged-batch measurement")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--no-precision", action="store_true", help="skip the n = 32 precision study")
    ap.add_argument("--precision-T", type=int, default=65536)
    ap.add_argument("--no-cross", action="store_true",
                    help="skip the generalised-cost (cross weight) measurement")
    ap.add_argument("--no-condensed", action="store_true",
                    help="skip the partial-condensing measurement")
    ap.add_argument("--no-nonlinear", action="store_true",
                    help="skip the iterated nonlinear LQT (unicycle) measurement")
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="profiling mode: run --warmup + this many solves of --T and exit "
                         "(no JSON line; for ncu captures)")
    ap.add_argument("--T", type=int, default=T_HEADLINE, help="horizon of --profile-solves")
    ap.add_argument("--refine", type=int, default=1, help="refinement in --profile-solves")
    ap.add_argument("--profile-workload",
                    choices=("vehicle", "precision", "cross", "nonlinear", "batch", "condensed"),
                    default="vehicle",
                    help="workload of --profile-solves: the vehicle (n = 4), the n = 32 "
                         "precision study, the vehicle with cross weights and offsets "
                         "(lqt_solve_cross), the unicycle (lqt_solve_nonlinear, 10 passes), or "
                         "the ragged batch (lqt_solve_batched, --batch-count problems), or the "
                         "vehicle condensed in blocks of --block steps (lqt_solve_condensed)")
    ap.add_argument("--block", type=int, default=2, help="block size of the condensed profile")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.profile_solves > 0:
        return run_profile_solves(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


def run_profile_solves(args):
    """A bare loop of solves on the vehicle (or precision-study) workload, for ncu
    captures."""
    import torch

    from paper_2104_03186_gb300 import inputs, lqt

    if args.profile_workload == "batch":
        Ps = [lqt.Problem.from_inputs(p, dtype=np.float32) for p in gen_batch(args.batch_count, 7)]
        outs = [P.allocate_outputs() for P in Ps]
        ws = torch_empty_bytes(lqt.lqt_batch_workspace_bytes(Ps, outs))
        for _ in range(args.warmup + args.profile_solves):
            lqt.lqt_solve_batched(Ps, outs, ws)
        torch.cuda.synchronize()
        st = lqt.lqt_workspace_status(ws)
        print("profile solves done: batch of %d status=%d" % (len(Ps), st))
        return 0 if st == lqt.LQT_OK else 1
    if args.profile_workload == "precision":
        pr = inputs.precision_study(T=args.T, seed=0)
    elif args.profile_workload == "nonlinear":
        pr = inputs.unicycle_track(args.T, seed=0)
    else:
        pr = inputs.vehicle(args.T, seed=0)
    P = lqt.Problem.from_inputs(pr.rounded_to(np.float32))
    out = P.allocate_outputs()
    if args.profile_workload == "cross":
        C = lqt.Cross.from_inputs(inputs.cross_terms(pr, seed=1, scale=0.5).rounded_to(np.float32))
        ws = torch_empty_bytes(lqt.lqt_cross_workspace_bytes(P, C, args.refine))
        call = lambda: lqt.lqt_solve_cross(P, C, out, ws, None, args.refine)  # noqa: E731
    elif args.profile_workload == "condensed":
        ws = torch_empty_bytes(lqt.lqt_condensed_workspace_bytes(P, args.block, args.refine))
        call = lambda: lqt.lqt_solve_condensed(P, args.block, out, ws, None, args.refine)  # noqa: E731
    elif args.profile_workload == "nonlinear":
        nl = lqt.nonlinear(10, 0.1)
        ws = torch_empty_bytes(lqt.lqt_nonlinear_workspace_bytes(P, nl, args.refine))
        call = lambda: lqt.lqt_solve_nonlinear(P, nl, out, ws, None, args.refine)  # noqa: E731
    else:
        ws = lqt.workspace_for(P, opts=args.refine)
        call = lambda: lqt.lqt_solve(P, out, ws, None, args.refine)  # noqa: E731
    for _ in range(args.warmup + args.profile_solves):
        call()
    torch.cuda.synchronize()
    st = lqt.lqt_workspace_status(ws)
    print("profile solves done: %s T=%d refine=%d status=%d" % (
        args.profile_workload, args.T, args.refine, st))
    return 0 if st == lqt.LQT_OK else 1


if __name__ == "__main__":
    sys.exit(main())
