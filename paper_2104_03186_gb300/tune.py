"""Autotuner of the ragged-batch launch plan (lqt_batch_set_tuning).

For the lane-group sizes (n = 8, 16) every problem of a batch is cut into a
power-of-two number of chunks of about B steps, one lane group per chunk
(Sec. V-C block processing); the chunk totals are then scanned over the tree
levels of Alg. 1.  Short chunks give more parallel groups and more tree
levels; long chunks the reverse, and which wins depends on how full the GPU
is.  The tuner times lqt_solve_batched on this GPU on a synthetic batch shaped
like the benchmark's ragged batch (diagonal tracking, m = n / 2), choosing the
chunk length of each (n, T-bucket) in turn with the others fixed, then times
the three launch modes (one launch per tree level, one persistent launch per
size, or the library's automatic choice between them by the number of chunk
waves) with that table on the whole batch and on a small batch of the size a
server forms, and keeps the mode that is fastest on the small batch among
those within 1% of the best on the whole batch.  The library applies a tuned
length only up to the batch's total steps over the resident lane groups, so
the small batches of a server keep their short chunks.

    python -m paper_2104_03186_gb300.tune [--out FILE] [--problems K] [--modes-only]

writes the table as JSON (default: tuned_batch_plans.json beside this file),
which the Python binding applies when it loads the library; --modes-only keeps
the committed chunk lengths and re-times the launch modes alone.  The
selection and file logic below needs no GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, List, Sequence, Tuple

import numpy as np

SIZES = (8, 16)
MODES = ("per_level", "persistent", "auto")  # lqt_batch_set_tuning's launch modes
SMALL_BATCH = 16  # problems in the small batch the launch modes are also timed on
BUCKETS = ((64, 512), (513, 2048), (2049, 4096))  # T ranges (inclusive)
CANDIDATES = (8, 16, 32, 64, 128, 256)
DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_batch_plans.json")


def choose(timings: Dict[Tuple[int, int], Dict[int, float]]) -> List[dict]:
    """Fastest chunk length per (n, bucket upper bound): timings maps
    (n, t_max) -> {chunk_steps: ms}.  Ties go to the longer chunk (fewer tree
    levels).  Entries sorted by n, then t_max, as the library matches them."""
    out = []
    for (n, t_max), per_b in sorted(timings.items()):
        if not per_b:
            continue
        best = min(per_b.items(), key=lambda kv: (kv[1], -kv[0]))[0]
        out.append({"n": int(n), "t_max": int(t_max), "chunk_steps": int(best),
                    "ms": {str(b): float(ms) for b, ms in sorted(per_b.items())}})
    return out


def choose_mode(mix_ms: Dict[str, float], small_ms: Dict[str, float],
                rel: float = 0.01) -> str:
    """The launch mode to keep: among the modes within `rel` of the fastest on
    the whole batch, the fastest on the small batch (ties in MODES order)."""
    best = min(mix_ms.values())
    near = [m for m in MODES if m in mix_ms and mix_ms[m] <= best * (1.0 + rel)]
    return min(near, key=lambda m: (small_ms.get(m, float("inf")), MODES.index(m)))


def plan_mode(plan: dict) -> str:
    """A plan's launch mode; plans written before there were three modes say
    only whether the persistent launch won."""
    if "launch_mode" in plan:
        return plan["launch_mode"]
    return "persistent" if plan.get("persistent", True) else "per_level"


def entries_for(plan: dict) -> List[Tuple[int, int, int]]:
    """(n, t_max, chunk_steps) triples of a plan, in the library's order."""
    return [(e["n"], e["t_max"], e["chunk_steps"])
            for e in sorted(plan["entries"], key=lambda e: (e["n"], e["t_max"]))]


def save(plan: dict, path: str = DEFAULT_OUT) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(plan, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)


def load(path: str = DEFAULT_OUT) -> dict:
    with open(path) as f:
        plan = json.load(f)
    for e in plan["entries"]:
        if not (e["n"] >= 1 and e["t_max"] >= 0 and e["chunk_steps"] >= 1):
            raise ValueError("bad tuning entry %r" % (e,))
    if plan_mode(plan) not in MODES:
        raise ValueError("bad launch mode %r" % (plan_mode(plan),))
    return plan


# ---------------------------------------------------------------------------
# measurement (GPU)
# ---------------------------------------------------------------------------

def _time_batch(Ps, outs, ws, reps: int) -> float:
    import torch

    from . import lqt

    stream = torch.cuda.current_stream()
    for _ in range(2):
        lqt.lqt_solve_batched(Ps, outs, ws, stream)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lqt.lqt_solve_batched(Ps, outs, ws, stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    st = lqt.lqt_workspace_status(ws, stream)
    if st != lqt.LQT_OK:
        raise lqt.LQTError(st, "tuning batch")
    return float(np.median(ts))


def _prepared(probs):
    import torch

    from . import lqt

    Ps = [lqt.Problem.from_inputs(p, dtype=np.float32) for p in probs]
    outs = [P.allocate_outputs() for P in Ps]
    return Ps, outs, torch


def _workspace(Ps, outs):
    import torch

    from . import lqt

    nbytes = lqt.lqt_batch_workspace_bytes(Ps, outs)
    if nbytes == 0:
        raise lqt.LQTError(lqt.LQT_EUNSUPPORTED, "tuning workspace")
    return torch.empty(nbytes, dtype=torch.uint8, device="cuda")


def measure(problems: int = 4096, reps: int = 3, sizes: Sequence[int] = SIZES,
            buckets=BUCKETS, candidates: Sequence[int] = CANDIDATES, seed: int = 11,
            fixed_entries: Sequence[Tuple[int, int, int]] = ()) -> dict:
    """Tune on this GPU and return the plan.  The best chunk length of a
    bucket depends on what else the batch holds (a batch that fills the GPU
    favours longer chunks than a small one), so every candidate is timed on
    the whole mixed batch (the benchmark's distribution, another draw: n
    uniform in {4, 8, 16}, T uniform in [64, 4096]): one pass of coordinate descent over
    the (n, T-bucket) entries from the untuned chunk length (64), then the
    launch modes with the resulting table, on the whole batch and on its first
    SMALL_BATCH problems.  fixed_entries: keep these (n, t_max, chunk_steps)
    and time the launch modes alone."""
    import torch

    from . import inputs, lqt

    from concurrent.futures import ThreadPoolExecutor

    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray((4, 8, 16)), size=problems)
    Ts = rng.integers(64, 4096 + 1, size=problems)

    def one(i):
        return inputs.diag_tracking(int(ns[i]), T=int(Ts[i]),
                                    seed=seed * 1_000_003 + i).astype(np.float32)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        mix = list(ex.map(one, range(problems)))
    Ps, outs, _ = _prepared(mix)
    del mix
    table = {(n, t_hi): 64 for n in sizes for (_, t_hi) in buckets}

    def run(tab, mode="per_level", Ps=Ps, outs=outs):
        lqt.lqt_batch_set_tuning([(n, t, b) for (n, t), b in sorted(tab.items())], mode)
        ws = _workspace(Ps, outs)
        ms = _time_batch(Ps, outs, ws, reps)
        del ws
        return ms

    if fixed_entries:
        table = {(n, t): b for n, t, b in fixed_entries}
        base_ms, entries = None, [{"n": n, "t_max": t, "chunk_steps": b}
                                  for n, t, b in fixed_entries]
    else:
        base_ms = run(table)
        timings: Dict[Tuple[int, int], Dict[int, float]] = {}
        for key in sorted(table):
            per_b = {}
            for b in candidates:
                if b > key[1]:
                    continue
                trial = dict(table)
                trial[key] = b
                per_b[b] = run(trial)
            timings[key] = per_b
            table[key] = min(per_b.items(), key=lambda kv: (kv[1], -kv[0]))[0]
        entries = choose(timings)
    mix_ms = {m: run(table, m) for m in MODES}
    small = slice(0, min(SMALL_BATCH, len(Ps)))
    small_ms = {m: run(table, m, Ps[small], outs[small]) for m in MODES}
    mode = choose_mode(mix_ms, small_ms)
    lqt.lqt_batch_set_tuning([(n, t, b) for (n, t), b in sorted(table.items())], mode)
    return {"entries": entries, "launch_mode": mode, "mix_ms": mix_ms,
            "small_batch_ms": small_ms, "small_batch": SMALL_BATCH,
            "untuned_ms": base_ms, "gpu": torch.cuda.get_device_name(0),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
            "problems": problems, "candidates": list(candidates),
            "buckets": [list(b) for b in buckets]}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--problems", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--modes-only", action="store_true",
                    help="keep the committed chunk lengths, time the launch modes")
    args = ap.parse_args(argv)
    old = load(args.out) if args.modes_only else None
    plan = measure(args.problems, args.reps,
                   fixed_entries=entries_for(old) if old else ())
    if old:
        # the chunk-length timings of the full tuning run stay with their entries
        plan["entries"], plan["untuned_ms"] = old["entries"], old.get("untuned_ms")
        plan["candidates"], plan["buckets"] = old["candidates"], old["buckets"]
    save(plan, args.out)
    print(json.dumps({"out": args.out, "launch_mode": plan["launch_mode"],
                      "entries": [(e["n"], e["t_max"], e["chunk_steps"]) for e in plan["entries"]],
                      "mix_ms": plan["mix_ms"], "small_batch_ms": plan["small_batch_ms"]}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
