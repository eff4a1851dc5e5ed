"""Continuous-batching LQT solver service on one GPU.

Requests are MPC-style solves: a horizon T over a model that is resident on
the device (a window into a time-varying model of state size n), plus the
request's own reference trajectory r and initial state x_0.  A "warm" request
continues a previous one: it reuses the previous request's model shifted by s
steps (a receding horizon) and starts from that request's device-resident
predicted state x*_s.

The loop admits arrived requests while their device memory fits the budget,
groups whatever has been admitted into a batch as soon as a stream is free,
and solves the batch with one lqt_solve_batched call (one persistent launch
per state size present).  Batches on different streams run concurrently, so
requests that arrive while others are on the GPU start without waiting for
them.  Per batch the references and initial states go up in one host-to-device
copy and the optimal controls u* come back in one device-to-host copy.
Latency is completion (observed by polling the batch's event) minus arrival.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque
from typing import Dict, List, Optional

import numpy as np

from . import inputs, lqt


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the stream
    n: int
    T: int
    offset: int             # first step of the model window
    warm_of: int = -1       # request this one continues (-1: cold)
    shift: int = 0          # steps the horizon moved for a warm request
    r: Optional[np.ndarray] = None   # (T, p) float32
    x0: Optional[np.ndarray] = None  # (n,) float32 (cold requests)
    # filled by the server
    done: float = math.nan
    u: Optional[np.ndarray] = None
    out: Optional[Dict[str, object]] = None
    refs: int = 0           # warm requests still pointing at this one's outputs


class ModelPool:
    """Device-resident time-varying models, one per state size: F_k, L_k,
    X_k = diag(U[0.5, 2]), U = 0.1 I, H = I, terminal weights (diag_tracking)."""

    def __init__(self, sizes, steps: int, seed: int = 0):
        import torch

        self.models = {}
        for n in sizes:
            pr = inputs.diag_tracking(n, T=steps, seed=seed + n).astype(np.float32)
            dev = {f: torch.from_numpy(getattr(pr, f)).cuda()
                   for f in ("F", "L", "U", "H", "X", "HT", "XT") if getattr(pr, f) is not None}
            self.models[n] = (pr, dev)
        self.steps = steps

    def problem(self, n: int, offset: int, T: int, r_dev, x0_dev, rT_dev):
        """An lqt.Problem over steps [offset, offset + T) of model n, whose
        arrays point into the pool (no copies)."""
        pr, dev = self.models[n]
        m, p = pr.m, pr.p
        s = lqt.lqt_problem()
        s.n, s.m, s.p, s.pT, s.T, s.dtype = n, m, p, pr.pT, T, lqt.LQT_F32
        s.F = lqt.lqt_in(dev["F"].data_ptr() + offset * n * n * 4, n * n)
        s.L = lqt.lqt_in(dev["L"].data_ptr() + offset * n * m * 4, n * m)
        s.U = lqt.lqt_in(dev["U"].data_ptr(), 0)
        s.H = lqt.lqt_in(dev["H"].data_ptr(), 0)
        s.X = lqt.lqt_in(dev["X"].data_ptr() + offset * p * p * 4, p * p)
        s.r = lqt.lqt_in(r_dev, p)
        s.c = lqt.lqt_in(None, 0)
        s.HT, s.XT, s.rT, s.x0 = dev["HT"].data_ptr(), dev["XT"].data_ptr(), rT_dev, x0_dev
        P = lqt.Problem.__new__(lqt.Problem)
        P.n, P.m, P.p, P.pT, P.T, P.dtype, P.arrays, P.struct = n, m, p, pr.pT, T, \
            lqt.LQT_F32, {}, s
        return P


def out_bytes(n: int, m: int, T: int) -> int:
    return 4 * ((T + 1) * n * n + (T + 1) * n + T * m * n + (T + 1) * n + T * m)


def make_requests(count: int, rate: float, seed: int = 0, sizes=(4, 8, 16, 32),
                  t_lo: int = 32, t_hi: int = 2048, warm_frac: float = 0.3,
                  pool_steps: int = 4096) -> List[Request]:
    """A Poisson stream: exponential inter-arrival times at `rate` per second,
    n uniform in `sizes`, T log-uniform in [t_lo, t_hi]; a fraction `warm_frac`
    continues the previous request of the same size with its horizon shifted
    by s ~ U{1 .. T/4}."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs: List[Request] = []
    last: Dict[int, Request] = {}
    for i in range(count):
        n = int(rng.choice(np.asarray(sizes)))
        prev = last.get(n)
        if prev is not None and rng.random() < warm_frac and prev.T >= 8:
            s = int(rng.integers(1, max(2, prev.T // 4) + 1))
            T = prev.T - s
            req = Request(i, float(t[i]), n, T, prev.offset + s, warm_of=prev.rid, shift=s)
        else:
            T = int(round(math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))))
            off = int(rng.integers(0, pool_steps - T + 1))
            req = Request(i, float(t[i]), n, T, off)
            req.x0 = rng.standard_normal(n).astype(np.float32)
        req.r = rng.standard_normal((req.T + 1, n)).astype(np.float32)  # row T is r_T
        reqs.append(req)
        last[n] = req
    return reqs


class Server:
    def __init__(self, pool: ModelPool, memory_budget: int = 4 << 30, streams: int = 4,
                 max_batch: int = 1024):
        import torch

        self.pool = pool
        self.budget = memory_budget
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.max_batch = max_batch
        self.mem = 0
        self.peak_mem = 0

    def _alloc(self, req: Request):
        import torch

        n = req.n
        m = self.pool.models[n][0].m
        T = req.T
        req.out = {"S": torch.empty((T + 1, n, n), device="cuda"),
                   "v": torch.empty((T + 1, n), device="cuda"),
                   "K": torch.empty((T, m, n), device="cuda"),
                   "x": torch.empty((T + 1, n), device="cuda"),
                   "u": torch.empty((T, m), device="cuda")}
        self.mem += out_bytes(n, m, T)
        self.peak_mem = max(self.peak_mem, self.mem)

    def _release(self, req: Request, keep: bool = False):
        """Free a finished request's outputs once no warm request still needs them."""
        if req.out is not None and req.refs == 0 and not math.isnan(req.done) and not keep:
            n = req.n
            self.mem -= out_bytes(n, self.pool.models[n][0].m, req.T)
            req.out = None

    def run(self, reqs: List[Request], realtime: bool = True):
        """Serve the stream; returns per-request latencies (s) and summary."""
        import torch

        byid = {r.rid: r for r in reqs}
        for q in reqs:  # warm requests that will read each request's outputs
            q.refs = 0
        for q in reqs:
            if q.warm_of >= 0:
                byid[q.warm_of].refs += 1
        queue = deque(sorted(reqs, key=lambda r: r.arrival))
        admitted: List[Request] = []
        inflight = []  # (stream, event, batch, host u buffer, device staging)
        free = list(self.streams)
        done = 0
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0 if realtime else math.inf
            # admission by device-memory budget, first come first served
            while queue and queue[0].arrival <= now:
                q = queue[0]
                need = out_bytes(q.n, self.pool.models[q.n][0].m, q.T)
                if self.mem + need > self.budget and (admitted or inflight):
                    break
                if q.warm_of >= 0 and math.isnan(byid[q.warm_of].done):
                    break  # continues a request that has not finished yet
                queue.popleft()
                self._alloc(q)
                admitted.append(q)
            # launch a batch on a free stream
            if admitted and free:
                batch, admitted = admitted[: self.max_batch], admitted[self.max_batch:]
                st = free.pop()
                inflight.append(self._launch(batch, st, byid))
            # completions
            still = []
            for item in inflight:
                st, ev, batch, hu, stage = item
                if ev.query():
                    tdone = time.perf_counter() - t0
                    off = 0
                    for q in batch:
                        mt = q.T * self.pool.models[q.n][0].m
                        q.u = hu[off: off + mt].numpy().reshape(q.T, -1).copy()
                        off += mt
                        q.done = tdone
                        done += 1
                        if q.warm_of >= 0:
                            prior = byid[q.warm_of]
                            prior.refs -= 1
                            self._release(prior)
                        self._release(q)  # kept while warm requests still need it
                    free.append(st)
                else:
                    still.append(item)
            inflight = still
            if not inflight and not admitted and queue and realtime:
                wait = queue[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        torch.cuda.synchronize()
        lat = np.array([q.done - q.arrival for q in reqs])
        span = max(q.done for q in reqs) - min(q.arrival for q in reqs)
        return lat, {"requests": len(reqs), "solves_per_s": len(reqs) / span,
                     "p50_ms": float(np.percentile(lat, 50) * 1e3),
                     "p99_ms": float(np.percentile(lat, 99) * 1e3),
                     "mean_ms": float(lat.mean() * 1e3), "peak_device_bytes": self.peak_mem,
                     "time_steps": int(sum(q.T for q in reqs)),
                     "warm_requests": int(sum(q.warm_of >= 0 for q in reqs))}

    def _launch(self, batch: List[Request], st, byid):
        import torch

        # one host-to-device copy of every reference (r_0..r_T) and cold x_0
        sizes = [q.r.size + (q.n if q.warm_of < 0 else 0) for q in batch]
        total = int(sum(sizes))
        host = torch.empty(total, dtype=torch.float32).pin_memory()
        hv = host.numpy()
        off = 0
        for q, sz in zip(batch, sizes):
            hv[off: off + q.r.size] = q.r.ravel()
            if q.warm_of < 0:
                hv[off + q.r.size: off + sz] = q.x0
            off += sz
        with torch.cuda.stream(st):
            dev = host.to("cuda", non_blocking=True)
            probs, outs = [], []
            off = 0
            for q, sz in zip(batch, sizes):
                n = q.n
                p = self.pool.models[n][0].p
                rptr = dev.data_ptr() + off * 4
                rT = rptr + q.T * p * 4
                if q.warm_of < 0:
                    x0 = dev.data_ptr() + (off + q.r.size) * 4
                else:
                    prior = byid[q.warm_of]
                    x0 = prior.out["x"].data_ptr() + q.shift * n * 4
                probs.append(self.pool.problem(n, q.offset, q.T, rptr, x0, rT))
                outs.append(q.out)
                off += sz
            ws = torch.empty(lqt.lqt_batch_workspace_bytes(len(batch)), dtype=torch.uint8,
                             device="cuda")
            lqt.lqt_solve_batched(probs, outs, ws, st)
            ucat = torch.cat([q.out["u"].reshape(-1) for q in batch])
            hu = torch.empty(ucat.numel(), dtype=torch.float32).pin_memory()
            hu.copy_(ucat, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return (st, ev, batch, hu, (host, dev, ws))
