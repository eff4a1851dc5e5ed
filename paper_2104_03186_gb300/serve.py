"""Continuous-batching LQT solver service on one GPU.

Requests are MPC-style solves: a horizon T over a model that is resident on
the device (a window into a time-varying model of state size n), plus the
request's own reference trajectory r and initial state x_0.  A "warm" request
continues a previous one: it reuses the previous request's model shifted by s
steps (a receding horizon) and starts from that request's device-resident
predicted state x*_s.

The loop admits arrived requests while their device memory fits the budget,
groups whatever has been admitted into a batch as soon as a stream is free,
and solves the batch's cold requests with one lqt_solve_batched call (per
state size present, one persistent launch for n = 4 and one chunked pipeline
for n >= 8).  A warm request's S_k and K_k are those of the request it
continues, shifted by s steps (same model, same terminal weights; they do not
depend on the reference or the initial state).  With reuse_warm (the
default), the warm requests of a state size n >= 8 that has no full solve in
the batch go to one lqt_solve_warm call, on a second stream beside the full
solves: it reads S and K in place from the device-resident outputs of the
request that computed them and computes only v, x* and u*.  (Where a size has
full solves anyway, its warm requests join them: a second pipeline of
launches would cost more host time than it saves on the device.)  Batches on
different streams run concurrently, so
requests that arrive while others are on the GPU start without waiting for
them.  Per batch the references and initial states go up in one host-to-device
copy and the optimal controls u* come back in one device-to-host copy.
Latency is completion (observed by polling the batch's event) minus arrival.
"""
from __future__ import annotations

import dataclasses
import gc
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
    result: Optional[Dict[str, np.ndarray]] = None  # S, v, K, x, u (keep_results only)
    refs: int = 0           # warm requests still pointing at this one's outputs
    owner: int = -1         # request whose outputs hold this one's S_k, K_k
    skoff: int = 0          # step of this request's S_0, K_0 in the owner's arrays
    reused: bool = False    # solved from the owner's S, K (lqt_solve_warm)
    holds: Optional[List[int]] = None  # requests whose outputs this one may read


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


def unpack_outputs(buf: np.ndarray, n: int, m: int, T: int) -> Dict[str, np.ndarray]:
    """Split a request's packed output buffer (S, v, K, x, as written by the
    solve) into arrays with the time step on the first axis."""
    sizes = ((T + 1) * n * n, (T + 1) * n, T * m * n, (T + 1) * n)
    shapes = ((T + 1, n, n), (T + 1, n), (T, m, n), (T + 1, n))
    out, a = {}, 0
    for name, size, shape in zip(("S", "v", "K", "x"), sizes, shapes):
        out[name] = buf[a: a + size].reshape(shape)
        a += size
    return out


def out_bytes(n: int, m: int, T: int) -> int:
    """Device bytes a request holds while admitted: S, v, K and x (its u goes to
    the stream's staging buffer)."""
    return 4 * ((T + 1) * n * n + (T + 1) * n + T * m * n + (T + 1) * n)



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


class _Slot:
    """One stream with its staging buffers, reused batch after batch: pinned
    host and device buffers for the packed references and initial states, a
    device buffer the kernels write u* into, its pinned host copy, the batch
    workspace and the descriptor array."""

    def __init__(self):
        import torch

        self.stream = torch.cuda.Stream()
        self.warm_stream = torch.cuda.Stream()  # the batch's warm solves, beside the cold ones
        self.cap_in = self.cap_u = self.cap_items = 0
        self.ensure(1 << 22, 1 << 21, 1024)

    def ensure(self, in_elems: int, u_elems: int, count: int):
        import torch

        if in_elems > self.cap_in:
            self.cap_in = max(in_elems, 2 * self.cap_in)
            self.h_in = torch.empty(self.cap_in, dtype=torch.float32).pin_memory()
            self.d_in = torch.empty(self.cap_in, dtype=torch.float32, device="cuda")
            self.h_in_np = self.h_in.numpy()
        if u_elems > self.cap_u:
            self.cap_u = max(u_elems, 2 * self.cap_u)
            self.h_u = torch.empty(self.cap_u, dtype=torch.float32).pin_memory()
            self.d_u = torch.empty(self.cap_u, dtype=torch.float32, device="cuda")
            self.h_u_np = self.h_u.numpy()
        if count > self.cap_items:
            self.cap_items = max(count, 2 * self.cap_items)
            self.items = np.zeros(self.cap_items, dtype=lqt.BATCH_ITEM)
        if not hasattr(self, "ws"):
            self.ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")

    def ensure_ws(self, nbytes: int, warm: bool = False):
        """The batch workspace (or, warm=True, the warm solves' own one: both
        run on the stream one after the other, each with its status word)."""
        import torch

        name = "ws_warm" if warm else "ws"
        cur = getattr(self, name, None)
        if cur is None or nbytes > cur.numel():
            size = max(nbytes, 2 * cur.numel() if cur is not None else 1 << 20)
            setattr(self, name, torch.empty(size, dtype=torch.uint8, device="cuda"))


class Server:
    def __init__(self, pool: ModelPool, memory_budget: int = 4 << 30, streams: int = 4,
                 max_batch: int = 1024, keep_results: bool = False, reuse_warm: bool = True):
        self.pool = pool
        # reuse_warm: warm requests take S_k, K_k from the request that computed
        # them (lqt_solve_warm); off, they are solved in full like cold ones
        self.reuse_warm = reuse_warm
        # keep_results: copy every request's S, v, K, x* and u* to the host as it
        # completes (Request.result), before its device outputs are released
        self.keep_results = keep_results
        self.budget = memory_budget
        self.slots = [_Slot() for _ in range(streams)]
        self.max_batch = max_batch
        self.mem = 0
        self.peak_mem = 0
        self.batches = 0
        self.launches = 0

    def _reused(self, req: Request) -> bool:
        """Solved from its owner's S and K (its own S and K regions unused)."""
        return req.reused

    def _bytes(self, req: Request) -> int:
        return out_bytes(req.n, self.pool.models[req.n][0].m, req.T)

    def _x_offset(self, req: Request) -> int:
        """Element offset of x in the request's own buffer."""
        n, T = req.n, req.T
        m = self.pool.models[n][0].m
        return (T + 1) * n * n + (T + 1) * n + T * m * n

    def _alloc(self, req: Request):
        import torch

        nb = self._bytes(req)
        req.out = torch.empty(nb // 4, dtype=torch.float32, device="cuda")
        self.mem += nb
        self.peak_mem = max(self.peak_mem, self.mem)

    def _release(self, req: Request):
        """Free a finished request's outputs once no warm request still needs them."""
        if req.out is not None and req.refs == 0 and not math.isnan(req.done):
            self.mem -= self._bytes(req)
            req.out = None

    def _results(self, q: Request, byid) -> Dict[str, np.ndarray]:
        """Host copies of a completed request's S, v, K, x* (u* is q.u)."""
        n, T = q.n, q.T
        m = self.pool.models[n][0].m
        res = unpack_outputs(q.out.cpu().numpy(), n, m, T)
        if self._reused(q):
            own = byid[q.owner]
            full = unpack_outputs(own.out.cpu().numpy(), n, m, own.T)
            res["S"] = full["S"][q.skoff: q.skoff + T + 1].copy()
            res["K"] = full["K"][q.skoff: q.skoff + T].copy()
        return res

    def run(self, reqs: List[Request], realtime: bool = True):
        """Serve the stream; returns per-request latencies (s) and summary.

        Python's cyclic garbage collector is paused for the run: one collection
        before the stream starts, the survivors frozen, then no automatic pass
        until the run ends.  A generation-2 pass over the request set and the
        model pool took 30-40 ms of the host loop (measured inside a batch
        launch), which every request that arrived meanwhile waited out."""
        gc_enabled = gc.isenabled()
        gc.collect()
        gc.freeze()
        gc.disable()
        try:
            return self._run(reqs, realtime)
        finally:
            gc.unfreeze()
            if gc_enabled:
                gc.enable()

    def _run(self, reqs: List[Request], realtime: bool):
        import torch

        byid = {r.rid: r for r in reqs}
        for q in reqs:
            q.refs, q.reused, q.owner, q.skoff, q.holds = 0, False, q.rid, 0, []
        # warm requests keep the outputs they may read: the predecessor's x*_s
        # and, when reusing, S_k and K_k, which sit with the first ancestor that
        # was solved in full (up the chain of warm requests to a cold one)
        for q in reqs:
            a = q.warm_of
            while a >= 0:
                byid[a].refs += 1
                q.holds.append(a)
                if not self.reuse_warm:
                    break
                a = byid[a].warm_of
        queue = deque(sorted(reqs, key=lambda r: r.arrival))
        ready: deque = deque()    # warm requests whose predecessor has finished
        parked: Dict[int, List[Request]] = {}  # predecessor rid -> warm requests
        admitted: List[Request] = []
        inflight = []  # (slot, event, batch, u offsets)
        free = list(self.slots)
        done = 0
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0 if realtime else math.inf
            # admission by device-memory budget, first come first served; a warm
            # request waits (parked) until the request it continues has finished
            blocked = False
            while not blocked and (ready or (queue and queue[0].arrival <= now)):
                src = ready if ready else queue
                q = src[0]
                if q.warm_of >= 0 and math.isnan(byid[q.warm_of].done):
                    src.popleft()
                    parked.setdefault(q.warm_of, []).append(q)
                    continue
                need = self._bytes(q)
                if self.mem + need > self.budget and (admitted or inflight):
                    blocked = True
                    break
                src.popleft()
                self._alloc(q)
                admitted.append(q)
            # launch a batch on a free stream
            if admitted and free:
                batch, admitted = admitted[: self.max_batch], admitted[self.max_batch:]
                inflight.append(self._launch(batch, free.pop(), byid))
            # completions
            still = []
            for item in inflight:
                slot, ev, batch, uoff = item
                if not ev.query():
                    still.append(item)
                    continue
                tdone = time.perf_counter() - t0
                hu = slot.h_u_np
                for q, off in zip(batch, uoff):
                    mt = q.T * self.pool.models[q.n][0].m
                    q.u = hu[off: off + mt].reshape(q.T, -1).copy()
                    q.done = tdone
                    if self.keep_results:
                        q.result = self._results(q, byid)
                        q.result["u"] = q.u
                    done += 1
                    for a in q.holds:
                        byid[a].refs -= 1
                        self._release(byid[a])
                    self._release(q)  # kept while warm requests still need it
                    if q.rid in parked:
                        ready.extend(parked.pop(q.rid))
                free.append(slot)
            inflight = still
            if not inflight and not admitted and not ready and queue and realtime:
                wait = queue[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-4))
        torch.cuda.synchronize()
        lat = np.array([q.done - q.arrival for q in reqs])
        span = max(q.done for q in reqs) - min(q.arrival for q in reqs)
        warm = np.array([q.warm_of >= 0 for q in reqs])

        def pct(sel, p):
            return float(np.percentile(lat[sel], p) * 1e3) if sel.any() else None

        return lat, {"requests": len(reqs), "solves_per_s": len(reqs) / span,
                     "p50_ms": float(np.percentile(lat, 50) * 1e3),
                     "p99_ms": float(np.percentile(lat, 99) * 1e3),
                     "cold_p50_ms": pct(~warm, 50), "cold_p99_ms": pct(~warm, 99),
                     "warm_p50_ms": pct(warm, 50), "warm_p99_ms": pct(warm, 99),
                     "mean_ms": float(lat.mean() * 1e3), "peak_device_bytes": self.peak_mem,
                     "time_steps": int(sum(q.T for q in reqs)),
                     "warm_requests": int(sum(q.warm_of >= 0 for q in reqs)),
                     "warm_reused": int(sum(self._reused(q) for q in reqs)),
                     "batches": self.batches, "mean_batch": len(reqs) / max(self.batches, 1)}

    def _launch(self, batch: List[Request], slot: _Slot, byid):
        import torch

        pool = self.pool
        k = len(batch)
        # packed layout of the host-to-device copy: per request r_0..r_T then x_0 (cold)
        in_sizes = [q.r.size + (q.n if q.warm_of < 0 else 0) for q in batch]
        u_sizes = [q.T * pool.models[q.n][0].m for q in batch]
        in_off = np.concatenate([[0], np.cumsum(in_sizes)]).astype(np.int64)
        u_off = np.concatenate([[0], np.cumsum(u_sizes)]).astype(np.int64)
        slot.ensure(int(in_off[-1]), int(u_off[-1]), k)
        hv = slot.h_in_np
        for q, a in zip(batch, in_off[:-1]):
            a = int(a)
            hv[a: a + q.r.size] = q.r.ravel()
            if q.warm_of < 0:
                hv[a + q.r.size: a + q.r.size + q.n] = q.x0
        din = np.uint64(slot.d_in.data_ptr())
        dup = np.uint64(slot.d_u.data_ptr())
        # A warm request is solved from its owner's S and K when its state size
        # has no request of the batch that needs a full solve anyway, and
        # n >= 8: the full solves of a size share their launches, so adding a
        # separate warm pipeline beside them would add launches (host time) for
        # little device time, and at n = 4 the full solve is one launch.
        full_sizes = {q.n for q in batch if q.warm_of < 0 or not self.reuse_warm or q.n < 8}
        for q in batch:
            q.reused = False
            if q.warm_of >= 0 and self.reuse_warm and q.n not in full_sizes:
                prior = byid[q.warm_of]
                q.reused = True
                if prior.reused:
                    q.owner, q.skoff = prior.owner, prior.skoff + q.shift
                else:
                    q.owner, q.skoff = prior.rid, q.shift
        cold = [i for i, q in enumerate(batch) if not self._reused(q)]
        warm = [i for i, q in enumerate(batch) if self._reused(q)]
        st = slot.stream
        with torch.cuda.stream(st):
            slot.d_in[: int(in_off[-1])].copy_(slot.h_in[: int(in_off[-1])], non_blocking=True)
            if warm:
                # the warm solves run on the slot's second stream, concurrently
                # with the cold ones, after the input copy; joined before u*
                # goes back
                fork = torch.cuda.Event()
                fork.record(st)
                slot.warm_stream.wait_event(fork)
                it = self._items(slot.items[len(cold): k], [batch[i] for i in warm],
                                 in_off[warm], u_off[warm], din, dup, byid)
                nbytes = lqt.lqt_warm_workspace_bytes_array(it)
                if nbytes == 0:
                    raise lqt.LQTError(lqt.LQT_EUNSUPPORTED, "warm workspace")
                slot.ensure_ws(nbytes, warm=True)
                lqt.lqt_solve_warm_array(it, slot.ws_warm, slot.warm_stream)
                join = torch.cuda.Event()
                join.record(slot.warm_stream)
            if cold:
                it = self._items(slot.items[: len(cold)], [batch[i] for i in cold],
                                 in_off[cold], u_off[cold], din, dup, byid)
                nbytes = lqt.lqt_batch_workspace_bytes_array(it)
                if nbytes == 0:
                    raise lqt.LQTError(lqt.LQT_EUNSUPPORTED, "batch workspace")
                slot.ensure_ws(nbytes)
                lqt.lqt_solve_batched_array(it, slot.ws, st)
            if warm:
                st.wait_event(join)
            nu_el = int(u_off[-1])
            slot.h_u[:nu_el].copy_(slot.d_u[:nu_el], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.batches += 1
        ns = [q.n for q in batch]
        self.launches += len(set(ns[i] for i in cold)) + len(set(ns[i] for i in warm))
        return (slot, ev, batch, [int(a) for a in u_off[:-1]])

    def _items(self, it, reqs: List[Request], in_off, u_off, din, dup, byid):
        """Descriptors of `reqs` in the BATCH_ITEM array `it`, column by column:
        model windows from the pool, references and cold initial states from
        the packed input copy, warm initial states from the predecessor's x*,
        outputs in each request's buffer (S and K of a reused warm request in
        its owner's), u* in the stream's staging buffer."""
        pool = self.pool
        k = len(reqs)
        ns = np.fromiter((q.n for q in reqs), np.int64, k)
        Ts = np.fromiter((q.T for q in reqs), np.int64, k)
        offs = np.fromiter((q.offset for q in reqs), np.int64, k)
        x0p = np.empty(k, np.uint64)
        for i, q in enumerate(reqs):
            if q.warm_of < 0:
                x0p[i] = din + np.uint64(4 * (int(in_off[i]) + q.r.size))
            else:
                prior = byid[q.warm_of]
                x0p[i] = np.uint64(prior.out.data_ptr() +
                                   4 * (self._x_offset(prior) + q.shift * q.n))
        ms = np.empty(k, np.int64)
        base = {f: np.empty(k, np.uint64) for f in ("F", "L", "U", "H", "X", "HT", "XT")}
        for n, (pr, dev) in pool.models.items():
            sel = ns == n
            if not sel.any():
                continue
            ms[sel] = pr.m
            for f in base:
                base[f][sel] = dev[f].data_ptr()
        P, S = it["problem"], it["solution"]
        P["n"], P["m"], P["p"], P["pT"], P["T"], P["dtype"] = ns, ms, ns, ns, Ts, lqt.LQT_F32
        n2 = (ns * ns).astype(np.uint64)
        nm = (ns * ms).astype(np.uint64)
        o = offs.astype(np.uint64)
        P["F"]["ptr"], P["F"]["step_stride"] = base["F"] + o * n2 * np.uint64(4), ns * ns
        P["L"]["ptr"], P["L"]["step_stride"] = base["L"] + o * nm * np.uint64(4), ns * ms
        P["X"]["ptr"], P["X"]["step_stride"] = base["X"] + o * n2 * np.uint64(4), ns * ns
        P["U"]["ptr"], P["U"]["step_stride"] = base["U"], 0
        P["H"]["ptr"], P["H"]["step_stride"] = base["H"], 0
        P["c"]["ptr"], P["c"]["step_stride"] = 0, 0
        rp = din + np.asarray(in_off, np.int64).astype(np.uint64) * np.uint64(4)
        P["r"]["ptr"], P["r"]["step_stride"] = rp, ns
        P["HT"], P["XT"] = base["HT"], base["XT"]
        P["rT"] = rp + Ts.astype(np.uint64) * ns.astype(np.uint64) * np.uint64(4)
        P["x0"] = x0p
        Tu, nu = Ts.astype(np.uint64), ns.astype(np.uint64)
        for i, q in enumerate(reqs):
            outp = np.uint64(q.out.data_ptr())
            if self._reused(q):
                own = byid[q.owner]
                obase = np.uint64(own.out.data_ptr())
                To = np.uint64(own.T)
                S["S"][i] = obase + np.uint64(4 * q.skoff * q.n * q.n)
                S["K"][i] = obase + np.uint64(4) * ((To + np.uint64(1)) * nu[i] * nu[i] +
                                                    (To + np.uint64(1)) * nu[i]) + \
                    np.uint64(4 * q.skoff * int(nm[i]))
                S["v"][i] = outp + np.uint64(4) * (Tu[i] + np.uint64(1)) * nu[i] * nu[i]
                S["x"][i] = outp + np.uint64(4 * self._x_offset(q))
            else:
                S["S"][i] = outp
                S["v"][i] = outp + np.uint64(4) * (Tu[i] + np.uint64(1)) * nu[i] * nu[i]
                S["K"][i] = S["v"][i] + np.uint64(4) * (Tu[i] + np.uint64(1)) * nu[i]
                S["x"][i] = S["K"][i] + np.uint64(4) * Tu[i] * nm[i]
        S["u"] = dup + np.asarray(u_off, np.int64).astype(np.uint64) * np.uint64(4)
        return it
