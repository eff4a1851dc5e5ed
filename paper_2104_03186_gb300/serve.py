"""Continuous-batching LQT solver service on one GPU.

Requests are MPC-style solves: a horizon T over a model that is resident on
the device (a window into a time-varying model of state size n), plus the
request's own reference trajectory r and initial state x_0.  A "warm" request
continues a previous one: it reuses the previous request's model shifted by s
steps (a receding horizon) and starts from that request's device-resident
predicted state x*_s.

The loop admits arrived requests while their device memory fits the budget
(the outputs of finished requests that warm requests will still read count
too; with nothing admitted or in flight the next request is admitted even
over the budget, so that the stream always moves and those outputs are
eventually released), groups whatever has been admitted into a batch as soon
as a stream is free,
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
    m: int = 0              # control size of the request's model
    nbytes: int = 0         # out_bytes(n, m, T)
    xoff: int = 0           # element offset of x* in the request's outputs
    out_ptr: int = 0        # device address of out


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


def pack_inputs(batch: List[Request], out: np.ndarray) -> np.ndarray:
    """Pack the batch's references and cold initial states into `out` (the
    host side of the batch's one host-to-device copy), per request r_0 .. r_T
    then x_0 if the request is cold; returns each request's first element."""
    parts = []
    for q in batch:
        parts.append(q.r.reshape(-1))
        if q.warm_of < 0:
            parts.append(q.x0)
    sizes = np.fromiter((a.size for a in parts), np.int64, len(parts))
    starts = np.zeros(len(parts) + 1, np.int64)
    np.cumsum(sizes, out=starts[1:])
    np.concatenate(parts, out=out[: starts[-1]])
    nparts = np.fromiter((1 + (q.warm_of < 0) for q in batch), np.int64, len(batch))
    first = np.zeros(len(batch), np.int64)
    np.cumsum(nparts[:-1], out=first[1:])
    return starts[first]


class _Arena:
    """Device blocks for request outputs, by size class.

    A request's block is its element count rounded up to one of eight classes
    per power of two (at most 12.5% more), taken from that class's free list
    when one is there, else allocated.  A released block goes back to its
    list.  torch.empty on the device costs about 10 us of host time per call
    (a quarter of the serving loop's host time at 50 000 requests/s, under a
    profiler); a list pop is a fraction of a microsecond.  The free lists are dropped whenever a new
    block would take the blocks in use plus those cached over `budget`."""

    def __init__(self, budget: int, device: str = "cuda"):
        self.budget = budget
        self.device = device
        self.free: Dict[int, List[object]] = {}
        self.cached = 0  # bytes in the free lists

    @staticmethod
    def size_class(nbytes: int) -> int:
        """Elements of the block that holds `nbytes` bytes of float32."""
        e = max(8, -(-nbytes // 4))
        step = 1 << max(0, e.bit_length() - 4)
        return -(-e // step) * step

    def take(self, nbytes: int, in_use: int):
        """A block for `nbytes` bytes: (tensor, bytes it holds)."""
        import torch

        cls = self.size_class(nbytes)
        lst = self.free.get(cls)
        if lst:
            self.cached -= 4 * cls
            return lst.pop(), 4 * cls
        if self.cached and in_use + self.cached + 4 * cls > self.budget:
            self.free.clear()
            self.cached = 0
        return torch.empty(cls, dtype=torch.float32, device=self.device), 4 * cls

    def give(self, block):
        """Return a block taken from take()."""
        self.free.setdefault(block.numel(), []).append(block)
        self.cached += 4 * block.numel()


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


_MODEL_FIELDS = ("F", "L", "U", "H", "X", "HT", "XT")


class Server:
    def __init__(self, pool: ModelPool, memory_budget: int = 4 << 30, streams: int = 8,
                 max_batch: int = 256, keep_results: bool = False, reuse_warm: bool = True):
        # streams, max_batch: up to `streams` batches in flight, of at most
        # `max_batch` requests each.  Larger batches lengthen every link of a
        # warm request's wait on its predecessor's batch: against 4 streams of
        # up to 1024 requests, 8 of up to 256 took p50 from 2.8 to 2.4 ms at
        # 10 000 requests/s and from 8.9-10.0 to 7.6-8.2 ms at 50 000/s, and
        # left 2 000/s unchanged.
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
        self.mem = 0          # bytes of the output blocks in use
        self.peak_mem = 0
        self.batches = 0
        # per batch, the state sizes of its cold requests plus those of its
        # reused warm ones: each runs as one pipeline (one launch at n = 4, one
        # chunked pipeline at n >= 8)
        self.launches = 0
        self.arena = _Arena(memory_budget)
        # per state size: m and the device addresses of the model's arrays
        self.model_ptrs = {n: (pr.m, {f: dev[f].data_ptr() for f in _MODEL_FIELDS})
                           for n, (pr, dev) in pool.models.items()}

    def _reused(self, req: Request) -> bool:
        """Solved from its owner's S and K (its own S and K regions unused)."""
        return req.reused

    def _alloc(self, req: Request):
        req.out, held = self.arena.take(req.nbytes, self.mem)
        req.out_ptr = req.out.data_ptr()
        self.mem += held
        self.peak_mem = max(self.peak_mem, self.mem)

    def _release(self, req: Request):
        """Free a finished request's outputs once no warm request still needs them."""
        if req.out is not None and req.refs == 0 and not math.isnan(req.done):
            self.mem -= 4 * req.out.numel()
            self.arena.give(req.out)
            req.out = None

    def _results(self, q: Request, byid) -> Dict[str, np.ndarray]:
        """Host copies of a completed request's S, v, K, x* (u* is q.u)."""
        n, T = q.n, q.T
        m = self.pool.models[n][0].m
        # copies (a block goes back to the arena once released)
        res = unpack_outputs(q.out[: q.nbytes // 4].to("cpu", copy=True).numpy(), n, m, T)
        if self._reused(q):
            own = byid[q.owner]
            full = unpack_outputs(own.out[: own.nbytes // 4].to("cpu", copy=True).numpy(),
                                  n, m, own.T)
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
            q.m = self.model_ptrs[q.n][0]
            q.nbytes = out_bytes(q.n, q.m, q.T)
            q.xoff = (q.T + 1) * q.n * q.n + (q.T + 1) * q.n + q.T * q.m * q.n
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
                need = 4 * _Arena.size_class(q.nbytes)
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
                # one copy out of the stream's staging buffer per batch; each
                # request's u* is a view of it
                hu = slot.h_u_np[: uoff[-1]].copy()
                for q, off in zip(batch, uoff):
                    q.u = hu[off: off + q.T * q.m].reshape(q.T, q.m)
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
                     "batches": self.batches, "mean_batch": len(reqs) / max(self.batches, 1),
                     "size_groups": self.launches}

    def _launch(self, batch: List[Request], slot: _Slot, byid):
        import torch

        k = len(batch)
        u_sizes = np.fromiter((q.T * q.m for q in batch), np.int64, k)
        u_off = np.zeros(k + 1, np.int64)
        np.cumsum(u_sizes, out=u_off[1:])
        n_in = sum(q.r.size + (q.n if q.warm_of < 0 else 0) for q in batch)
        slot.ensure(n_in, int(u_off[-1]), k)
        in_off = pack_inputs(batch, slot.h_in_np)
        din = slot.d_in.data_ptr()
        dup = slot.d_u.data_ptr()
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
        cold = [i for i, q in enumerate(batch) if not q.reused]
        warm = [i for i, q in enumerate(batch) if q.reused]
        st = slot.stream
        with torch.cuda.stream(st):
            slot.d_in[:n_in].copy_(slot.h_in[:n_in], non_blocking=True)
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
        return (slot, ev, batch, u_off.tolist())

    def _items(self, it, reqs: List[Request], in_off, u_off, din: int, dup: int, byid):
        """Descriptors of `reqs` in the BATCH_ITEM array `it`, column by column:
        model windows from the pool, references and cold initial states from
        the packed input copy (request i's r_0 at element in_off[i], its x_0
        after r_T), warm initial states from the predecessor's x*, outputs in
        each request's buffer (S and K of a reused warm request in its
        owner's), u* in the stream's staging buffer at element u_off[i].
        Addresses are computed as int64 (device addresses are below 2^63)."""
        k = len(reqs)
        i64 = np.int64
        ns = np.fromiter((q.n for q in reqs), i64, k)
        ms = np.fromiter((q.m for q in reqs), i64, k)
        Ts = np.fromiter((q.T for q in reqs), i64, k)
        offs = np.fromiter((q.offset for q in reqs), i64, k)
        in_off = np.asarray(in_off, i64)
        # x_0: after r_T in the packed copy (cold), else the predecessor's x*_s
        cold = np.fromiter((q.warm_of < 0 for q in reqs), bool, k)
        wx = np.fromiter((0 if q.warm_of < 0 else
                          byid[q.warm_of].out_ptr + 4 * (byid[q.warm_of].xoff + q.shift * q.n)
                          for q in reqs), i64, k)
        rp = din + 4 * in_off
        x0p = np.where(cold, rp + 4 * (Ts + 1) * ns, wx)
        base = {f: np.empty(k, i64) for f in _MODEL_FIELDS}
        for n, (m, ptrs) in self.model_ptrs.items():
            sel = ns == n
            if sel.any():
                for f in base:
                    base[f][sel] = ptrs[f]
        P, S = it["problem"], it["solution"]
        P["n"], P["m"], P["p"], P["pT"], P["T"], P["dtype"] = ns, ms, ns, ns, Ts, lqt.LQT_F32
        P["F"]["ptr"], P["F"]["step_stride"] = base["F"] + 4 * offs * ns * ns, ns * ns
        P["L"]["ptr"], P["L"]["step_stride"] = base["L"] + 4 * offs * ns * ms, ns * ms
        P["X"]["ptr"], P["X"]["step_stride"] = base["X"] + 4 * offs * ns * ns, ns * ns
        P["U"]["ptr"], P["U"]["step_stride"] = base["U"], 0
        P["H"]["ptr"], P["H"]["step_stride"] = base["H"], 0
        P["c"]["ptr"], P["c"]["step_stride"] = 0, 0
        P["r"]["ptr"], P["r"]["step_stride"] = rp, ns
        P["HT"], P["XT"] = base["HT"], base["XT"]
        P["rT"] = rp + 4 * Ts * ns
        P["x0"] = x0p
        # outputs, packed S | v | K | x per request; S and K of a reused warm
        # request are its owner's from step skoff on (owner = itself, skoff =
        # 0, for every other request)
        own = [byid[q.owner] for q in reqs]
        optr = np.fromiter((o.out_ptr for o in own), i64, k)
        To = np.fromiter((o.T for o in own), i64, k)
        sk = np.fromiter((q.skoff for q in reqs), i64, k)
        outp = np.fromiter((q.out_ptr for q in reqs), i64, k)
        S["S"] = optr + 4 * sk * ns * ns
        S["K"] = optr + 4 * ((To + 1) * ns * ns + (To + 1) * ns + sk * ns * ms)
        S["v"] = outp + 4 * (Ts + 1) * ns * ns
        S["x"] = outp + 4 * ((Ts + 1) * ns * ns + (Ts + 1) * ns + Ts * ns * ms)
        S["u"] = dup + 4 * np.asarray(u_off, i64)
        return it
