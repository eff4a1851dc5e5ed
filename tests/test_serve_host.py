"""Host logic of the serving loop (no GPU): the request stream of the serving
workload and the packing of a request's outputs.

The stream is a Poisson process with n uniform over the sizes, T log-uniform,
and a fraction of warm requests that continue the previous request of the same
size over a horizon shifted by s in [1, T/4] (a receding horizon over the same
model window).  These checks pin the generator's statistics and the invariants
the server relies on: a warm request's window ends where its predecessor's
does, so the predecessor's S and K cover it step for step."""
import math

import numpy as np
import pytest

from paper_2104_03186_gb300 import serve


@pytest.fixture(scope="module")
def stream():
    return serve.make_requests(20000, rate=5000.0, seed=3)


def test_arrivals_are_a_poisson_stream(stream):
    t = np.array([q.arrival for q in stream])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * 5000.0 - 1.0) < 0.03
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    assert [q.rid for q in stream] == list(range(len(stream)))


def test_sizes_and_horizons(stream):
    ns = np.array([q.n for q in stream])
    assert set(ns.tolist()) == {4, 8, 16, 32}
    for n in (4, 8, 16, 32):
        assert abs((ns == n).mean() - 0.25) < 0.02
    cold = [q for q in stream if q.warm_of < 0]
    Ts = np.array([q.T for q in cold])
    assert Ts.min() >= 32 and Ts.max() <= 2048
    # log-uniform: log T is uniform on [ln 32, ln 2048]
    u = (np.log(Ts) - math.log(32)) / (math.log(2048) - math.log(32))
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1.0 / 12) < 0.01
    for q in stream:
        assert q.r.shape == (q.T + 1, q.n) and q.r.dtype == np.float32
        assert 0 <= q.offset and q.offset + q.T <= 4096


def test_warm_requests_continue_their_predecessor(stream):
    byid = {q.rid: q for q in stream}
    warm = [q for q in stream if q.warm_of >= 0]
    # about 30% of the requests whose size had a predecessor of at least 8 steps
    assert 0.25 < len(warm) / len(stream) < 0.32
    last = {}
    for q in stream:
        if q.warm_of >= 0:
            p = byid[q.warm_of]
            assert p.rid == last[q.n].rid  # the previous request of the same size
            assert p.n == q.n and p.arrival < q.arrival
            assert 1 <= q.shift <= max(2, p.T // 4)
            assert q.T == p.T - q.shift and q.offset == p.offset + q.shift
            # the windows end together: S_k, K_k of q are those of p at k + shift
            assert q.offset + q.T == p.offset + p.T
            assert q.x0 is None
        else:
            assert q.x0 is not None and q.x0.shape == (q.n,)
        last[q.n] = q


def test_stream_is_reproducible():
    a = serve.make_requests(500, rate=2000.0, seed=11)
    b = serve.make_requests(500, rate=2000.0, seed=11)
    assert [(q.arrival, q.n, q.T, q.offset, q.warm_of) for q in a] == \
        [(q.arrival, q.n, q.T, q.offset, q.warm_of) for q in b]
    assert all(np.array_equal(x.r, y.r) for x, y in zip(a, b))


@pytest.mark.parametrize("n,m,T", [(4, 2, 1), (8, 4, 37), (32, 16, 300)])
def test_output_packing(n, m, T):
    nbytes = serve.out_bytes(n, m, T)
    buf = np.arange(nbytes // 4, dtype=np.float32)
    out = serve.unpack_outputs(buf, n, m, T)
    assert out["S"].shape == (T + 1, n, n) and out["v"].shape == (T + 1, n)
    assert out["K"].shape == (T, m, n) and out["x"].shape == (T + 1, n)
    # the four parts tile the buffer in order, with nothing left over
    parts = np.concatenate([out[k].ravel() for k in ("S", "v", "K", "x")])
    assert np.array_equal(parts, buf)


def test_pack_inputs_layout(stream):
    batch = stream[:300]
    n_in = sum(q.r.size + (q.n if q.warm_of < 0 else 0) for q in batch)
    out = np.full(n_in + 7, np.nan, np.float32)
    in_off = serve.pack_inputs(batch, out)
    assert in_off.shape == (300,) and in_off[0] == 0
    for i, q in enumerate(batch):
        a = int(in_off[i])
        assert np.array_equal(out[a: a + q.r.size], q.r.ravel())
        end = a + q.r.size
        if q.warm_of < 0:
            assert np.array_equal(out[end: end + q.n], q.x0)
            end += q.n
        # the parts follow one another with no gap
        assert end == (int(in_off[i + 1]) if i + 1 < len(batch) else n_in)
    assert np.all(np.isnan(out[n_in:]))


def test_arena_size_classes():
    cls = [serve._Arena.size_class(b) for b in range(1, 1 << 16, 3)]
    for b, c in zip(range(1, 1 << 16, 3), cls):
        e = -(-b // 4)
        assert c >= e and c >= 8
        assert c <= max(8, e * 1.125)  # at most 12.5% over
    assert cls == sorted(cls)
    # eight classes per power of two above 64 elements
    assert len({serve._Arena.size_class(4 * e) for e in range(1025, 2049)}) == 8


def test_arena_reuses_and_bounds_its_cache():
    arena = serve._Arena(budget=1 << 20, device="cpu")
    a, ha = arena.take(4000, in_use=0)
    assert ha == 4 * a.numel() == 4 * serve._Arena.size_class(4000)
    arena.give(a)
    b, hb = arena.take(3990, in_use=0)  # same class: the same block back
    assert b is a and hb == ha and arena.cached == 0
    c, _ = arena.take(100_000, in_use=hb)
    arena.give(c)
    assert arena.cached == 4 * c.numel()
    # a new block that would take in-use + cached over the budget drops the cache
    d, hd = arena.take(1_000_000, in_use=hb)
    assert arena.cached == 0 and not arena.free
    assert hd >= 1_000_000


def _cpu_server(sizes, steps):
    """A Server with models on the host, enough to build descriptors."""
    import torch

    pool = serve.ModelPool.__new__(serve.ModelPool)
    pool.steps = steps
    pool.models = {}
    for n in sizes:
        pr = serve.inputs.diag_tracking(n, T=steps, seed=n).astype(np.float32)
        dev = {f: torch.from_numpy(getattr(pr, f)) for f in serve._MODEL_FIELDS}
        pool.models[n] = (pr, dev)
    srv = serve.Server.__new__(serve.Server)
    srv.pool, srv.reuse_warm = pool, True
    srv.model_ptrs = {n: (pr.m, {f: dev[f].data_ptr() for f in serve._MODEL_FIELDS})
                      for n, (pr, dev) in pool.models.items()}
    return srv


def test_descriptors_address_each_request(stream):
    """The batch descriptors, built array-wise, against the layout written out
    request by request: model windows, packed references and x_0, warm x_0 at
    the predecessor's x*_s, and S, K of a reused warm request in its owner's
    outputs from step skoff on."""
    from paper_2104_03186_gb300 import lqt

    sizes, steps = (4, 8, 16, 32), 4096
    srv = _cpu_server(sizes, steps)
    batch = stream[:400]
    byid = {q.rid: q for q in stream}
    base = 0x7F0000000000
    for q in stream[:400]:
        q.m = q.n // 2
        q.nbytes = serve.out_bytes(q.n, q.m, q.T)
        q.xoff = (q.T + 1) * q.n * q.n + (q.T + 1) * q.n + q.T * q.m * q.n
        q.out_ptr = base + (q.rid << 24)
        q.owner, q.skoff, q.reused = q.rid, 0, False
    # warm requests of n >= 8 whose predecessor is in the batch reuse its S, K
    for q in batch:
        if q.warm_of >= 0 and q.n >= 8 and q.warm_of in byid and byid[q.warm_of].out_ptr:
            prior = byid[q.warm_of]
            q.reused = True
            q.owner, q.skoff = ((prior.owner, prior.skoff + q.shift) if prior.reused
                                else (prior.rid, q.shift))
    assert sum(q.reused for q in batch) > 20
    din, dup = 0x7E0000000000, 0x7D0000000000
    in_off = np.cumsum([0] + [q.r.size + 7 for q in batch])[:-1]
    u_off = np.cumsum([0] + [q.T * q.m for q in batch])[:-1]
    it = srv._items(np.zeros(len(batch), lqt.BATCH_ITEM), batch, in_off, u_off, din, dup, byid)
    for i, q in enumerate(batch):
        n, m, T = q.n, q.m, q.T
        P, S = it["problem"][i], it["solution"][i]
        ptr = srv.model_ptrs[n][1]
        assert (P["n"], P["m"], P["p"], P["pT"], P["T"]) == (n, m, n, n, T)
        assert P["F"]["ptr"] == ptr["F"] + 4 * q.offset * n * n and P["F"]["step_stride"] == n * n
        assert P["L"]["ptr"] == ptr["L"] + 4 * q.offset * n * m and P["L"]["step_stride"] == n * m
        assert P["X"]["ptr"] == ptr["X"] + 4 * q.offset * n * n
        assert (P["U"]["ptr"], P["U"]["step_stride"], P["H"]["ptr"]) == (ptr["U"], 0, ptr["H"])
        assert (P["HT"], P["XT"], P["c"]["ptr"]) == (ptr["HT"], ptr["XT"], 0)
        r0 = din + 4 * int(in_off[i])
        assert P["r"]["ptr"] == r0 and P["r"]["step_stride"] == n
        assert P["rT"] == r0 + 4 * T * n
        if q.warm_of < 0:
            assert P["x0"] == r0 + 4 * (T + 1) * n
        else:
            prior = byid[q.warm_of]
            assert P["x0"] == prior.out_ptr + 4 * (prior.xoff + q.shift * n)
        v = q.out_ptr + 4 * (T + 1) * n * n
        assert S["v"] == v and S["x"] == q.out_ptr + 4 * q.xoff
        assert S["u"] == dup + 4 * int(u_off[i])
        if q.reused:
            own = byid[q.owner]
            To = own.T
            assert S["S"] == own.out_ptr + 4 * q.skoff * n * n
            assert S["K"] == own.out_ptr + 4 * ((To + 1) * n * n + (To + 1) * n) + 4 * q.skoff * n * m
        else:
            assert S["S"] == q.out_ptr
            assert S["K"] == v + 4 * (T + 1) * n


def _fview(ptr, count):
    """float32 view of host memory at a raw address (the fake solves below)."""
    import ctypes

    if count == 0:
        return np.zeros(0, np.float32)
    return np.ctypeslib.as_array((ctypes.c_float * count).from_address(int(ptr)))


def _rollout(x0, r):
    """x_0 = x0, x_{k+1} = x_k + r_k: a stand-in trajectory that depends on
    the initial state and every reference."""
    T = r.shape[0] - 1
    x = np.empty((T + 1, r.shape[1]), np.float32)
    x[0] = x0
    for k in range(T):
        x[k + 1] = x[k] + r[k]
    return x


def _fake_solve(it, warm):
    """Reads each descriptor's inputs through its addresses and writes outputs
    that identify them: S_k[0,0] = F_k[0,0] and K_k[0,0] = L_k[0,0] of the
    model window (a warm solve instead checks that the S and K it is given
    are those), x* = _rollout(x_0, r), u*_k = r_k[:m] + x*_k[:m] + K_k[0,0]."""
    for row in it:
        P, S = row["problem"], row["solution"]
        n, m, T = int(P["n"]), int(P["m"]), int(P["T"])
        F = _fview(P["F"]["ptr"], T * n * n).reshape(T, n, n)
        L = _fview(P["L"]["ptr"], T * n * m).reshape(T, n, m)
        r = _fview(P["r"]["ptr"], (T + 1) * n).reshape(T + 1, n)
        assert int(P["rT"]) == int(P["r"]["ptr"]) + 4 * T * n
        x0 = _fview(P["x0"], n).copy()
        Sk = _fview(S["S"], (T + 1) * n * n).reshape(T + 1, n, n)
        K = _fview(S["K"], T * m * n).reshape(T, m, n)
        if warm:
            assert np.array_equal(Sk[:T, 0, 0], F[:, 0, 0])
            assert np.array_equal(K[:, 0, 0], L[:, 0, 0])
        else:
            Sk[:T, 0, 0] = F[:, 0, 0]
            K[:, 0, 0] = L[:, 0, 0]
        x = _fview(S["x"], (T + 1) * n).reshape(T + 1, n)
        x[:] = _rollout(x0, r)
        _fview(S["u"], T * m).reshape(T, m)[:] = r[:T, :m] + x[:T, :m] + K[:, 0, 0][:, None]


class _FakeStream:
    def wait_event(self, ev):
        pass


class _FakeEvent:
    """Completes on its second query, so batches stay in flight a while."""

    def __init__(self):
        self.polls = 0

    def record(self, stream=None):
        pass

    def query(self):
        self.polls += 1
        return self.polls >= 2


class _FakeSlot:
    """A stream slot with its staging buffers in host memory."""

    def __init__(self):
        self.stream, self.warm_stream = _FakeStream(), _FakeStream()
        self.cap_in = self.cap_u = self.cap_items = 0
        self.ws = self.ws_warm = None
        self.ensure(1 << 12, 1 << 11, 4)

    def ensure(self, in_elems, u_elems, count):
        import torch

        from paper_2104_03186_gb300 import lqt

        if in_elems > self.cap_in:
            self.cap_in = max(in_elems, 2 * self.cap_in)
            self.h_in, self.d_in = torch.zeros(self.cap_in), torch.zeros(self.cap_in)
            self.h_in_np = self.h_in.numpy()
        if u_elems > self.cap_u:
            self.cap_u = max(u_elems, 2 * self.cap_u)
            self.h_u, self.d_u = torch.zeros(self.cap_u), torch.zeros(self.cap_u)
            self.h_u_np = self.h_u.numpy()
        if count > self.cap_items:
            self.cap_items = max(count, 2 * self.cap_items)
            self.items = np.zeros(self.cap_items, dtype=lqt.BATCH_ITEM)

    def ensure_ws(self, nbytes, warm=False):
        pass


def test_serving_loop_plumbing_on_host(monkeypatch):
    """The serving loop (admission, parking of warm requests, batching, warm
    reuse, the output arena, release of outputs) run on the host: device
    buffers and streams replaced by host ones and the solver by _fake_solve,
    which reads and writes through the descriptors' addresses.  Every
    request's u*, x* and S must be the ones its own inputs give (its model
    window, its references, its x_0 or its predecessor's x*_s), read back
    after the loop has recycled blocks for later requests."""
    import contextlib

    import torch

    from paper_2104_03186_gb300 import lqt

    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(lqt, "lqt_batch_workspace_bytes_array", lambda it: 1)
    monkeypatch.setattr(lqt, "lqt_warm_workspace_bytes_array", lambda it: 1)
    monkeypatch.setattr(lqt, "lqt_solve_batched_array", lambda it, ws, st: _fake_solve(it, False))
    monkeypatch.setattr(lqt, "lqt_solve_warm_array", lambda it, ws, st: _fake_solve(it, True))

    srv = _cpu_server((4, 8, 16, 32), 1024)
    pool = srv.pool
    budget = 6 << 20
    srv.budget, srv.max_batch, srv.keep_results = budget, 12, True
    srv.mem = srv.peak_mem = srv.batches = srv.launches = 0
    srv.slots = [_FakeSlot() for _ in range(3)]
    srv.arena = serve._Arena(budget, device="cpu")
    reqs = serve.make_requests(400, rate=1e5, seed=21, t_lo=8, t_hi=256, pool_steps=1024,
                               warm_frac=0.5)
    # the budget binds except when nothing is admitted or in flight: every
    # admission that takes the blocks in use over it must find the loop idle
    over, pending, inflight = [], [0], set()
    alloc, launch = srv._alloc, srv._launch

    def checked_alloc(q):
        before = srv.mem
        alloc(q)
        if srv.mem > budget:
            over.append(before)
            assert pending[0] == 0 and not any(ev.polls < 2 for ev in inflight)
        pending[0] += 1

    def counted_launch(batch, slot, byid):
        pending[0] -= len(batch)
        item = launch(batch, slot, byid)
        inflight.add(item[1])
        return item

    srv._alloc, srv._launch = checked_alloc, counted_launch
    _, summary = srv.run(reqs, realtime=False)

    assert summary["requests"] == 400 and summary["batches"] > 10
    # per batch, at least one size group and at most four sizes, cold and warm
    assert summary["batches"] <= summary["size_groups"] <= 8 * summary["batches"]
    assert summary["warm_reused"] > 10, summary
    assert srv.mem == 0 and all(q.out is None for q in reqs)  # every block released
    # over the budget only on top of blocks still held for warm requests
    assert all(0 < before for before in over) and len(over) < 20
    xs = {}
    for q in reqs:  # a predecessor precedes its warm successors
        pr = pool.models[q.n][0]
        x0 = q.x0 if q.warm_of < 0 else xs[q.warm_of][q.shift]
        xs[q.rid] = _rollout(x0, q.r)
        w = slice(q.offset, q.offset + q.T)
        m = pr.m
        assert np.array_equal(q.u, q.r[: q.T, :m] + xs[q.rid][: q.T, :m] + pr.L[w, 0, 0][:, None])
        assert np.array_equal(q.result["x"], xs[q.rid])
        assert np.array_equal(q.result["S"][: q.T, 0, 0], pr.F[w, 0, 0])
        assert np.array_equal(q.result["K"][:, 0, 0], pr.L[w, 0, 0])
