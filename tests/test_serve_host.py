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
