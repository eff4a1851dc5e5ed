"""The continuous-batching service: every request of a mixed Poisson stream
(n in {4, 8, 16, 32}, cold and warm requests, several batches in flight) gives
the same S, v, K, x* and u* as the same request solved alone, each of them
matches the FP64 oracle on the request's own inputs, and warm requests start
from their predecessor's predicted state."""
import dataclasses

import numpy as np
import pytest

from gpu_util import FP32_TOL, compare

pytestmark = pytest.mark.gpu

NAMES = ("S", "v", "K", "x", "u")


def _request_problem(pool, q, x0):
    """The request as an inputs.LQTProblem (FP64 copies of the FP32 values the
    device holds): the model window [offset, offset + T), its reference, x_0."""
    pr = pool.models[q.n][0]
    w = slice(q.offset, q.offset + q.T)
    r = q.r.astype(np.float64)
    return dataclasses.replace(
        pr.astype(np.float64), F=pr.F[w].astype(np.float64), L=pr.L[w].astype(np.float64),
        X=pr.X[w].astype(np.float64), r=r[: q.T], rT=r[q.T], x0=np.asarray(x0, np.float64),
        T=q.T)


@pytest.mark.parametrize("reuse_warm", [True, False])
def test_results_alone_equal_results_in_the_mix(reuse_warm):
    """With reuse_warm, warm requests are solved from their owner's S and K
    (lqt_solve_warm); the request alone is a full solve, so the two agree to
    rounding, not bit for bit."""
    import torch

    import oracle
    from paper_2104_03186_gb300 import lqt, serve

    pool = serve.ModelPool((4, 8, 16, 32), steps=1024, seed=3)
    reqs = serve.make_requests(120, rate=20000.0, seed=5, t_lo=16, t_hi=512, pool_steps=1024)
    srv = serve.Server(pool, memory_budget=256 << 20, streams=3, max_batch=16,
                       keep_results=True, reuse_warm=reuse_warm)
    lat, summary = srv.run(reqs)
    assert summary["requests"] == 120 and np.all(np.isfinite(lat)) and np.all(lat >= 0)
    assert summary["warm_requests"] > 0
    if reuse_warm:
        assert 0 < summary["warm_reused"] <= summary["warm_requests"], summary
    else:
        assert summary["warm_reused"] == 0
    assert summary["batches"] > 1
    byid = {q.rid: q for q in reqs}
    bitwise = 0
    for q in reqs:
        mix = q.result
        assert mix is not None, q.rid
        # the initial state the request solved from: its own x_0, or its
        # predecessor's predicted state x*_s as computed in the mix
        x0 = q.x0 if q.warm_of < 0 else byid[q.warm_of].result["x"][q.shift]
        # the same request again, alone in its own batch
        r_dev = torch.from_numpy(q.r).cuda()
        x0_dev = torch.from_numpy(np.ascontiguousarray(x0, np.float32)).cuda()
        P = pool.problem(q.n, q.offset, q.T, r_dev.data_ptr(), x0_dev.data_ptr(),
                         r_dev.data_ptr() + q.T * pool.models[q.n][0].p * 4)
        alone = {k: v.cpu().numpy() for k, v in lqt.solve_batched([P])[0].items()}
        compare({k: mix[k] for k in NAMES}, {k: alone[k].astype(np.float64) for k in NAMES},
                FP32_TOL)
        bitwise += all(np.array_equal(mix[k], alone[k]) for k in NAMES)
        # against the FP64 oracle on the request's own inputs
        ref = oracle.riccati(_request_problem(pool, q, x0), keep_kv_kc=False)
        compare({k: mix[k].astype(np.float64) for k in NAMES}, ref, FP32_TOL)
    print("requests identical bit for bit alone and in the mix: %d of %d" % (bitwise, len(reqs)))


def test_admission_respects_memory_budget():
    """The output blocks in use stay within the budget, except that with nothing
    admitted and nothing in flight the loop admits the next request anyway
    (blocks kept for warm requests may fill the budget until those run)."""
    from paper_2104_03186_gb300 import serve

    pool = serve.ModelPool((4, 16), steps=1024, seed=1)
    reqs = serve.make_requests(60, rate=50000.0, seed=2, sizes=(4, 16), t_lo=16, t_hi=512,
                               pool_steps=1024)
    budget = 4 << 20
    srv = serve.Server(pool, memory_budget=budget, streams=2, max_batch=8)
    over, pending, launched = [], [0], []
    alloc, launch = srv._alloc, srv._launch

    def checked_alloc(q):
        alloc(q)
        if srv.mem > budget:
            over.append(srv.mem)
            assert pending[0] == 0 and all(ev.query() for ev in launched)
        pending[0] += 1

    def counted_launch(batch, slot, byid):
        pending[0] -= len(batch)
        item = launch(batch, slot, byid)
        launched.append(item[1])
        return item

    srv._alloc, srv._launch = checked_alloc, counted_launch
    _, summary = srv.run(reqs)
    assert summary["requests"] == 60 and srv.mem == 0
    assert summary["peak_device_bytes"] == max([m for m in over] + [0]) or \
        summary["peak_device_bytes"] <= budget
