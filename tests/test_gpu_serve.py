"""The continuous-batching service: every request of a mixed Poisson stream
(n in {4, 8, 16, 32}, cold and warm requests, several batches in flight) gives
the same result as the same request solved alone, and warm requests start from
their predecessor's predicted state."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_results_alone_equal_results_in_the_mix():
    import torch

    from paper_2104_03186_gb300 import lqt, serve

    pool = serve.ModelPool((4, 8, 16, 32), steps=1024, seed=3)
    reqs = serve.make_requests(120, rate=20000.0, seed=5, t_lo=16, t_hi=512, pool_steps=1024)
    srv = serve.Server(pool, memory_budget=256 << 20, streams=3, max_batch=16)
    lat, summary = srv.run(reqs)
    assert summary["requests"] == 120 and np.all(np.isfinite(lat)) and np.all(lat >= 0)
    assert summary["warm_requests"] > 0
    byid = {q.rid: q for q in reqs}
    # each request again, alone in its own batch, with the same inputs
    for q in reqs[:60]:
        n = q.n
        r_dev = torch.from_numpy(q.r).cuda()
        if q.warm_of < 0:
            x0 = torch.from_numpy(q.x0).cuda()
        else:
            # the predecessor's predicted state, recomputed alone
            prior = byid[q.warm_of]
            x0 = torch.from_numpy(prior.alone_x[q.shift].copy()).cuda()
        P = pool.problem(n, q.offset, q.T, r_dev.data_ptr(), x0.data_ptr(),
                         r_dev.data_ptr() + q.T * pool.models[n][0].p * 4)
        out = lqt.solve_batched([P])[0]
        q.alone_x = out["x"].cpu().numpy()
        u = out["u"].cpu().numpy()
        assert np.array_equal(u, q.u), q.rid


def test_admission_respects_memory_budget():
    from paper_2104_03186_gb300 import serve

    pool = serve.ModelPool((4, 16), steps=1024, seed=1)
    reqs = serve.make_requests(60, rate=50000.0, seed=2, sizes=(4, 16), t_lo=16, t_hi=512,
                               pool_steps=1024)
    budget = 4 << 20
    srv = serve.Server(pool, memory_budget=budget, streams=2, max_batch=8)
    _, summary = srv.run(reqs)
    biggest = max(serve.out_bytes(q.n, q.n // 2, q.T) for q in reqs)
    assert summary["peak_device_bytes"] <= max(budget, biggest)
